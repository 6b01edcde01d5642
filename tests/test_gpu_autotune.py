"""Block-shape autotuner (lsb_autotune): every candidate is timed on the same
case, rejected shapes report NaN, and the returned shape is the fastest one and
creates a working handle."""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_autotune_picks_the_fastest_valid_shape():
    from paper_2601_05936_gb300 import lsb, workloads
    case = workloads.stratified_channel(nx=128, ny=64, h=32.2, steps=10)
    cands = [(32, 8), (32, 16), (64, 4), (3, 8)]  # the last edge is not a power of two
    best, ms = lsb.autotune(case, candidates=cands, steps=5)
    assert math.isnan(ms[(3, 8, 1)])
    valid = {k: v for k, v in ms.items() if not math.isnan(v)}
    assert len(valid) == 3 and all(v > 0 for v in valid.values())
    assert best == min(valid, key=valid.get)
    g = lsb.Grid(dict(case, block=best[:2]))
    g.step(3)
    assert np.isfinite(g.get("u")).all()
    g.close()


def test_autotune_builtin_shapes_3d():
    from paper_2601_05936_gb300 import lsb, workloads
    case = workloads.rising_bubble_3d(scale=0.25)
    best, ms = lsb.autotune(case, steps=2)
    assert len(ms) == 6
    assert best in {(32, 4, 4), (32, 8, 2), (16, 8, 4), (64, 4, 2), (32, 2, 8), (16, 4, 8)}
    assert sum(not math.isnan(v) for v in ms.values()) >= 1
