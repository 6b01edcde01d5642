"""Persistent level-set driver (lsb_set_driver(g, 1)): the extension, transport
and reinitialisation passes of a finest step run as one cooperative launch with
bounded device-wide barriers between passes.  The passes are the same code as
the per-pass launches, so the state must match them exactly, with and without
CUDA-graph replay, for single cases and ensembles."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _run(cases, steps, driver, graphs=False):
    import torch

    from paper_2601_05936_gb300 import lsb
    st = torch.cuda.Stream()
    g = lsb.Grid(cases, stream=st)
    g.set_driver(driver)
    if graphs:
        g.use_graphs(True)
    g.step(steps)
    g.sync()
    out = []
    for k, c in enumerate(g.cases):
        L = int(c.get("n_levels", 1))
        out += [g.get(f, k, l) for l in range(L) for f in ("rho", "u")] + [g.get("phi", k), g.get("tag", k)]
    g.close()
    return out


def _same(a, b):
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


def test_persistent_matches_per_pass_2d_bubble_with_regrid():
    from tests.test_gpu_parity import _bubble2d
    case = _bubble2d(N=64, R=6.0, levels=2, rr=100.0, nu=(0.06, 0.6), g=2e-5, sigma=2e-3)
    case["refine_dist"] = [8.0]
    case["regrid_every"] = 6
    _same(_run(case, 15, 0), _run(case, 15, 1))


def test_persistent_with_graphs_matches_eager():
    from tests.test_gpu_parity import _bubble2d
    case = _bubble2d(N=64, R=6.0, levels=2, rr=100.0, nu=(0.06, 0.6), g=2e-5, sigma=2e-3)
    _same(_run(case, 12, 0), _run(case, 12, 1, graphs=True))


def test_persistent_matches_per_pass_3d_and_ensemble():
    from paper_2601_05936_gb300 import workloads
    c3 = workloads.rising_bubble_3d(scale=0.25)
    _same(_run(c3, 6, 0), _run(c3, 6, 1))
    ens = workloads.ensemble(n_cases=3, w_range=(96, 128))
    _same(_run(ens, 6, 0), _run(ens, 6, 1))


def test_set_driver_rejects_bad_mode():
    from paper_2601_05936_gb300 import lsb, workloads
    g = lsb.Grid(workloads.stratified_channel(steps=1))
    with pytest.raises(lsb.LsbError):
        g.set_driver(2)
    g.close()


def test_single_step_graph_replay_matches_eager():
    """lsb_step(1) calls replay one-step graphs (one per starting parity of level 0),
    across a regrid and an odd total; a change of the level-set iteration counts through
    lsb_set_params drops the graphs."""
    import torch

    from paper_2601_05936_gb300 import lsb
    from tests.test_gpu_parity import _bubble2d
    case = _bubble2d(N=64, R=6.0, levels=2, rr=100.0, nu=(0.06, 0.6), g=2e-5, sigma=2e-3)
    case["refine_dist"] = [8.0]
    case["regrid_every"] = 6

    def run(graphs, one_at_a_time, change_at=None):
        st = torch.cuda.Stream()
        g = lsb.Grid(case, stream=st)
        g.use_graphs(graphs)
        for k in range(13):
            if k == change_at:
                c2 = dict(case, n_ext=6)
                g.set_params(c2)
            if one_at_a_time:
                g.step(1)
            elif k % 2 == 0:
                g.step(2 if k < 12 else 1)
        g.sync()
        out = [g.get(f, 0, l) for l in range(2) for f in ("rho", "u")] + [g.get("phi"), g.get("tag")]
        launches = g.kernel_launches()
        g.close()
        return out, launches

    ref, n_ref = run(False, True)
    for mode in (True, False):
        got, n = run(True, mode)
        _same(ref, got)
        assert n == n_ref
    ref2, _ = run(False, True, change_at=9)
    got2, _ = run(True, True, change_at=9)
    _same(ref2, got2)


@pytest.mark.parametrize("dim", [3, 2])
def test_side_stream_coarse_collide_matches_serial(dim):
    """With a stream of its own and kernel timing off, a coarser level's collide-and-stream
    runs on a side stream beside the first fine sub-step, and the deepest level's second
    ghost ring fills on another beside the first sub-step's interface and level-set
    passes; with kernel timing on both run in line.  Both orders give the same state bit
    for bit (eager and graph replay; two levels in 3D, three in 2D, where the middle
    level's collide and the deepest ring's fill both leave the main stream)."""
    import torch

    from paper_2601_05936_gb300 import lsb, workloads
    if dim == 3:
        case = workloads.rising_bubble_3d(scale=0.25)
    else:
        case = workloads.rising_bubble_2d(nx=64, ny=128, levels=3, radius_base=8.0)
        case["regrid_every"] = 3
    nl = case["n_levels"]

    def run(timed, graphs):
        st = torch.cuda.Stream()
        g = lsb.Grid(case, stream=st)
        g.use_graphs(graphs)
        g.profile(1 if timed else 0)
        g.step(6)
        g.sync()
        if timed:
            g.profile_read()
            g.profile(0)
        out = [g.get(f, 0, l) for l in range(nl) for f in ("rho", "u")] + [g.get("phi"), g.get("tag")]
        g.close()
        return out

    ref = run(True, False)
    _same(ref, run(False, False))
    _same(ref, run(False, True))


def test_switching_driver_mid_run_matches_per_pass():
    """The per-pass launches read stage arrays that mirror phi and u~ outside the band;
    the persistent launch keeps no such mirror, so after steps with it the handle
    restores the mirror before the next per-pass step.  Switching 0 -> 1 -> 0 mid-run
    gives the state of per-pass launches throughout, bit for bit."""
    from paper_2601_05936_gb300 import lsb
    from tests.test_gpu_parity import _bubble2d
    case = _bubble2d(N=64, R=6.0, levels=2, rr=100.0, nu=(0.06, 0.6), g=2e-5, sigma=2e-3)
    case["refine_dist"] = [8.0]
    case["regrid_every"] = 5
    ref = _run(case, 12, 0)
    g = lsb.Grid(case)
    g.step(3)
    g.set_driver(1)
    g.step(4)
    g.set_driver(0)
    g.step(5)
    g.sync()
    got = [g.get(f, 0, l) for l in range(2) for f in ("rho", "u")] + [g.get("phi"), g.get("tag")]
    g.close()
    _same(ref, got)
