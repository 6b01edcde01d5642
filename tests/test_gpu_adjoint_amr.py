"""GPU adjoint on block-refined grids against the oracle's multi-level adjoint.

The oracle (oracle/adjoint_amr.py) is pinned to central differences of the
float64 forward map; here the CUDA reverse sweep over a two-level recording
must reproduce its parameter gradients, the per-level adjoint populations
dJ/df_0 and dJ/dphi on the same frozen-interface window after the same
forward warm-up.  FP32 state and adjoint against float64: the tolerances are
those of the single-level adjoint test (1e-3 per parameter gradient, 1e-3
relative L2 on dJ/df_0 per level, 5e-3 on dJ/dphi).  The layouts hold coarse
leaves, a restriction layer and a fine ghost ring, so every transposed
transfer is on the compared path.
"""
import numpy as np
import pytest

from gpu_util import as_fp32_phi, rel_l2

pytestmark = pytest.mark.gpu

CASES = [("D2Q9", (48, 24), (8, 8), 4.0, 6, 10), ("D3Q19", (12, 8, 12), (4, 4, 4), 2.0, 4, 6),
         # refinement distance below a cell: coarse leaves meet the other phase (plain bounce-back)
         ("D2Q9", (48, 24), (8, 8), 0.2, 6, 10), ("D3Q19", (12, 8, 12), (4, 4, 4), 0.2, 4, 6)]


def _case(lattice, n, block, rd):
    from paper_2601_05936_gb300 import workloads
    return as_fp32_phi(workloads.adjoint_window(lattice, n=n, levels=2, block=block, refine_dist=rd))


def _weights(D, seed=0):
    a = np.random.default_rng(seed).standard_normal(4 + 2 * D)
    a[4 + D:] *= 100.0
    return a


def _gpu(case, warmup, steps, a, every, want_phi=False):
    from paper_2601_05936_gb300 import lsb
    g = lsb.Grid(case)
    g.step(warmup)
    g.record(every)
    g.step(steps)
    res = g.backward(a.reshape(1, -1), want_phi=want_phi)
    dp, dphi = res if want_phi else (res, None)
    lam = [g.get("adj_f", 0, l).reshape(g.Q, -1).astype(np.float64) for l in range(2)]
    return g, dp[0], lam, dphi


@pytest.mark.parametrize("lattice,n,block,rd,warmup,steps", CASES)
def test_amr_adjoint_matches_oracle(lattice, n, block, rd, warmup, steps):
    from oracle.adjoint_amr import AMRFrozenStep, gradients, params_of
    from oracle.sim import Sim
    case = _case(lattice, n, block, rd)
    D = len(n)
    a = _weights(D)
    sim = Sim(case)
    sim.step(warmup)
    assert sim.masks[0][0].any() and sim.masks[0][2].any() and sim.masks[1][3].any()
    st = AMRFrozenStep(sim)
    _, dp_o, lam_o, dphi_o = gradients(st, [f.copy() for f in sim.f], params_of(sim), steps, a, want_phi=True)
    g, dp_g, lam_g, dphi_g = _gpu(case, warmup, steps, a, every=4, want_phi=True)
    for l in range(2):
        assert np.array_equal(g.get("blocks", 0, l), sim.status[l]), l
    for k in range(5):
        assert abs(dp_g[k] - dp_o[k]) <= 1e-3 * abs(dp_o[k]) + 1e-9, (k, dp_g, dp_o)
    for l in range(2):
        assert rel_l2(lam_g[l], lam_o[l]) < 1e-3, (l, rel_l2(lam_g[l], lam_o[l]))
        assert np.abs(lam_g[l][:, ~sim.masks[l][0]]).max() == 0.0  # zero off the leaves
    d_g = dphi_g[0].reshape(-1).astype(np.float64)
    assert rel_l2(d_g, dphi_o) < 5e-3, rel_l2(d_g, dphi_o)
    g.close()


def test_amr_checkpoint_spacing_and_state_restore():
    from paper_2601_05936_gb300 import lsb
    lattice, n, block, rd, warmup, steps = CASES[0]
    case = _case(lattice, n, block, rd)
    a = _weights(2, seed=3)
    res = [_gpu(case, warmup, steps, a, every) for every in (1, 3, 100)]
    for _, dp, lam, _ in res[1:]:
        assert np.allclose(dp, res[0][1], rtol=1e-5, atol=0)
        for l in range(2):
            assert rel_l2(lam[l], res[0][2][l]) < 1e-6
    # after backward the state is the last recorded one, and stepping on matches a plain run
    g = res[0][0]
    ref = lsb.Grid(case)
    ref.step(warmup + steps)

    def same_leaves():  # non-leaf cells of the buffers hold values the step never reads
        for l in range(2):
            leaf = (g.get("tag", 0, l).reshape(-1) & 64) != 0
            fg, fr = g.get("f", 0, l).reshape(g.Q, -1), ref.get("f", 0, l).reshape(g.Q, -1)
            assert np.array_equal(fg[:, leaf], fr[:, leaf]), l
    same_leaves()
    g.step(3)
    ref.step(3)
    same_leaves()
    for r in res:
        r[0].close()
    ref.close()


def test_amr_recording_needs_equal_levels():
    from paper_2601_05936_gb300 import lsb, workloads
    c2 = _case(*CASES[0][:4])
    c1 = workloads.adjoint_window("D2Q9", n=(48, 24))
    c1["block"] = (8, 8)
    g = lsb.Grid([c2, c1])
    with pytest.raises(lsb.LsbError) as e:
        g.record(3)
    assert e.value.status == 6
    g.close()
