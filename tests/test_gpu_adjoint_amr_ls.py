"""GPU adjoint on block-refined grids with the level set transported, against the oracle's
AMRMovingStep (pinned to central differences in test_oracle_adjoint_amr_ls.py).

Two levels, the finest level's level set live; the CUDA reverse sweep replays each coarse
step with its per-call record (populations, and phi and u~ at every finest sub-step) and
transposes the recursion with the moving finest sub-steps.  Tolerances as for the
single-level moving adjoint: parameter gradients and dJ/df within 1e-4 (relative), dJ/dphi
within 1e-3 (relative L2), FP32 against float64; dJ/du~ (norm ~1e-4, summed with FP32
atomics through the transport and extension transposes of every fine sub-step) within 3e-3
(measured 1.1e-3).
"""
import numpy as np
import pytest

from gpu_util import as_fp32_phi, rel_l2

pytestmark = pytest.mark.gpu

CASES = [("D2Q9", (48, 24), (8, 8), 4.0, 6158, 2, 3), ("D3Q19", (16, 8, 12), (4, 4, 4), 2.0, 6159, 1, 2)]


def _case(lattice, n, block, rd, seed):
    from paper_2601_05936_gb300 import workloads
    c = workloads.adjoint_window(lattice, seed=seed, n=n, levels=2, block=block, refine_dist=rd)
    c.update(ls_active=True, n_ext=4, dtau_ext=0.5, reinit_every=1, n_reinit=1, dtau_reinit=0.3)
    return as_fp32_phi(c)


@pytest.mark.parametrize("lattice,n,block,rd,seed,warmup,steps", CASES)
def test_amr_moving_adjoint_matches_oracle(lattice, n, block, rd, seed, warmup, steps):
    from oracle.adjoint_amr import AMRMovingStep, gradients, params_of
    from oracle.sim import Sim
    from paper_2601_05936_gb300 import lsb
    case = _case(lattice, n, block, rd, seed)
    D = len(n)
    a = np.random.default_rng(3).standard_normal(4 + 2 * D)
    a[4 + D:] *= 100.0
    sim = Sim(case)
    sim.step(warmup)
    st = AMRMovingStep(sim)
    S0 = ([f.copy() for f in sim.f], sim.phi.copy(), sim.ut.copy())
    J, dp_o, (lf_o, lphi_o, lut_o) = gradients(st, S0, params_of(sim), steps, a)
    g = lsb.Grid(case)
    g.step(warmup)
    g.record(2)
    g.step(steps)
    dp_g, dphi_g = g.backward(a.reshape(1, -1), want_phi=True)
    rel = np.abs(dp_g[0] - dp_o) / np.abs(dp_o)
    assert (rel < 1e-4).all(), (rel, dp_g[0], dp_o)
    for l in range(2):
        lf_g = g.get("adj_f", 0, l).reshape(g.Q, -1).astype(np.float64)
        assert rel_l2(lf_g, lf_o[l]) < 1e-4, (l, rel_l2(lf_g, lf_o[l]))
    lphi_g = dphi_g[0].reshape(-1).astype(np.float64)
    assert rel_l2(lphi_g, lphi_o) < 1e-3, rel_l2(lphi_g, lphi_o)
    lut_g = g.get("adj_uext").reshape(D, -1).astype(np.float64)
    assert rel_l2(lut_g, lut_o) < 3e-3, rel_l2(lut_g, lut_o)
    g.close()
