"""GPU adjoint with a moving level set against oracle/adjoint_ls.py.

The oracle's transposed step (pinned to finite differences of the float64
forward map in test_oracle_adjoint_ls.py) and the CUDA reverse sweep must
agree on the parameter gradients and on the adjoints of the window's start
state (f, phi, u~), after the same warm-up, on windows in which no cell
changes phase.  FP32 forward and reverse arithmetic; measured agreement
~1e-7 on parameter gradients and dJ/df, ~3e-6 on dJ/dphi and ~4e-5 on dJ/du~
(relative L2); the tolerances below are 1e-4 (parameters, dJ/df) and 1e-3
(dJ/dphi, dJ/du~).
"""
import numpy as np
import pytest

from gpu_util import as_fp32_phi, rel_l2

pytestmark = pytest.mark.gpu


def _case(lattice, n):
    from paper_2601_05936_gb300 import workloads
    c = workloads.adjoint_window(lattice, seed=6055, n=n)
    c.update(ls_active=True, n_ext=4, dtau_ext=0.5, reinit_every=1, n_reinit=1, dtau_reinit=0.3)
    return as_fp32_phi(c)


CASES = [("D2Q9", (48, 32), 3, 8), ("D3Q19", (32, 16, 20), 3, 4)]


@pytest.mark.parametrize("lattice,n,warmup,steps", CASES)
def test_moving_adjoint_matches_oracle(lattice, n, warmup, steps):
    from oracle.adjoint_ls import MovingStep, gradients, params_of
    from oracle.sim import Sim
    from paper_2601_05936_gb300 import lsb
    case = _case(lattice, n)
    D = len(n)
    rng = np.random.default_rng(3)
    a = rng.standard_normal(4 + 2 * D)
    a[4 + D:] *= 100.0
    sim = Sim(case)
    sim.step(warmup)
    st = MovingStep(sim)
    J, dp_o, (lf_o, lphi_o, lut_o) = gradients(st, (sim.f[0].copy(), sim.phi.copy(), sim.ut.copy()),
                                               params_of(sim), steps, a)
    g = lsb.Grid(case)
    g.step(warmup)
    g.record(5)
    g.step(steps)
    dp_g, dphi_g = g.backward(a.reshape(1, -1), want_phi=True)
    lf_g = g.get("adj_f").reshape(g.Q, -1).astype(np.float64)
    lut_g = g.get("adj_uext").reshape(D, -1).astype(np.float64)
    err = dict(dp=np.abs(dp_g[0] - dp_o) / np.abs(dp_o), lf=rel_l2(lf_g, lf_o),
               lphi=rel_l2(dphi_g[0].reshape(-1).astype(np.float64), lphi_o), lut=rel_l2(lut_g, lut_o))
    print(lattice, err)
    assert (err["dp"] <= 1e-4).all(), err
    assert err["lf"] < 1e-4 and err["lphi"] < 1e-3 and err["lut"] < 1e-3, err
    g.close()


def test_moving_record_rejects_unsupported_settings():
    from paper_2601_05936_gb300 import lsb
    case = _case("D2Q9", (48, 32))
    g = lsb.Grid(dict(case, reinit_every=2))
    with pytest.raises(lsb.LsbError) as e:
        g.record(4)
    assert e.value.status == 6
    g.close()
