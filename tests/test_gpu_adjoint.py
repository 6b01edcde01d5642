"""GPU adjoint (lsb_record / lsb_backward) against the oracle's adjoint.

The oracle adjoint is pinned to finite differences of the float64 forward map
(test_oracle_adjoint.py); here the CUDA reverse sweep must reproduce its
parameter gradients and its adjoint populations dJ/df_0 on the same
frozen-interface window, after the same forward warm-up.  The library's
forward state is FP32 (relative error ~1e-6 against the oracle) and the
reverse sweep runs in FP32 with FP64 parameter sums, so gradients agree to
~1e-4 relative; the tolerances below (1e-3 on each parameter gradient, the
agreement with finite differences that the adjoint is held to, and 1e-3
relative L2 on dJ/df_0) leave room for the accumulation over the window.
"""
import numpy as np
import pytest

from gpu_util import as_fp32_phi, rel_l2

pytestmark = pytest.mark.gpu


def _weights(D, ncase=1, seed=0):
    rng = np.random.default_rng(seed)
    a = rng.standard_normal((ncase, 4 + 2 * D))
    a[:, 4 + D:] *= 100.0
    return a


def _oracle(case, warmup, steps, a):
    from oracle.adjoint import FrozenStep, gradients, params_of
    from oracle.sim import Sim
    sim = Sim(case)
    sim.step(warmup)
    st = FrozenStep(sim)
    J, dp, lam0, dphi = gradients(st, sim.f[0], params_of(sim), steps, a, want_phi=True)
    return J, dp, lam0, dphi


def _gpu(case, warmup, steps, a, every, want_phi=False):
    from paper_2601_05936_gb300 import lsb
    g = lsb.Grid(case)
    g.step(warmup)
    g.record(every)
    g.step(steps)
    if want_phi:
        dp, dphi = g.backward(a.reshape(1, -1), want_phi=True)
    else:
        dp, dphi = g.backward(a.reshape(1, -1)), None
    lam0 = g.get("adj_f").reshape(g.Q, -1).astype(np.float64)
    return g, dp[0], lam0, dphi


CASES = [("D2Q9", (48, 32), 10, 30), ("D3Q19", (32, 16, 20), 6, 16)]


@pytest.mark.parametrize("lattice,n,warmup,steps", CASES)
def test_adjoint_matches_oracle(lattice, n, warmup, steps):
    from paper_2601_05936_gb300 import workloads
    case = as_fp32_phi(workloads.adjoint_window(lattice, n=n))
    D = len(n)
    a = _weights(D)[0]
    _, dp_o, lam_o, dphi_o = _oracle(case, warmup, steps, a)
    g, dp_g, lam_g, dphi_g = _gpu(case, warmup, steps, a, every=7, want_phi=True)
    for k in range(5):
        assert abs(dp_g[k] - dp_o[k]) <= 1e-3 * abs(dp_o[k]) + 1e-9, (k, dp_g, dp_o)
    assert rel_l2(lam_g, lam_o) < 1e-3
    # dJ/dphi of the frozen level set (q, normal, curvature): FP32 link arithmetic with
    # 1/q^2 and 1/(phi_x - phi_y)^2 factors; relative L2 over the whole field
    d_g = dphi_g[0].reshape(-1).astype(np.float64)
    assert rel_l2(d_g, dphi_o) < 5e-3, rel_l2(d_g, dphi_o)
    assert np.abs(d_g[dphi_o == 0]).max() == 0.0
    g.close()


def test_checkpoint_spacing_does_not_change_the_result():
    from paper_2601_05936_gb300 import workloads
    case = workloads.adjoint_window("D2Q9", n=(48, 32))
    a = _weights(2)[0]
    res = [_gpu(case, 5, 20, a, every)[1:3] for every in (1, 6, 100)]
    for dp, lam in res[1:]:
        assert np.allclose(dp, res[0][0], rtol=1e-5, atol=0)
        assert rel_l2(lam, res[0][1]) < 1e-6


def test_backward_restores_the_state_and_extends_the_recording():
    from paper_2601_05936_gb300 import lsb, workloads
    case = workloads.adjoint_window("D2Q9", n=(48, 32))
    a = _weights(2)
    g = lsb.Grid(case)
    g.step(4)
    g.record(5)
    g.step(12)
    f_before = g.get("f")
    dp1 = g.backward(a)
    assert np.array_equal(g.get("f"), f_before)
    dp2 = g.backward(a)  # the recording stays open: same result again
    assert np.allclose(dp1, dp2, rtol=1e-6)
    ref = lsb.Grid(case)  # stepping on after backward is the same as never having run it
    ref.step(4 + 12 + 3)
    g.step(3)
    assert np.array_equal(g.get("f"), ref.get("f"))
    dp3 = g.backward(a)  # 15 recorded steps now
    ref.close()
    h = lsb.Grid(case)
    h.step(4)
    h.record(5)
    h.step(15)
    assert np.allclose(dp3, h.backward(a), rtol=1e-5)
    g.close()
    h.close()


def test_ensemble_cases_are_independent():
    from paper_2601_05936_gb300 import lsb, workloads
    c0 = workloads.adjoint_window("D2Q9", seed=6001, n=(48, 32))
    c1 = workloads.adjoint_window("D2Q9", seed=6002, n=(64, 32))
    a = _weights(2, 2, seed=4)
    g = lsb.Grid([c0, c1])
    g.step(3)
    g.record(4)
    g.step(10)
    dp, dphi = g.backward(a, want_phi=True)
    for k, c in enumerate((c0, c1)):
        s = lsb.Grid(c)
        s.step(3)
        s.record(4)
        s.step(10)
        dps, dphis = s.backward(a[k:k + 1], want_phi=True)
        assert np.allclose(dp[k], dps[0], rtol=1e-5)
        assert rel_l2(dphi[k].astype(np.float64), dphis[0].astype(np.float64)) < 1e-5
        s.close()
    g.close()


def test_adjoint_state_errors():
    from paper_2601_05936_gb300 import lsb, workloads
    case = workloads.adjoint_window("D2Q9", n=(48, 32))
    g = lsb.Grid(case)
    a = _weights(2)
    with pytest.raises(lsb.LsbError) as e:
        g.backward(a)  # nothing recorded
    assert e.value.status == 6
    with pytest.raises(lsb.LsbError):
        g.get("adj_f")
    g.record(3)
    g.step(2)
    g.set_params(case)  # ends the recording
    with pytest.raises(lsb.LsbError):
        g.backward(a)
    g.close()
    live = dict(case, ls_active=True)
    h = lsb.Grid([case, live])  # live and frozen level sets in one recording
    with pytest.raises(lsb.LsbError) as e:
        h.record(3)
    assert e.value.status == 6
    h.close()


def test_autograd_function_returns_the_adjoint_gradient():
    import torch
    from paper_2601_05936_gb300 import autograd, lsb, workloads
    case = workloads.adjoint_window("D2Q9", n=(48, 32))
    g = lsb.Grid(case)
    g.step(5)
    f0 = g.get("f")
    p = autograd.params_tensor([case])
    obs = autograd.window(g, p, 12, checkpoint_every=5)
    loss = obs[0, 4 + 2 + 1]  # vertical gas velocity
    (grad,) = torch.autograd.grad(loss, p)
    # the same through the plain binding, from the same start state
    h = lsb.Grid(case)
    h.step(5)
    assert np.array_equal(h.get("f"), f0)
    h.record(5)
    h.step(12)
    w = np.zeros((1, 8))
    w[0, 7] = 1.0
    assert np.allclose(grad.numpy(), h.backward(w), rtol=1e-5)
    assert float(loss.detach()) == pytest.approx(h.observables()[0]["velocity"][1], rel=1e-12)
    g.close()
    h.close()
