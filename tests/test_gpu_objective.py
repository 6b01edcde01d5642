"""The smoothed-indicator objective on the GPU (lsb_set_objective) against the
oracle (oracle/objective.py, pinned in test_oracle_objective.py).

* lsb_observables with H_eps: gas volume, centroid and velocity against the
  oracle's smoothed observables on the same state (two levels, 3D).
* The reverse sweep of a window with the level set moving, J = the gas
  centroid: dJ/dparams against the oracle adjoint (1e-4 relative) and against
  central differences of the FP64 forward oracle in sigma (1e-3 relative, the
  agreement the adjoint is held to); dJ/dphi_0 against the oracle adjoint.  The
  sharp indicator gives a centroid gradient of exactly zero.
* autograd.window_from: the initial interface as a differentiable input; dJ/dR
  of the centroid height with respect to the initial bubble radius (phi_0 = R -
  |x - x_c| built in torch) against the oracle adjoint and central differences
  of the oracle in R.
"""
import numpy as np
import pytest

from gpu_util import as_fp32_phi, rel_l2

pytestmark = pytest.mark.gpu

EPS = 1.5


def test_smoothed_observables_match_oracle():
    from oracle import objective
    from oracle.sim import Sim
    from paper_2601_05936_gb300 import lsb, workloads
    case = as_fp32_phi(workloads.rising_bubble_3d(scale=0.25))
    g = lsb.Grid(case)
    g.set_objective(EPS)
    g.step(3)
    s = Sim(case)
    s.step(3)
    og = g.observables()[0]
    oo = objective.observables(s.lat, objective.levels_of(s), s.f, s.phi, EPS)
    D = 3
    assert abs(og["volume"] / oo[2] - 1.0) < 1e-6, (og["volume"], oo[2])
    assert np.abs(og["centroid"] - oo[4:4 + D]).max() < 1e-4, (og["centroid"], oo[4:4 + D])
    vmag = np.abs(oo[4 + D:]).max()
    assert np.abs(og["velocity"] - oo[4 + D:]).max() < 1e-3 * vmag, (og["velocity"], oo[4 + D:])
    assert np.abs(og["mass"] / oo[:2] - 1.0).max() < 1e-7
    with pytest.raises(lsb.LsbError) as e:
        g.set_objective(-1.0)
    assert e.value.status == 1
    g.close()


def _moving_case(lattice, n):
    from paper_2601_05936_gb300 import workloads
    c = workloads.adjoint_window(lattice, seed=6055, n=n)
    c.update(ls_active=True, n_ext=4, dtau_ext=0.5, reinit_every=1, n_reinit=1, dtau_reinit=0.3)
    return as_fp32_phi(c)


@pytest.mark.parametrize("lattice,n,warmup,steps", [("D2Q9", (48, 32), 3, 8), ("D3Q19", (32, 16, 20), 3, 4)])
def test_centroid_gradient_matches_oracle_and_differences(lattice, n, warmup, steps):
    from oracle.adjoint_ls import MovingStep, gradients, objective as window_objective, params_of
    from oracle.sim import Sim
    from paper_2601_05936_gb300 import lsb
    case = _moving_case(lattice, n)
    D = len(n)
    a = np.zeros(4 + 2 * D)
    a[4 + D - 1] = 1.0  # vertical centroid
    a[4] = 0.3          # and some of the horizontal one
    sim = Sim(case)
    sim.step(warmup)
    st = MovingStep(sim, eps=EPS)
    s0 = (sim.f[0].copy(), sim.phi.copy(), sim.ut.copy())
    p = params_of(sim)
    J, dp_o, (lf_o, lphi_o, lut_o) = gradients(st, s0, p, steps, a)
    g = lsb.Grid(case)
    g.set_objective(EPS)
    g.step(warmup)
    g.record(5)
    g.step(steps)
    dp_g, dphi_g = g.backward(a.reshape(1, -1), want_phi=True)
    dp_g = dp_g[0]
    err = np.abs(dp_g - dp_o) / np.abs(dp_o)
    print(lattice, "dJ/dp gpu", dp_g, "oracle", dp_o, "rel", err)
    assert np.abs(dp_o[0]) > 0 and (err <= 1e-4).all(), err
    lphi_err = rel_l2(dphi_g[0].reshape(-1).astype(np.float64), lphi_o)
    assert lphi_err < 1e-3, lphi_err
    # central differences of the FP64 forward oracle in sigma: the adjoint's target
    e = 1e-4 * p[0]
    pp, pm = p.copy(), p.copy()
    pp[0] += e
    pm[0] -= e
    fd = (window_objective(st, s0, pp, steps, a) - window_objective(st, s0, pm, steps, a)) / (2 * e)
    assert abs(dp_g[0] - fd) <= 1e-3 * abs(fd), (dp_g[0], fd)
    # the sharp indicator: the centroid does not depend on sigma between flips
    h = lsb.Grid(case)
    h.step(warmup)
    h.record(5)
    h.step(steps)
    assert h.backward(a.reshape(1, -1))[0][0] == 0.0
    g.close()
    h.close()


def _radius_case(R, N=48, seed=11):
    rng = np.random.default_rng(seed)
    x = np.arange(N) + 0.5
    xc, yc = N / 2 + 0.37 * rng.random(), N / 2 + 0.37 * rng.random()
    return dict(lattice="D2Q9", base=(N, N), block=(32, 8), periodic=(False, False), rho_phys=(1.0, 0.1),
                nu=(0.1, 0.1), sigma=5e-3, gravity=(0.0, -4e-5), x_ref=(xc, yc), p_gas0=5e-3 / R, ls_active=True,
                n_ext=4, dtau_ext=0.5, reinit_every=1, n_reinit=1, dtau_reinit=0.3, R=R), (x, xc, yc)


def test_autograd_initial_radius_gradient():
    """J = the gas centroid height after 8 steps from the initial state, differentiated
    with respect to the initial radius R through phi_0 = R - |x - x_c| (torch)."""
    import torch

    from oracle.adjoint_ls import MovingStep, gradients, params_of
    from oracle.sim import Sim
    from paper_2601_05936_gb300 import autograd
    R0 = 9.3
    case, (x, xc, yc) = _radius_case(R0)
    X, Y = np.meshgrid(x, x)
    dist = np.sqrt((X - xc) ** 2 + (Y - yc) ** 2).reshape(-1)
    phi_f32 = (R0 - dist).astype(np.float32).astype(np.float64)
    assert np.abs(phi_f32).min() > 2e-3  # perturbations of R below that flip no cell
    steps = 8
    R = torch.tensor(R0, dtype=torch.float64, requires_grad=True)
    phi0 = (R - torch.from_numpy(dist)).to(torch.float32)
    p = autograd.params_tensor([case])
    obs = autograd.window_from(case, p, phi0.reshape(1, -1), steps, checkpoint_every=4, eps=EPS)
    J = obs[0, 4 + 1]
    (dR, dp) = torch.autograd.grad(J, (R, p))
    # oracle adjoint: the initial state depends on phi_0 only through its signs, so
    # dJ/dR is the sum of dJ/dphi_0
    c = dict(case, phi0=phi_f32)
    sim = Sim(c)
    st = MovingStep(sim, eps=EPS)
    a = np.zeros(8)
    a[5] = 1.0
    Jo, dp_o, (lf, lphi, lut) = gradients(st, (sim.f[0].copy(), sim.phi.copy(), sim.ut.copy()), params_of(sim),
                                          steps, a)
    assert sim.stats["flipped"] == 0
    assert abs(float(J.detach()) - Jo) < 1e-4
    dR_o = float(lphi.sum())
    assert abs(float(dR) - dR_o) <= 1e-3 * abs(dR_o), (float(dR), dR_o)
    # central differences of the oracle in R (same phases, same initial populations)
    hR = 1e-3

    def J_of(r):
        s = Sim(dict(case, phi0=phi_f32 + (r - R0)))
        s2 = MovingStep(s, eps=EPS)
        from oracle.adjoint_ls import objective as wobj
        return wobj(s2, (s.f[0].copy(), s.phi.copy(), s.ut.copy()), params_of(s), steps, a)
    fd = (J_of(R0 + hR) - J_of(R0 - hR)) / (2 * hR)
    assert abs(float(dR) - fd) <= 1e-3 * abs(fd), (float(dR), fd)
    assert np.allclose(dp.numpy()[0], dp_o, rtol=1e-3)
