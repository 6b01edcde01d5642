"""Pins for oracle/objective.py: the smoothed-indicator observables of the adjoint
objective (Sec. 3.2's volume, centroid and rise velocity as H_eps-weighted sums).

* H_eps against its closed-form properties: 1/2 on the interface, H(phi) +
  H(-phi) = 1, continuous with its derivative at +-eps, unit integral of H'.
* The smoothed volume of a disk and of a sphere converges to pi R^2 and
  4/3 pi R^3 with the grid; eps -> 0 gives the sharp observables.
* The adjoint of the observables against central differences in phi and f,
  on one level and on two.
* Window gradients of the smoothed centroid height with the level set moving:
  dJ/dsigma and dJ/dphi_0 against central differences of the forward oracle;
  the same objective with the sharp indicator has a centroid gradient of
  exactly zero.
"""
import numpy as np
import pytest

from oracle import objective
from oracle.adjoint import FrozenStep, params_of
from oracle.adjoint import gradients as frozen_gradients
from oracle.adjoint_ls import MovingStep, gradients, objective as window_objective
from oracle.lbm import equilibrium
from oracle.sim import Sim
from paper_2601_05936_gb300 import workloads


def test_heaviside_closed_form_properties():
    eps = 1.5
    phi = np.linspace(-3, 3, 1201)
    h = objective.heaviside(phi, eps)
    assert objective.heaviside(0.0, eps) == 0.5
    assert np.allclose(h + objective.heaviside(-phi, eps), 1.0, atol=1e-15)
    assert np.all(np.diff(h) >= -1e-15)
    assert abs(objective.heaviside(eps, eps) - 1.0) < 1e-15 and abs(objective.heaviside(-eps, eps)) < 1e-15
    d = objective.dheaviside(phi, eps)
    assert abs(objective.dheaviside(eps, eps)) < 1e-15 and abs(objective.dheaviside(-eps, eps)) < 1e-15
    # derivative against central differences, and unit integral (trapezoid over [-eps, eps])
    hstep = 1e-6
    for x in (-1.2, -0.3, 0.0, 0.7, 1.4):
        fd = (objective.heaviside(x + hstep, eps) - objective.heaviside(x - hstep, eps)) / (2 * hstep)
        assert abs(fd - objective.dheaviside(x, eps)) < 1e-8
    xs = np.linspace(-eps, eps, 20001)
    assert abs(np.trapezoid(objective.dheaviside(xs, eps), xs) - 1.0) < 1e-8
    assert d.max() == pytest.approx(1.0 / eps)


def _disk_case(n, R, D):
    x = np.arange(n) + 0.5
    mesh = np.meshgrid(*([x] * D), indexing="ij")[::-1]
    c = n / 2 + 0.31
    r = np.sqrt(sum((m - c) ** 2 for m in mesh))
    lat = "D2Q9" if D == 2 else "D3Q19"
    return dict(lattice=lat, base=(n,) * D, block=(n,) * D, periodic=(True,) * D, rho_phys=(1.0, 0.1),
                nu=(0.1, 0.1), phi0=(R - r).reshape(-1), ls_active=False)


@pytest.mark.parametrize("D,sizes", [(2, ((24, 8.0), (48, 16.0), (96, 32.0))), (3, ((16, 5.0), (32, 10.0)))])
def test_smoothed_volume_converges_to_the_ball(D, sizes):
    errs = []
    for n, R in sizes:
        s = Sim(_disk_case(n, R, D))
        obs = objective.observables(s.lat, objective.levels_of(s), s.f, s.phi, 1.5)
        exact = np.pi * R ** 2 if D == 2 else 4.0 / 3.0 * np.pi * R ** 3
        errs.append(abs(obs[2] / exact - 1.0))
        # centroid of the ball at its centre
        assert np.abs(obs[4:4 + D] - (n / 2 + 0.31)).max() < 0.05
    assert errs[-1] < 0.01 and errs[-1] < errs[0], errs


def test_sharp_limit():
    s = Sim(_disk_case(24, 7.3, 2))
    st = FrozenStep(s)
    sharp = st.observables(s.f[0])
    smooth = objective.observables(s.lat, objective.levels_of(s), s.f, s.phi, 1e-9)
    assert np.allclose(sharp, smooth, rtol=1e-12, atol=1e-12)


def _bubble_state(levels, seed=3):
    case = workloads.adjoint_window("D2Q9", seed=6055, n=(32, 24) if levels == 1 else (24, 16), levels=levels,
                                    block=None if levels == 1 else (8, 8))
    s = Sim(case)
    rng = np.random.default_rng(seed)
    F = []
    for f in s.f:
        N = f.shape[1]
        rho = 1.0 + 0.002 * rng.standard_normal(N)
        u = 0.005 * rng.standard_normal((2, N))
        F.append(equilibrium(s.lat, rho, u))
    return s, F, rng


@pytest.mark.parametrize("levels", [1, 2])
def test_observables_adjoint_matches_central_differences(levels):
    s, F, rng = _bubble_state(levels)
    lv = objective.levels_of(s)
    eps_h = 1.5
    a = rng.standard_normal(8)
    phi = s.phi.copy()
    lamF, lphi = objective.observables_adjoint(s.lat, lv, F, phi, eps_h, a)
    J = lambda F_, phi_: float(a @ objective.observables(s.lat, lv, F_, phi_, eps_h))
    # fourth-order central differences (the masses, ~1e3, would bury a second-order
    # difference at small steps in round-off)
    h = 1e-4
    # phi: random direction on the cells within 2 eps of the interface (where H' lives)
    v = rng.standard_normal(phi.size) * (np.abs(phi) < 3.0)
    Jh = [J(F, phi + m * h * v) for m in (-2, -1, 1, 2)]
    fd = (Jh[0] - 8 * Jh[1] + 8 * Jh[2] - Jh[3]) / (12 * h)
    assert abs(fd - float(v @ lphi)) <= 1e-7 * abs(fd), (fd, float(v @ lphi))
    assert np.abs(lphi).max() > 0
    # populations, every level
    V = [1e-3 * rng.standard_normal(f.shape) * s.lat.w[:, None] for f in F]
    hf = 1e-2  # J is a ratio of polynomials in f: a larger step keeps the masses' round-off small
    Jh = [J([f + m * hf * x for f, x in zip(F, V)], phi) for m in (-2, -1, 1, 2)]
    fd = (Jh[0] - 8 * Jh[1] + 8 * Jh[2] - Jh[3]) / (12 * hf)
    ad = sum(float((x * lam).sum()) for x, lam in zip(V, lamF))
    assert abs(fd - ad) <= 1e-7 * abs(fd), (fd, ad)


def _moving_setup(eps_h):
    c = workloads.adjoint_window("D2Q9", seed=6055, n=(32, 24))
    c.update(ls_active=True, n_ext=4, dtau_ext=0.5, reinit_every=1, n_reinit=1, dtau_reinit=0.3)
    sim = Sim(c)
    st = MovingStep(sim, eps=eps_h)
    rng = np.random.default_rng(2)
    lat, N = sim.lat, st.g.N
    rho = 1.0 + 0.002 * rng.standard_normal(N)
    u = 0.002 * rng.standard_normal((lat.D, N))
    f0 = equilibrium(lat, rho, u) + 2e-4 * rng.standard_normal((lat.Q, N)) * lat.w[:, None]
    ut0 = 0.002 * rng.standard_normal((lat.D, N))
    return sim, st, (f0, sim.phi.copy(), ut0), rng


def test_window_gradient_of_the_smoothed_centroid_height():
    """J = vertical centroid of the gas after 4 steps with the level set moving: dJ/dsigma
    and dJ/dphi_0 (along a smooth perturbation of the band) against central differences;
    with the sharp indicator the same J does not depend on sigma at all."""
    sim, st, s0, rng = _moving_setup(1.5)
    p = params_of(sim)
    a = np.zeros(8)
    a[5] = 1.0  # centroid, y component
    nsteps = 4
    J, dp, lam0 = gradients(st, s0, p, nsteps, a)
    e = 1e-4 * p[0]
    pp, pm = p.copy(), p.copy()
    pp[0] += e
    pm[0] -= e
    fd = (window_objective(st, s0, pp, nsteps, a) - window_objective(st, s0, pm, nsteps, a)) / (2 * e)
    assert abs(fd) > 0 and abs(fd - dp[0]) <= 1e-5 * abs(fd), (fd, dp[0])
    v = rng.standard_normal(st.g.N) * st.band * 1e-2
    h = 1e-4
    Jh = [window_objective(st, (s0[0], s0[1] + m * h * v, s0[2]), p, nsteps, a) for m in (-2, -1, 1, 2)]
    fd = (Jh[0] - 8 * Jh[1] + 8 * Jh[2] - Jh[3]) / (12 * h)
    ad = float(v @ lam0[1])
    assert abs(fd - ad) <= 2e-5 * abs(fd), (fd, ad)
    # the sharp indicator: the centroid is a function of the fixed phases only
    sharp = MovingStep(sim)
    _, dps, _ = gradients(sharp, s0, p, nsteps, a)
    assert dps[0] == 0.0


def test_frozen_window_dphi_includes_the_direct_term():
    """Frozen level set: dJ/dphi of the smoothed volume objective is H_eps' at the cells
    plus the terms through the link fractions and the curvature fit."""
    s, F, rng = _bubble_state(1)
    st = FrozenStep(s, eps=1.5)
    p = params_of(s)
    a = np.zeros(8)
    a[2] = 1.0
    a[6] = 50.0  # gas velocity x
    J, dp, lam0, dphi = frozen_gradients(st, F[0], p, 3, a, want_phi=True)
    v = rng.standard_normal(s.phi.size) * (np.abs(s.phi) < 3.0) * 1e-2
    h = 1e-4

    def Jphi(ph):
        return float(a @ FrozenStep(s, ph, eps=1.5).observables(
            __import__("oracle.adjoint", fromlist=["trajectory"]).trajectory(FrozenStep(s, ph, eps=1.5), F[0], p, 3)[-1]))
    Jh = [Jphi(s.phi + m * h * v) for m in (-2, -1, 1, 2)]
    fd = (Jh[0] - 8 * Jh[1] + 8 * Jh[2] - Jh[3]) / (12 * h)
    assert abs(fd - float(v @ dphi)) <= 1e-5 * abs(fd), (fd, float(v @ dphi))
