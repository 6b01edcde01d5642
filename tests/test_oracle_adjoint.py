"""Pins for oracle/adjoint.py: the frozen-interface adjoint of one step and of a window.

The adjoint is checked against the forward oracle itself, not against a
second copy of its formulas: central finite differences of the float64
forward map in every parameter, and the dot-product identity
<J v, w> = <v, J^T w> with J v from central differences, both on random
directions.  Truncation error of central differences is O(h^2) on a smooth
map, so agreement to ~1e-7 relative pins every term (a dropped term, a
wrong sign or a transposed index moves the result by O(1) of that term's
share).  The cases contain cut links of all three bounce-back branches of
Eq. bb, walls with a moving lid, gravity and a body force.
"""
import numpy as np
import pytest

from oracle.adjoint import FrozenStep, NPARAM, gradients, objective, params_of
from oracle.lbm import equilibrium
from oracle.sim import Sim
from paper_2601_05936_gb300 import workloads


def _setup(lattice, n, seed=1):
    case = workloads.adjoint_window(lattice, n=n)
    sim = Sim(case)
    st = FrozenStep(sim)
    rng = np.random.default_rng(seed)
    lat = sim.lat
    N = st.g.N
    # perturbed initial state: random densities and velocities near rest, plus a non-equilibrium part
    rho = 1.0 + 0.01 * rng.standard_normal(N)
    u = 0.02 * rng.standard_normal((lat.D, N))
    f0 = equilibrium(lat, rho, u) + 1e-3 * rng.standard_normal((lat.Q, N)) * lat.w[:, None]
    return sim, st, f0, rng


CASES = [("D2Q9", (32, 24)), ("D3Q19", (10, 10, 14))]


def _near_interface(st):
    """Cells of the cut links (both sides): where the interface terms act."""
    m = np.zeros(st.g.N)
    m[st.x] = 1.0
    m[st.y] = 1.0
    return m[None, :]


@pytest.mark.parametrize("lattice,n", CASES)
def test_every_bounce_back_branch_occurs(lattice, n):
    _, st, _, _ = _setup(lattice, n)
    hi = st.q >= 0.5
    assert hi.sum() > 0
    assert (st.ok & ~hi).sum() > 0
    assert (~st.ok & ~hi).sum() > 0


@pytest.mark.parametrize("lattice,n", CASES)
def test_frozen_step_is_the_oracle_step_without_level_set(lattice, n):
    sim, st, _, _ = _setup(lattice, n)
    f = sim.f[0].copy()
    p = params_of(sim)
    for _ in range(3):
        f = st.step(f, p)
    sim.step(3)
    assert np.abs(f - sim.f[0]).max() < 1e-15


@pytest.mark.parametrize("local", [False, True], ids=["everywhere", "interface"])
@pytest.mark.parametrize("lattice,n", CASES)
def test_dot_product_identity_one_step(lattice, n, local):
    _, st, f0, rng = _setup(lattice, n)
    p = params_of(st.sim)
    m = _near_interface(st) if local else 1.0
    v = rng.standard_normal(f0.shape) * 1e-3 * m
    w = rng.standard_normal(f0.shape) * m
    eps = 1e-4
    Jv = (st.step(f0 + eps * v, p) - st.step(f0 - eps * v, p)) / (2 * eps)
    lam, dp = st.step_adjoint(f0, p, w)
    lhs = (Jv * w).sum()
    rhs = (v * lam).sum()
    assert abs(lhs - rhs) <= 1e-8 * abs(lhs), (lhs, rhs)
    # parameter directions of the same step
    for kp in range(NPARAM):
        e = np.zeros(NPARAM)
        h = 1e-5 * abs(p[kp])
        e[kp] = h
        Jp = (st.step(f0, p + e) - st.step(f0, p - e)) / (2 * h)
        ref = (Jp * w).sum()
        assert abs(ref - dp[kp]) <= 1e-6 * max(abs(ref), 1e-9 * np.abs(w).sum()), (kp, ref, dp[kp])


@pytest.mark.parametrize("lattice,n", CASES)
def test_window_gradients_match_central_differences(lattice, n):
    _, st, f0, rng = _setup(lattice, n, seed=2)
    p = params_of(st.sim)
    D = st.D
    a = rng.standard_normal(4 + 2 * D)
    a[4 + D:] *= 100.0  # the gas velocity dominates, as for a rise-velocity objective
    nsteps = 6
    J, dp, lam0 = gradients(st, f0, p, nsteps, a)
    assert abs(J - objective(st, f0, p, nsteps, a)) < 1e-13 * max(1.0, abs(J))
    for kp in range(NPARAM):
        h = 1e-5 * abs(p[kp])
        e = np.zeros(NPARAM)
        e[kp] = h
        fd = (objective(st, f0, p + e, nsteps, a) - objective(st, f0, p - e, nsteps, a)) / (2 * h)
        assert abs(fd - dp[kp]) <= 2e-6 * abs(fd) + 1e-10, (kp, fd, dp[kp])
        assert abs(fd) > 0
    # the initial-state adjoint: directional derivative along a random perturbation
    v = rng.standard_normal(f0.shape) * 1e-3
    eps = 1e-4
    fd = (objective(st, f0 + eps * v, p, nsteps, a) - objective(st, f0 - eps * v, p, nsteps, a)) / (2 * eps)
    assert abs(fd - (lam0 * v).sum()) <= 1e-7 * abs(fd)


@pytest.mark.parametrize("piece", ["cvt", "Snn", "eb"])
def test_pins_detect_a_planted_mistake(monkeypatch, piece):
    """A wrong intermediate in the adjoint alone (the forward map is untouched)
    breaks the one-step identities (state or parameter directions) by far more
    than their tolerances."""
    _, st, f0, rng = _setup("D2Q9", (32, 24), seed=3)
    p = params_of(st.sim)
    orig = FrozenStep._link_pieces

    def planted(self, rho, u, S, pp):
        P = orig(self, rho, u, S, pp)  # df, the only piece the forward uses, is already formed
        P[piece] = -P[piece] if piece != "eb" else 1.1 * P[piece]
        return P

    monkeypatch.setattr(FrozenStep, "_link_pieces", planted)
    m = _near_interface(st)
    v = rng.standard_normal(f0.shape) * 1e-3 * m
    w = rng.standard_normal(f0.shape) * m
    eps = 1e-4
    Jv = (st.step(f0 + eps * v, p) - st.step(f0 - eps * v, p)) / (2 * eps)
    lam, dp = st.step_adjoint(f0, p, w)
    lhs, rhs = (Jv * w).sum(), (v * lam).sum()
    worst = abs(lhs - rhs) / abs(lhs)
    for kp in range(NPARAM):
        e = np.zeros(NPARAM)
        e[kp] = 1e-5 * abs(p[kp])
        ref = ((st.step(f0, p + e) - st.step(f0, p - e)) / (2 * e[kp]) * w).sum()
        worst = max(worst, abs(ref - dp[kp]) / abs(ref))
    assert worst > 1e-4, worst


@pytest.mark.parametrize("lattice,n", CASES)
def test_level_set_gradient_matches_central_differences(lattice, n):
    """dJ/dphi through q, n and kappa: directional derivatives along random
    perturbations of the level set near the interface (no sign changes)."""
    sim, st, f0, rng = _setup(lattice, n, seed=5)
    p = params_of(sim)
    D = st.D
    a = rng.standard_normal(4 + 2 * D)
    a[4 + D:] *= 100.0
    nsteps = 4
    J, dp, lam0, dphi = gradients(st, f0, p, nsteps, a, want_phi=True)
    # cells within the fit stencils of interface cells
    near = np.zeros(st.g.N, dtype=bool)
    for o in np.array(np.meshgrid(*[[-1, 0, 1]] * D, indexing="ij")).reshape(D, -1).T:
        near[st.g.clamp_shift(st.icells, o)] = True
    assert np.abs(dphi[~near]).max() == 0.0
    phi = st.phi
    for trial in range(3):
        v = rng.standard_normal(st.g.N) * near
        eps = 1e-3 * np.abs(phi[near]).min() / np.abs(v).max()
        Jp = objective(FrozenStep(sim, phi + eps * v), f0, p, nsteps, a)
        Jm = objective(FrozenStep(sim, phi - eps * v), f0, p, nsteps, a)
        fd = (Jp - Jm) / (2 * eps)
        assert abs(fd - (dphi * v).sum()) <= 1e-5 * abs(fd), (fd, (dphi * v).sum())
    # single cells: an interface cell and a neighbour that enters only through the fit
    c0 = st.icells[len(st.icells) // 2]
    for c in (c0, st.g.clamp_shift(np.array([c0]), np.eye(D, dtype=int)[0] * -1)[0]):
        e = np.zeros(st.g.N)
        e[c] = 1.0
        eps = 1e-4 * abs(phi[c])
        fd = (objective(FrozenStep(sim, phi + eps * e), f0, p, nsteps, a)
              - objective(FrozenStep(sim, phi - eps * e), f0, p, nsteps, a)) / (2 * eps)
        assert abs(fd - dphi[c]) <= 1e-5 * abs(fd) + 1e-12, (c, fd, dphi[c])
