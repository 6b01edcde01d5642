"""Pins for oracle/adjoint_ls.py: the adjoint of the step with a moving level set.

As for the frozen interface, the transposed step is checked against the
forward oracle: MovingStep.step must equal Sim.step; the one-step dot-product
identity <J v, w> = <v, J^T w> with J v from central differences must hold
for perturbations of f, phi and u~ together (and each alone), and for every
parameter; window gradients must match central differences of the objective.
The windows are short enough that no cell changes phase and no discrete
choice (upwind side, Godunov branch, frozen cell) switches under the
perturbations, so the map is smooth there.
"""
import numpy as np
import pytest

from oracle.adjoint_ls import NPARAM, MovingStep, gradients, objective, params_of
from oracle.lbm import equilibrium
from oracle.sim import Sim
from paper_2601_05936_gb300 import workloads


def _case(lattice, n):
    # seed 6055: no cell centre within 0.038 of the interface, so short windows with
    # the velocities below change no phase
    c = workloads.adjoint_window(lattice, seed=6055, n=n)
    c.update(ls_active=True, n_ext=4, dtau_ext=0.5, reinit_every=1, n_reinit=1, dtau_reinit=0.3)
    return c


def _setup(lattice, n, seed=1, amp=0.005):
    sim = Sim(_case(lattice, n))
    st = MovingStep(sim)
    rng = np.random.default_rng(seed)
    lat, N = sim.lat, st.g.N
    rho = 1.0 + 0.002 * rng.standard_normal(N)
    u = amp * rng.standard_normal((lat.D, N))
    f0 = equilibrium(lat, rho, u) + 2e-4 * rng.standard_normal((lat.Q, N)) * lat.w[:, None]
    ut0 = amp * rng.standard_normal((lat.D, N))
    return sim, st, (f0, sim.phi.copy(), ut0), rng


def _rand_dir(st, rng, scale=(1e-3, 1e-2, 1e-3)):
    """Random perturbation of (f, phi, u~); phi only on band cells."""
    g = st.g
    vf = scale[0] * rng.standard_normal((st.lat.Q, g.N)) * st.lat.w[:, None]
    vphi = scale[1] * rng.standard_normal(g.N) * st.band
    vut = scale[2] * rng.standard_normal((st.D, g.N))
    return vf, vphi, vut


def _dot(a, b):
    return sum(float((x * y).sum()) for x, y in zip(a, b))


def _axpy(s, eps, v):
    return tuple(x + eps * y for x, y in zip(s, v))


CASES = [("D2Q9", (32, 24)), ("D3Q19", (10, 10, 14))]


@pytest.mark.parametrize("lattice,n", CASES)
def test_moving_step_is_the_oracle_step(lattice, n):
    sim = Sim(_case(lattice, n))
    st = MovingStep(sim)
    s = (sim.f[0].copy(), sim.phi.copy(), sim.ut.copy())
    p = params_of(sim)
    for _ in range(3):
        s = st.step(s, p)
    sim.step(3)
    assert np.abs(s[0] - sim.f[0]).max() < 1e-14
    assert np.abs(s[1] - sim.phi).max() < 1e-13
    assert np.abs(s[2] - sim.ut).max() < 1e-14
    assert sim.stats["flipped"] == 0


@pytest.mark.parametrize("part", ["all", "f", "phi", "ut"])
@pytest.mark.parametrize("lattice,n", CASES)
def test_dot_product_identity_one_step(lattice, n, part):
    sim, st, s0, rng = _setup(lattice, n)
    p = params_of(sim)
    v = _rand_dir(st, rng)
    keep = {"all": (1, 1, 1), "f": (1, 0, 0), "phi": (0, 1, 0), "ut": (0, 0, 1)}[part]
    v = tuple(k * x for k, x in zip(keep, v))
    w = (rng.standard_normal(s0[0].shape), rng.standard_normal(st.g.N) * st.band,
         rng.standard_normal(s0[2].shape))
    # small steps: the WENO5 weights (epsilon 1e-6) make the phi direction strongly
    # nonlinear, and central differences lose O(eps^2) to it (measured 2e-4 at 1e-3)
    eps = 1e-4
    sp, sm = st.step(_axpy(s0, eps, v), p), st.step(_axpy(s0, -eps, v), p)
    Jv = tuple((a - b) / (2 * eps) for a, b in zip(sp, sm))
    lam, dp = st.step_adjoint(s0, p, w)
    lhs, rhs = _dot(Jv, w), _dot(v, lam)
    assert abs(lhs - rhs) <= 2e-5 * max(abs(lhs), 1e-12), (lhs, rhs)
    if part == "all":
        for kp in range(NPARAM):
            e = np.zeros(NPARAM)
            e[kp] = 1e-5 * abs(p[kp])
            Jp = [(a - b) / (2 * e[kp]) for a, b in zip(st.step(s0, p + e), st.step(s0, p - e))]
            ref = _dot(Jp, w)
            assert abs(ref - dp[kp]) <= 1e-6 * abs(ref), (kp, ref, dp[kp])


@pytest.mark.parametrize("lattice,n", CASES)
def test_window_gradients_match_central_differences(lattice, n):
    sim, st, s0, rng = _setup(lattice, n, seed=2, amp=0.002)
    p = params_of(sim)
    D = st.D
    a = rng.standard_normal(4 + 2 * D)
    a[:4] = 0.0  # velocity observables only: the masses would bury the small u~ effect in round-off
    nsteps = 4
    J, dp, lam0 = gradients(st, s0, p, nsteps, a)
    assert abs(J - objective(st, s0, p, nsteps, a)) < 1e-13 * max(1.0, abs(J))
    for kp in range(NPARAM):
        e = np.zeros(NPARAM)
        e[kp] = 1e-5 * abs(p[kp])
        fd = (objective(st, s0, p + e, nsteps, a) - objective(st, s0, p - e, nsteps, a)) / (2 * e[kp])
        assert abs(fd - dp[kp]) <= 1e-5 * abs(fd) + 1e-12, (kp, fd, dp[kp])
    # fourth-order central differences; u~ moves J by ~1e-8, so it takes a larger step
    for part, (eps, tol) in enumerate(((1e-4, 2e-5), (1e-4, 2e-5), (3e-3, 1e-4))):
        v = _rand_dir(st, rng)
        v = tuple(x if k == part else 0 * x for k, x in enumerate(v))
        Jh = [objective(st, _axpy(s0, m * eps, v), p, nsteps, a) for m in (-2, -1, 1, 2)]
        fd = (Jh[0] - 8 * Jh[1] + 8 * Jh[2] - Jh[3]) / (12 * eps)
        assert abs(fd - _dot(v, lam0)) <= tol * abs(fd), (part, fd, _dot(v, lam0))


@pytest.mark.parametrize("plant", ["weno_linear_weights", "no_q_in_interface_velocity", "no_S_prime"])
def test_pins_detect_a_planted_mistake(monkeypatch, plant):
    """Mistakes planted in the transposed passes alone break the phi-direction identity."""
    import oracle.adjoint_ls as M
    if plant == "weno_linear_weights":
        orig = M._weno5_grad

        def bad(v):
            val, _ = orig(v)
            lin = np.array([[0.1 / 3, 0.1 * -7 / 6 - 0.6 / 6, 0.1 * 11 / 6 + 0.6 * 5 / 6 + 0.3 / 3,
                             0.6 / 3 + 0.3 * 5 / 6, -0.3 / 6]]).T
            return val, np.broadcast_to(lin, v.shape).copy()
        monkeypatch.setattr(M, "_weno5_grad", bad)
    elif plant == "no_q_in_interface_velocity":
        orig = M.MovingStep._ext_init_T

        def bad(self, lam_ut0, f, phi, F):
            lut, lf, lphi = orig(self, lam_ut0, f, phi, F)
            return lut, lf, 0 * lphi
        monkeypatch.setattr(M.MovingStep, "_ext_init_T", bad)
    else:
        orig = M.MovingStep._extend_T

        def bad(self, lam_ut, phi, F):
            lam, lphi = orig(self, lam_ut, phi, F)
            return lam, 0 * lphi
        monkeypatch.setattr(M.MovingStep, "_extend_T", bad)
    sim, st, s0, rng = _setup("D2Q9", (32, 24))
    p = params_of(sim)
    v = _rand_dir(st, rng)
    v = (0 * v[0], v[1], 0 * v[2])
    w = (rng.standard_normal(s0[0].shape), rng.standard_normal(st.g.N) * st.band,
         rng.standard_normal(s0[2].shape))
    eps = 1e-4
    Jv = tuple((a - b) / (2 * eps) for a, b in zip(st.step(_axpy(s0, eps, v), p), st.step(_axpy(s0, -eps, v), p)))
    lam, _ = st.step_adjoint(s0, p, w)
    lhs, rhs = _dot(Jv, w), _dot(v, lam)
    assert abs(lhs - rhs) > 1e-4 * abs(lhs), (lhs, rhs)  # five times the identity test's tolerance
