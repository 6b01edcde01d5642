"""Pins for oracle/adjoint_amr.py's AMRMovingStep: the adjoint of a two-level coarse step
with the finest level's level set transported.

Checked against the forward oracle itself, as for the frozen and single-level moving
adjoints: AMRMovingStep.step must be Sim.step (two levels, level set live); the one-step
dot-product identity <J v, w> = <v, J^T w> with J v from central differences must hold for
perturbations of the populations of both levels, phi and u~ together and apart, and for
every parameter; window gradients must match central differences of the objective.  The
seeds keep every cell centre at least 0.05 finest cells from the interface, so short
windows change no phase and no discrete choice.  The phi direction is strongly nonlinear
(WENO5 weights): central differences with step 1e-4 are off by ~3e-5 there, falling as the
square of the step (measured 2.7e-5, 2.2e-6, 2.5e-7 at 1e-4, 3e-5, 1e-5), so the
identity uses 1e-5.
"""
import numpy as np
import pytest

from oracle.adjoint_amr import NPARAM, AMRMovingStep, gradients, objective, params_of
from oracle.lbm import equilibrium
from oracle.sim import Sim
from paper_2601_05936_gb300 import workloads

CASES = [("D2Q9", (48, 24), (8, 8), 4.0, 6158), ("D3Q19", (16, 8, 12), (4, 4, 4), 2.0, 6159)]


def _case(lattice, n, block, rd, seed):
    c = workloads.adjoint_window(lattice, seed=seed, n=n, levels=2, block=block, refine_dist=rd)
    c.update(ls_active=True, n_ext=4, dtau_ext=0.5, reinit_every=1, n_reinit=1, dtau_reinit=0.3)
    return c


def _setup(lattice, n, block, rd, seed, rseed=1):
    sim = Sim(_case(lattice, n, block, rd, seed))
    st = AMRMovingStep(sim)
    rng = np.random.default_rng(rseed)
    lat = sim.lat
    F0 = []
    for f in sim.f:
        N = f.shape[1]
        rho = 1.0 + 0.002 * rng.standard_normal(N)
        u = 0.005 * rng.standard_normal((lat.D, N))
        F0.append(equilibrium(lat, rho, u) + 2e-4 * rng.standard_normal((lat.Q, N)) * lat.w[:, None])
    NF = st.geoms[-1].N
    S0 = (F0, sim.phi.copy(), 0.005 * rng.standard_normal((lat.D, NF)))
    return sim, st, S0, rng


def _dir(st, S0, rng, keep=(1, 1, 1)):
    lat, band = st.lat, st.moving.band
    return ([keep[0] * 1e-3 * rng.standard_normal(f.shape) * lat.w[:, None] for f in S0[0]],
            keep[1] * 1e-2 * rng.standard_normal(S0[1].shape) * band,
            keep[2] * 1e-3 * rng.standard_normal(S0[2].shape))


def _axpy(S, e, V):
    return ([a + e * b for a, b in zip(S[0], V[0])], S[1] + e * V[1], S[2] + e * V[2])


def _dot(A, B):
    return (sum(float((a * b).sum()) for a, b in zip(A[0], B[0])) + float((A[1] * B[1]).sum())
            + float((A[2] * B[2]).sum()))


def _jv(st, S0, p, V, eps):
    Sp, Sm = st.step(_axpy(S0, eps, V), p), st.step(_axpy(S0, -eps, V), p)
    return ([(a - b) / (2 * eps) for a, b in zip(Sp[0], Sm[0])], (Sp[1] - Sm[1]) / (2 * eps),
            (Sp[2] - Sm[2]) / (2 * eps))


@pytest.mark.parametrize("lattice,n,block,rd,seed", CASES)
def test_amr_moving_step_is_the_oracle_step(lattice, n, block, rd, seed):
    sim = Sim(_case(lattice, n, block, rd, seed))
    assert sim.masks[0][0].any() and sim.masks[0][2].any() and sim.masks[1][3].any()
    st = AMRMovingStep(sim)
    p = params_of(sim)
    S = ([f.copy() for f in sim.f], sim.phi.copy(), sim.ut.copy())
    for _ in range(3):
        S = st.step(S, p)
    sim.step(3)
    for a, b in zip(S[0], sim.f):
        assert np.abs(a - b).max() < 1e-14
    assert np.abs(S[1] - sim.phi).max() < 1e-13
    assert np.abs(S[2] - sim.ut).max() < 1e-14
    assert sim.stats["flipped"] == 0


@pytest.mark.parametrize("part", ["all", "f", "phi", "ut"])
@pytest.mark.parametrize("lattice,n,block,rd,seed", CASES)
def test_dot_product_identity_one_coarse_step(lattice, n, block, rd, seed, part):
    sim, st, S0, rng = _setup(lattice, n, block, rd, seed)
    p = params_of(sim)
    keep = {"all": (1, 1, 1), "f": (1, 0, 0), "phi": (0, 1, 0), "ut": (0, 0, 1)}[part]
    V = _dir(st, S0, rng, keep)
    W = ([rng.standard_normal(f.shape) for f in S0[0]], rng.standard_normal(S0[1].shape) * st.moving.band,
         rng.standard_normal(S0[2].shape))
    lam, dp = st.step_adjoint(S0, p, W)
    lhs, rhs = _dot(_jv(st, S0, p, V, 1e-5), W), _dot(V, lam)
    assert abs(lhs - rhs) <= 2e-5 * abs(lhs), (lhs, rhs)
    if part == "all":
        for kp in range(NPARAM):
            e = np.zeros(NPARAM)
            e[kp] = 1e-5 * abs(p[kp])
            Sp, Sm = st.step(S0, p + e), st.step(S0, p - e)
            Jp = ([(a - b) / (2 * e[kp]) for a, b in zip(Sp[0], Sm[0])], (Sp[1] - Sm[1]) / (2 * e[kp]),
                  (Sp[2] - Sm[2]) / (2 * e[kp]))
            ref = _dot(Jp, W)
            assert abs(ref - dp[kp]) <= 1e-6 * abs(ref), (kp, ref, dp[kp])


@pytest.mark.parametrize("lattice,n,block,rd,seed", CASES)
def test_window_gradients_match_central_differences(lattice, n, block, rd, seed):
    sim, st, S0, rng = _setup(lattice, n, block, rd, seed, rseed=2)
    p = params_of(sim)
    D = sim.D
    a = rng.standard_normal(4 + 2 * D)
    a[:4 + D] = 0.0  # velocity observables only: the masses and the (constant) centroid would
    # make J ~ 50 and bury the small u~ and sigma effects in round-off
    nsteps = 2
    J, dp, lam0 = gradients(st, S0, p, nsteps, a)
    assert abs(J - objective(st, S0, p, nsteps, a)) < 1e-13 * max(1.0, abs(J))
    for kp in range(NPARAM):
        e = np.zeros(NPARAM)
        e[kp] = 1e-5 * abs(p[kp])
        fd = (objective(st, S0, p + e, nsteps, a) - objective(st, S0, p - e, nsteps, a)) / (2 * e[kp])
        assert abs(fd - dp[kp]) <= 1e-5 * abs(fd) + 1e-12, (kp, fd, dp[kp])
    # fourth-order central differences per part; u~ moves J little, so it takes a larger step
    for part, (eps, tol) in enumerate(((1e-4, 2e-5), (1e-5, 2e-5), (3e-3, 1e-4))):
        V = _dir(st, S0, rng, tuple(int(k == part) for k in range(3)))
        Jh = [objective(st, _axpy(S0, m * eps, V), p, nsteps, a) for m in (-2, -1, 1, 2)]
        fd = (Jh[0] - 8 * Jh[1] + 8 * Jh[2] - Jh[3]) / (12 * eps)
        assert abs(fd - _dot(V, lam0)) <= tol * abs(fd), (part, fd, _dot(V, lam0))


def test_pins_detect_a_dropped_ghost_adjoint(monkeypatch):
    """Planted: the finest sub-step's adjoint forgets the ghost-ring values it pulled."""
    import oracle.adjoint_ls as M
    orig = M.MovingStep.step_adjoint

    def bad(self, state, p, lam, lam_gh=None):
        return orig(self, state, p, lam, None if lam_gh is None else np.zeros_like(lam_gh))
    monkeypatch.setattr(M.MovingStep, "step_adjoint", bad)
    sim, st, S0, rng = _setup(*CASES[0])
    p = params_of(sim)
    V = _dir(st, S0, rng, (1, 0, 0))
    V = ([V[0][0], 0 * V[0][1]], V[1], V[2])  # coarse populations only
    W = ([rng.standard_normal(f.shape) for f in S0[0]], rng.standard_normal(S0[1].shape) * st.moving.band,
         rng.standard_normal(S0[2].shape))
    lam, _ = st.step_adjoint(S0, p, W)
    lhs, rhs = _dot(_jv(st, S0, p, V, 1e-5), W), _dot(V, lam)
    assert abs(lhs - rhs) > 1e-3 * abs(lhs), (lhs, rhs)
