"""Pins for oracle/adjoint_amr.py: the frozen-interface adjoint of a two-level coarse step.

As for one level, the transposed step is checked against the forward oracle
itself: AMRFrozenStep.step must be Sim.step; the dot-product identity
<J v, w> = <v, J^T w> of one coarse step with J v from central differences
must hold for perturbations of either level; every parameter partial, window
gradients in the parameters, the initial populations and the finest level
set must match central differences of the float64 objective.  The layouts
hold coarse leaves, a restriction layer and a fine ghost ring, so every
transfer (restriction with its tau ratio, ghost interpolation at t and
t + 1/2 with its tau ratio and fine collision) lies on the checked paths.
"""
import numpy as np
import pytest

from oracle import adjoint as single
from oracle.adjoint_amr import NPARAM, AMRFrozenStep, gradients, objective, params_of
from oracle.lbm import equilibrium
from oracle.sim import Sim
from paper_2601_05936_gb300 import workloads

CASES = [("D2Q9", (48, 24), (8, 8), 4.0), ("D3Q19", (12, 8, 12), (4, 4, 4), 2.0)]
# refinement distances below a cell: parts of the interface stay on coarse leaves, where a
# link into the other phase takes plain bounce-back
CUT_CASES = [("D2Q9", (48, 24), (8, 8), 0.2), ("D3Q19", (12, 8, 12), (4, 4, 4), 0.2)]


def _case(lattice, n, block, rd):
    return workloads.adjoint_window(lattice, n=n, levels=2, block=block, refine_dist=rd)


def _setup(lattice, n, block, rd, seed=1):
    sim = Sim(_case(lattice, n, block, rd))
    st = AMRFrozenStep(sim)
    rng = np.random.default_rng(seed)
    lat = sim.lat
    F0 = []
    for f in sim.f:
        N = f.shape[1]
        rho = 1.0 + 0.01 * rng.standard_normal(N)
        u = 0.02 * rng.standard_normal((lat.D, N))
        F0.append(equilibrium(lat, rho, u) + 1e-3 * rng.standard_normal((lat.Q, N)) * lat.w[:, None])
    return sim, st, F0, rng


def _axpy(F, eps, V):
    return [a + eps * b for a, b in zip(F, V)]


def _dot(A, B):
    return sum(float((a * b).sum()) for a, b in zip(A, B))


@pytest.mark.parametrize("lattice,n,block,rd", CASES + CUT_CASES)
def test_amr_step_is_the_oracle_step(lattice, n, block, rd):
    sim = Sim(_case(lattice, n, block, rd))
    leaf0, _, rl0, _ = sim.masks[0]
    ghost1 = sim.masks[1][3]
    assert leaf0.sum() > 0 and rl0.sum() > 0 and ghost1.sum() > 0
    st = AMRFrozenStep(sim)
    F, p = [f.copy() for f in sim.f], params_of(sim)
    for _ in range(3):
        F = st.step(F, p)
    sim.step(3)
    assert (sim.stats["coarse_cut"] > 0) == (rd < 1.0)
    for a, b in zip(F, sim.f):
        assert np.abs(a - b).max() < 1e-14
    obs = sim.observables()
    mine = st.observables(F)
    D = sim.D
    assert np.allclose(mine[:2], obs["mass"], rtol=1e-14) and mine[2] == obs["volume"]
    assert np.allclose(mine[4:4 + D], obs["centroid"], rtol=1e-14)
    vel = obs["velocity"]
    assert np.allclose(mine[4 + D:], vel, rtol=1e-12, atol=1e-12 * np.abs(vel).max())


@pytest.mark.parametrize("part", ["all", "coarse", "fine"])
@pytest.mark.parametrize("lattice,n,block,rd", CASES + CUT_CASES)
def test_dot_product_identity_one_coarse_step(lattice, n, block, rd, part):
    sim, st, F0, rng = _setup(lattice, n, block, rd)
    p = params_of(sim)
    keep = {"all": (1, 1), "coarse": (1, 0), "fine": (0, 1)}[part]
    V = [k * 1e-3 * rng.standard_normal(f.shape) for k, f in zip(keep, F0)]
    W = [rng.standard_normal(f.shape) for f in F0]
    eps = 1e-4
    Fp, Fm = st.step(_axpy(F0, eps, V), p), st.step(_axpy(F0, -eps, V), p)
    lhs = _dot([(a - b) / (2 * eps) for a, b in zip(Fp, Fm)], W)
    lam, dp = st.step_adjoint(F0, p, W)
    rhs = _dot(V, lam)
    assert abs(lhs - rhs) <= 1e-8 * abs(lhs), (lhs, rhs)
    if part == "all":
        for kp in range(NPARAM):
            e = np.zeros(NPARAM)
            e[kp] = 1e-5 * abs(p[kp])
            Fp, Fm = st.step(F0, p + e), st.step(F0, p - e)
            ref = _dot([(a - b) / (2 * e[kp]) for a, b in zip(Fp, Fm)], W)
            assert abs(ref - dp[kp]) <= 1e-6 * abs(ref), (kp, ref, dp[kp])


@pytest.mark.parametrize("lattice,n,block,rd", CASES)
def test_window_gradients_match_central_differences(lattice, n, block, rd):
    sim, st, F0, rng = _setup(lattice, n, block, rd, seed=2)
    p = params_of(sim)
    D = sim.D
    a = rng.standard_normal(4 + 2 * D)
    a[4 + D:] *= 100.0
    nsteps = 3
    J, dp, lam0 = gradients(st, F0, p, nsteps, a)
    assert abs(J - objective(st, F0, p, nsteps, a)) < 1e-13 * max(1.0, abs(J))
    for kp in range(NPARAM):
        e = np.zeros(NPARAM)
        e[kp] = 1e-5 * abs(p[kp])
        fd = (objective(st, F0, p + e, nsteps, a) - objective(st, F0, p - e, nsteps, a)) / (2 * e[kp])
        assert abs(fd - dp[kp]) <= 2e-5 * abs(fd) + 1e-12, (kp, fd, dp[kp])
    # fourth-order central differences along a random direction of both levels
    V = [1e-3 * rng.standard_normal(f.shape) for f in F0]
    eps = 1e-3
    Jh = [objective(st, _axpy(F0, m * eps, V), p, nsteps, a) for m in (-2, -1, 1, 2)]
    fd = (Jh[0] - 8 * Jh[1] + 8 * Jh[2] - Jh[3]) / (12 * eps)
    assert abs(fd - _dot(V, lam0)) <= 1e-6 * abs(fd), (fd, _dot(V, lam0))


def test_level_set_gradient_on_the_finest_level():
    """dJ/dphi of the finest level's frozen level set through q, n and kappa."""
    sim, st, F0, rng = _setup(*CASES[0], seed=5)
    p = params_of(sim)
    a = rng.standard_normal(8)
    a[6:] *= 100.0
    nsteps = 2
    _, _, _, dphi = gradients(st, F0, p, nsteps, a, want_phi=True)
    fine = st.fine
    near = np.zeros(fine.g.N, dtype=bool)
    for o in np.array(np.meshgrid(*[[-1, 0, 1]] * 2, indexing="ij")).reshape(2, -1).T:
        near[fine.g.clamp_shift(fine.icells, o)] = True
    assert np.abs(dphi[~near]).max() == 0.0
    phi = fine.phi
    for _ in range(2):
        v = rng.standard_normal(fine.g.N) * near
        eps = 1e-3 * np.abs(phi[near]).min() / np.abs(v).max()
        Jp = objective(AMRFrozenStep(sim, phi + eps * v), F0, p, nsteps, a)
        Jm = objective(AMRFrozenStep(sim, phi - eps * v), F0, p, nsteps, a)
        fd = (Jp - Jm) / (2 * eps)
        assert abs(fd - (dphi * v).sum()) <= 1e-5 * abs(fd), (fd, (dphi * v).sum())


def test_single_level_reduces_to_the_frozen_adjoint():
    case = workloads.adjoint_window("D2Q9", n=(32, 24))
    sim = Sim(case)
    sim.step(3)
    p = params_of(sim)
    a = np.random.default_rng(0).standard_normal(8)
    J1, dp1, lam1 = single.gradients(single.FrozenStep(sim), sim.f[0], p, 4, a)
    J2, dp2, lam2 = gradients(AMRFrozenStep(sim), [sim.f[0]], p, 4, a)
    assert J1 == J2
    assert np.array_equal(dp1, dp2) and np.array_equal(lam1, lam2[0])


@pytest.mark.parametrize("plant", ["restriction_without_rescale", "mid_ghost_weight",
                                   "interpolation_delta_sign", "ghost_tau_ratio_constant"])
def test_pins_detect_a_planted_mistake(monkeypatch, plant):
    """Mistakes planted in the transposed transfers alone break the one-step checks."""
    import oracle.adjoint_amr as M
    if plant == "restriction_without_rescale":
        def bad(self, l, Ff, p, lam_rl, dp):
            t = self.tr[l]
            out = np.zeros_like(Ff)
            for j in range(t["ch"].shape[0]):
                out[:, t["ch"][j]] += lam_rl / t["ch"].shape[0]
            return out
        monkeypatch.setattr(M.AMRFrozenStep, "_restrict_T", bad)
    elif plant == "mid_ghost_weight":
        orig = M.AMRFrozenStep._ghost_T
        calls = []

        def bad(self, l, F, p, lam_gh, dp):
            calls.append(1)
            out = orig(self, l, F, p, lam_gh, dp)
            return 2.0 * out if len(calls) % 2 == 1 else out  # the t + 1/2 transfer comes first
        monkeypatch.setattr(M.AMRFrozenStep, "_ghost_T", bad)
    elif plant == "interpolation_delta_sign":
        orig = M.interpolate_T

        def bad(gc, gf, usable, fine_cells, lam, Nc):
            full = orig(gc, gf, usable, fine_cells, lam, Nc)
            par = M.amr.parent_cells(gc, gf, fine_cells)
            base = np.zeros_like(full)
            for q in range(lam.shape[0]):
                np.add.at(base[q], par, lam[q])
            return 2 * base - full  # every gradient term with the opposite sign
        monkeypatch.setattr(M, "interpolate_T", bad)
    else:
        orig = M.AMRFrozenStep._fac_g

        def bad(self, l, ph, p):
            fac, _ = orig(self, l, ph, p)
            return fac, 0.0 * fac
        monkeypatch.setattr(M.AMRFrozenStep, "_fac_g", bad)
    sim, st, F0, rng = _setup(*CASES[0])
    p = params_of(sim)
    V = [1e-3 * rng.standard_normal(f.shape) for f in F0]
    W = [rng.standard_normal(f.shape) for f in F0]
    eps = 1e-4
    Fp, Fm = st.step(_axpy(F0, eps, V), p), st.step(_axpy(F0, -eps, V), p)
    lhs = _dot([(a - b) / (2 * eps) for a, b in zip(Fp, Fm)], W)
    lam, dp = st.step_adjoint(F0, p, W)
    bad_f = abs(lhs - _dot(V, lam)) > 1e-6 * abs(lhs)  # a hundred times the identity test's tolerance
    bad_p = False
    for kp in (3, 4):
        e = np.zeros(NPARAM)
        e[kp] = 1e-5 * abs(p[kp])
        ref = _dot([(a - b) / (2 * e[kp]) for a, b in zip(st.step(F0, p + e), st.step(F0, p - e))], W)
        bad_p |= abs(ref - dp[kp]) > 1e-4 * abs(ref)
    assert bad_f or bad_p
