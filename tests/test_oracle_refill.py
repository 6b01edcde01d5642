"""Pins for the composition of the oracle's refill (Sec. 2.4, oracle/coupling.py).

A cell that changes phase gets the equilibrium of density and velocity
extrapolated along e_min from the interface point Gamma (at -q) and the nodes
x_r + e_min, x_r + 2 e_min of its new phase, plus the non-equilibrium part of
x_r + e_min.  The checks below build fields whose answer is known without the
oracle's formulas:

* the new phase's density and velocity are polynomials along e_min (degree 2
  when x_r + 2 e_min is usable, else degree 1) whose value at the interface
  point is what the normal stress balance demands: the old phase's pressure at
  x_r plus the Laplace jump sigma kappa_new (kappa_new = div of the new phase's
  outward normal), and the old phase's velocity (no slip across Gamma).  A
  Lagrange extrapolation of such a polynomial is exact, so the refilled cell
  must carry the polynomial's value at x_r, for any q and either branch;
* a static drop (constant pressures obeying p_gas - p_liquid = sigma (D-1)/R):
  a cell that flips either way must come back at the pressure of its new
  phase, which fixes the sign of the jump;
* a planted moment-free non-equilibrium part at x_r + e_min must be copied
  unchanged, and the one at x_r + 2 e_min must not be;
* a cell without a usable neighbour falls back to the rest state.

Mistakes planted in a copy of the oracle's refill (the sign of sigma kappa,
the whole populations copied instead of f^neq, the two extrapolation nodes
swapped, q taken on the wrong side) must fail these checks.
"""
import inspect
import textwrap
import types

import numpy as np
import pytest

from oracle import coupling
from oracle.grid import LevelGeom
from oracle.lattice import CS2, D2Q9, D3Q19
from oracle.lbm import equilibrium, moments


def _feq(lat, rho, u):
    return equilibrium(lat, np.array([float(rho)]), np.asarray(u, float)[:, None])[:, 0]


def _moment_free(lat, rng):
    """A random population vector with zero mass and zero momentum."""
    v = rng.standard_normal(lat.Q)
    A = np.vstack([np.ones(lat.Q), lat.cf.T])  # (1 + D, Q)
    v -= A.T @ np.linalg.solve(A @ A.T, A @ v)
    return 1e-3 * v


class Setup:
    """A box with a flat interface normal to axis 0 and one flipped cell x_r.

    The new phase occupies cells with coordinate 0 >= c (c = the centre cell's
    index); the old phase cells with coordinate 0 < c; x_r = the centre cell
    changed from the old to the new phase.  e_min is the unit vector +x.  The
    box ends after x_r + 2 e_min (quad) or after x_r + e_min (linear branch).
    """

    def __init__(self, lat, Pn, q, quad, rng, sigma, rp, kappa):
        D = lat.D
        self.lat, self.D = lat, D
        n = 7
        self.c = 3
        dims = (self.c + (3 if quad else 2),) + (n,) * (D - 1)
        self.g = LevelGeom(dims, (False,) * D, dims)
        g = self.g
        xr_co = np.array([self.c] + [n // 2] * (D - 1))
        self.xr = int(g.flat(xr_co.reshape(-1, 1))[0])
        Po = 1 - Pn
        x = g.coord[0]
        self.phase_new = np.where(x >= self.c, Pn, Po).astype(np.int64)
        self.phase_old = self.phase_new.copy()
        self.phase_old[self.xr] = Po
        self.fluid = np.ones(g.N, dtype=bool)
        # phi: linear in x with its zero at distance q behind x_r (between x_r - e and x_r);
        # phi < 0 liquid.  sgn = +1 where the new phase is gas.
        s = x.astype(float) - self.c  # position along e_min relative to x_r
        self.phi = (s + q) * (1.0 if Pn == 1 else -1.0)
        self.q = q
        # normal of the level set (points to the gas) and the given curvature at x_r
        self.nvec = np.zeros((D, g.N))
        self.nvec[0] = 1.0 if Pn == 1 else -1.0
        self.kappa = np.zeros(g.N)
        self.kappa[self.xr] = kappa
        self.prm = dict(rho_phys=np.asarray(rp, float), nu=np.array([0.1, 0.1]), sigma=sigma)
        self.Pn, self.Po = Pn, Po
        self.s = s
        self.rng = rng

    def kappa_new(self):
        """div of the new phase's outward normal: kappa (normal to the gas) for the liquid."""
        return self.kappa[self.xr] if self.Pn == 0 else -self.kappa[self.xr]


def _fields(st, deg, rho_o, u_o):
    """Old-phase state at x_r and new-phase polynomials along e_min meeting the interface
    conditions at Gamma (s = -q); returns f and the expected refilled (rho, u)."""
    lat, g, rng, q = st.lat, st.g, st.rng, st.q
    rp = st.prm["rho_phys"]
    p_old = rp[st.Po] * CS2 * (rho_o - 1.0)
    p_gamma = p_old + st.prm["sigma"] * st.kappa_new()  # normal stress balance at Gamma
    rho_gamma = 1.0 + p_gamma / (rp[st.Pn] * CS2)
    a_r, b_r = rng.uniform(-0.02, 0.02, 2)
    a_u, b_u = rng.uniform(-0.01, 0.01, (2, st.D))
    if deg == 1:
        b_r, b_u = 0.0, np.zeros(st.D)

    def rho_new(s):  # value rho_gamma at s = -q by construction
        return rho_gamma + a_r * (s + q) + b_r * (s + q) * (s - 1.0)

    def u_new(s):
        return u_o + a_u * (s + q) + b_u * (s + q) * (s - 1.0)

    # other axes: any smooth variation (extrapolation runs along e_min only)
    t = g.coord[1:].astype(float) - g.coord[1:, st.xr][:, None]
    f = np.zeros((lat.Q, g.N))
    for cell in range(g.N):
        s = st.s[cell]
        if st.phase_new[cell] == st.Pn and cell != st.xr:
            r = rho_new(s) + 0.003 * t[:, cell].sum()
            u = u_new(s) + 0.001 * t[:, cell].sum()
        else:
            r = rho_o + 0.002 * s + 0.001 * t[:, cell].sum()
            u = u_o + 0.002 * s
        f[:, cell] = _feq(lat, r, u)
    f[:, st.xr] = _feq(lat, rho_o, u_o)
    return f, rho_new(0.0), u_new(0.0)


def _run_refill(refill, st, f):
    f = f.copy()
    n_fail = refill(st.lat, st.g, f, np.array([st.xr]), st.phase_old, st.phase_new, st.fluid, st.phi,
                    st.nvec, st.kappa, st.prm)
    return f, n_fail


def check_polynomial_extrapolation(refill, lat, seed=0):
    rng = np.random.default_rng(seed)
    for trial in range(24):
        Pn = trial % 2
        quad = (trial // 2) % 2 == 0
        q = [0.05, 0.3, 0.5, 0.77, 0.999, 1.0][trial % 6]
        rp = (1.0, float(rng.uniform(0.001, 0.5)))
        st = Setup(lat, Pn, q, quad, rng, sigma=float(rng.uniform(0, 0.02)), rp=rp,
                   kappa=float(rng.uniform(-0.3, 0.3)))
        rho_o = 1.0 + rng.uniform(-0.01, 0.01)
        u_o = rng.uniform(-0.02, 0.02, lat.D)
        f, rho_want, u_want = _fields(st, 2 if quad else 1, rho_o, u_o)
        out, n_fail = _run_refill(refill, st, f)
        assert n_fail == 0
        want = _feq(lat, rho_want, u_want)
        assert np.abs(out[:, st.xr] - want).max() < 1e-13, (trial, out[:, st.xr] - want)


def check_laplace_jump_sign(refill, lat):
    """Static drop: gas pressure sigma (D-1)/R above the liquid's; kappa = -(D-1)/R for a
    gas bubble (normal to the gas points inwards).  Either flip must land on the new
    phase's pressure."""
    D = lat.D
    R, sigma = 6.0, 0.01
    rp = (1.0, 0.01)
    kappa = -(D - 1) / R
    p_l, p_g = 0.0, sigma * (D - 1) / R
    rng = np.random.default_rng(3)
    for Pn in (0, 1):
        st = Setup(lat, Pn, 0.4, True, rng, sigma=sigma, rp=rp, kappa=kappa)
        rho_of = {0: 1.0 + p_l / (rp[0] * CS2), 1: 1.0 + p_g / (rp[1] * CS2)}
        f = np.zeros((lat.Q, st.g.N))
        for cell in range(st.g.N):
            ph = st.phase_old[cell]
            f[:, cell] = lat.w * rho_of[int(ph)]
        out, _ = _run_refill(refill, st, f)
        rho, u = moments(lat, out[:, [st.xr]])
        assert abs(rho[0] - rho_of[Pn]) < 1e-13, (Pn, rho[0], rho_of[Pn])
        assert np.abs(u).max() < 1e-13


def check_fneq_copy(refill, lat):
    rng = np.random.default_rng(4)
    for Pn in (0, 1):
        st = Setup(lat, Pn, 0.6, True, rng, sigma=0.0, rp=(1.0, 1.0), kappa=0.0)
        f, rho_want, u_want = _fields(st, 2, 1.0, np.zeros(lat.D))
        g1 = _moment_free(lat, rng)
        g2 = _moment_free(lat, rng)
        a1 = int(st.g.shift(np.array([st.xr]), np.eye(lat.D, dtype=np.int64)[0])[0][0])
        a2 = int(st.g.shift(np.array([st.xr]), 2 * np.eye(lat.D, dtype=np.int64)[0])[0][0])
        f[:, a1] += g1
        f[:, a2] += g2
        out, _ = _run_refill(refill, st, f)
        got = out[:, st.xr] - _feq(lat, rho_want, u_want)
        assert np.abs(got - g1).max() < 1e-14, (Pn, got - g1)


CHECKS = (check_polynomial_extrapolation, check_laplace_jump_sign, check_fneq_copy)


@pytest.mark.parametrize("lat", [D2Q9, D3Q19], ids=lambda l: l.name)
@pytest.mark.parametrize("check", CHECKS, ids=lambda c: c.__name__)
def test_refill_composition(lat, check):
    check(coupling.refill, lat)


@pytest.mark.parametrize("lat", [D2Q9, D3Q19], ids=lambda l: l.name)
def test_refill_without_usable_neighbour_is_rest_state(lat):
    D = lat.D
    g = LevelGeom((3,) * D, (False,) * D, (3,) * D)
    xr = int(g.flat(np.ones((D, 1), dtype=np.int64))[0])
    phase_old = np.zeros(g.N, dtype=np.int64)
    phase_new = phase_old.copy()
    phase_new[xr] = 1  # the only gas cell: no neighbour of the new phase
    f = np.tile(lat.w[:, None], (1, g.N)) * 1.01
    n_fail = coupling.refill(lat, g, f, np.array([xr]), phase_old, phase_new, np.ones(g.N, bool),
                             np.where(phase_new == 1, 0.5, -0.5).astype(float), np.zeros((D, g.N)),
                             np.zeros(g.N), dict(rho_phys=np.array([1.0, 0.1]), nu=np.array([0.1, 0.1]),
                                                 sigma=0.0))
    assert n_fail == 1
    assert np.array_equal(f[:, xr], lat.w)


def _mutant(func, old, new):
    """A copy of ``func`` with one source fragment replaced (a planted mistake)."""
    src = textwrap.dedent(inspect.getsource(func))
    assert src.count(old) == 1, f"fragment not found once in {func.__name__}: {old!r}"
    ns = dict(func.__globals__)
    exec(compile(src.replace(old, new), inspect.getsourcefile(func), "exec"), ns)
    return ns[func.__name__]


PLANTS = {
    "sigma_kappa_sign": ('+ prm["sigma"] * sg * kappa[xr]', '- prm["sigma"] * sg * kappa[xr]'),
    "f_instead_of_fneq": ("fneq = f_new[:, a1[0]] - equilibrium(lat, r1, u1)[:, 0]", "fneq = f_new[:, a1[0]]"),
    "nodes_swapped": ("w0, w1, w2 = extrapolation_weights(q, quad)", "w0, w2, w1 = extrapolation_weights(q, quad)"),
    "q_wrong_side": ("b, _ = geom.shift(np.array([xr]), -ce)", "b, _ = geom.shift(np.array([xr]), ce)"),
    "density_ratio_dropped": ("rho_g = 1.0 + p_gamma / (rp[Pn] * CS2)", "rho_g = 1.0 + p_gamma / CS2"),
}


@pytest.mark.parametrize("plant", sorted(PLANTS))
def test_refill_checks_detect_a_planted_mistake(plant):
    bad = _mutant(coupling.refill, *PLANTS[plant])
    failed = 0
    for lat in (D2Q9, D3Q19):
        for check in CHECKS:
            try:
                check(bad, lat)
            except AssertionError:
                failed += 1
    assert failed > 0, plant


def test_mutant_helper_reproduces_the_oracle():
    same = _mutant(coupling.refill, "n_fail = 0", "n_fail = 0")
    for check in CHECKS:
        check(same, D2Q9)
    assert isinstance(same, types.FunctionType)
