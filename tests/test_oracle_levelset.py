"""Pins for oracle/levelset.py (Sec. 2.2): convergence orders, rigid rotation,
extension, constrained reinitialisation, least-squares curvature."""
import numpy as np
import pytest

from oracle import levelset
from oracle.grid import LevelGeom
from oracle.lattice import D2Q9, D3Q19


def _sine_err(N, a=0, D=1):
    dims = (N, 3) if D == 1 else (N, N)
    g = LevelGeom(dims, (True, True), dims)
    x = (g.coord[a] + 0.5) / N
    phi = np.sin(2 * np.pi * x)
    cells = np.arange(g.N)
    errs = []
    for side in (-1, 1):
        d = levelset.d5(g, phi, cells, a, side) * N
        errs.append(np.abs(d - 2 * np.pi * np.cos(2 * np.pi * x)).max())
    return max(errs)


def test_upwind5_is_fifth_order():
    e1, e2 = _sine_err(16), _sine_err(32)
    order = np.log2(e1 / e2)
    assert 4.7 < order < 5.5, order


def test_upwind5_weights_exact_for_quintics():
    g = LevelGeom((20, 1), (True, True), (20, 1))
    x = g.coord[0].astype(float)
    cells = np.arange(6, 14)
    for p in range(6):
        phi = x ** p
        want = p * x[cells] ** (p - 1) if p > 0 else 0 * cells
        for side in (-1, 1):
            assert np.allclose(levelset.d5(g, phi, cells, 0, side), want, rtol=1e-9, atol=1e-9)


def test_rk3_is_third_order():
    def run(dt):
        phi = np.array([1.0])
        for _ in range(int(round(1.0 / dt))):
            phi = levelset.rk3(phi, np.array([0]), lambda p: -p[[0]], dt)
        return abs(phi[0] - np.exp(-1.0))
    r = run(0.1) / run(0.05)
    assert 7.0 < r < 9.0


def test_rigid_rotation_return():
    N = 48
    g = LevelGeom((N, N), (False, False), (N, N))
    x = g.coord[0] + 0.5 - N / 2
    y = g.coord[1] + 0.5 - N / 2
    R, cx = 8.0, 10.0
    phi0 = np.sqrt((x - cx) ** 2 + y ** 2) - R
    T = 600
    om = 2 * np.pi / T
    ut = np.stack([-om * y, om * x])
    phi = phi0.copy()
    cells = np.arange(g.N)
    for _ in range(T):
        phi = levelset.advect(g, phi, ut, cells)
    # zero set returns: compare signs and the interface-cell values
    near = np.abs(phi0) < 2
    assert np.abs(phi[near] - phi0[near]).max() < 0.05
    assert (np.sign(phi[near]) == np.sign(phi0[near])).mean() > 0.99


def test_extension_constant_along_normals():
    N = 40
    g = LevelGeom((N, N), (False, False), (N, N))
    x = g.coord[0] + 0.5 - N / 2
    y = g.coord[1] + 0.5 - N / 2
    r = np.sqrt(x ** 2 + y ** 2)
    phi = r - 10.0
    th = np.arctan2(y, x)
    iface = levelset.frozen_cells(g, D2Q9, phi)
    ut = np.zeros((2, g.N))
    ut[0, iface] = np.cos(th[iface])
    ut[1, iface] = 0.0
    upd = np.flatnonzero((np.abs(phi) < 6) & ~iface)
    ut = levelset.extend(g, phi, ut, upd, 60, 0.5)
    band = (np.abs(phi) < 5) & ~iface
    err = np.abs(ut[0, band] - np.cos(th[band]))
    assert np.median(err) < 0.05 and err.max() < 0.25


def test_reinit_keeps_zero_set_and_restores_distance():
    N = 40
    g = LevelGeom((N, N), (False, False), (N, N))
    x = g.coord[0] + 0.5 - N / 2
    y = g.coord[1] + 0.5 - N / 2
    r = np.sqrt(x ** 2 + y ** 2)
    phi0 = (r - 10.3) * (1.0 + 0.6 * np.cos(3 * np.arctan2(y, x))) * 1.7
    band = np.ones(g.N, dtype=bool)
    phi = levelset.reinit(g, D2Q9, phi0, band, 60, 0.3)
    # every cut link keeps its zero crossing (frozen interface cells)
    fr = levelset.frozen_cells(g, D2Q9, phi0)
    assert np.array_equal(phi[fr], phi0[fr])
    assert np.array_equal(levelset.classify(phi), levelset.classify(phi0))
    # |grad phi| -> 1 away from the interface
    sel = (np.abs(r - 10.3) > 2) & (np.abs(r - 10.3) < 6)
    cells = np.flatnonzero(sel)
    gr = np.zeros(len(cells))
    for a in range(2):
        gr += (0.5 * (phi[g.clamp_shift(cells, np.eye(2, dtype=int)[a])]
                      - phi[g.clamp_shift(cells, -np.eye(2, dtype=int)[a])])) ** 2
    assert np.median(np.abs(np.sqrt(gr) - 1)) < 0.05


@pytest.mark.parametrize("D", [2, 3])
def test_fit_exact_on_quadratics(D):
    N = 7
    dims = (N,) * D
    g = LevelGeom(dims, (True,) * D, dims)
    rng = np.random.default_rng(4)
    b = rng.standard_normal(D)
    H = rng.standard_normal((D, D))
    H = H + H.T
    X = g.coord.astype(float) - 3
    phi = 0.3 + b @ X + 0.5 * np.einsum("an,ab,bn->n", X, H, X)
    c = g.flat(np.full((D, 1), 3))
    n, kap, grad, hess = levelset.fit_geometry(g, phi, c)
    assert np.allclose(grad[:, 0], b, atol=1e-12)
    assert np.allclose(hess[:, :, 0], H, atol=1e-12)
    want = ((b @ b) * np.trace(H) - b @ H @ b) / np.linalg.norm(b) ** 3
    assert abs(kap[0] - want) < 1e-10


@pytest.mark.parametrize("D", [2, 3])
def test_curvature_of_circle_sphere_converges(D):
    errs = []
    for R in (6.0, 12.0):
        N = int(2 * R + 8)
        dims = (N,) * D
        g = LevelGeom(dims, (False,) * D, dims)
        X = g.coord + 0.5 - N / 2
        r = np.sqrt((X ** 2).sum(0))
        phi = r - R
        lat = D2Q9 if D == 2 else D3Q19
        cells = np.flatnonzero(levelset.frozen_cells(g, lat, phi))
        n, kap, _, _ = levelset.fit_geometry(g, phi, cells)
        exact = (D - 1) / r[cells]
        errs.append(np.abs(kap - exact).max() * R)  # relative to 1/R
        assert np.allclose((n * X[:, cells] / r[cells]).sum(0), 1.0, atol=2e-2)
    assert errs[0] / errs[1] > 3.0, errs


def test_weno5_matches_upwind5_on_smooth_data_and_is_fifth_order():
    N = 64
    g = LevelGeom((N, 3), (True, True), (N, 3))
    x = (g.coord[0] + 0.5) / N
    phi = np.sin(2 * np.pi * x)
    cells = np.arange(g.N)
    for side in (-1, 1):
        w = levelset.weno5(g, phi, cells, 0, side)
        u = levelset.d5(g, phi, cells, 0, side)
        assert np.abs(w - u).max() < 1e-3 * np.abs(u).max()
    # exact on linear data, both sides
    phi = 3.0 * g.coord[0].astype(float)
    inner = np.flatnonzero((g.coord[0] > 3) & (g.coord[0] < N - 4))
    for side in (-1, 1):
        assert np.allclose(levelset.weno5(g, phi, inner, 0, side), 3.0, atol=1e-12)
