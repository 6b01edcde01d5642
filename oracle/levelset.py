"""Level-set transport, velocity extension, reinitialisation and geometry (Sec. 2.2).

Sign convention (Sec. 2.2, first equation): phi < 0 liquid, phi > 0 gas; a
node with phi == 0 exactly is counted as gas (liquid iff phi < 0), matching
the stratified-flow statement "y < 0 fluid 1, y >= 0 fluid 2" (Sec. 3.1).

Readings of passages that the paper leaves open (all parameters are inputs):

* "fifth-order upwind-central" space scheme: the linear fifth-order
  upwind-biased first derivative with weights (-2, 15, -60, 20, 30, -3)/60 on
  offsets -3..+2 (mirrored when the velocity component is negative), applied
  axis by axis; time: Shu-Osher TVD-RK3 with dt = 1 lattice step.
* narrow band: the finest-level blocks that hold an interface cell plus their
  3^D block neighbours; phi outside the band is not updated.
* hyperbolic extension (Eq. hyperbolicExtension): interface cells hold the
  mean interface velocity u_I of their cut links (Dirichlet data); the other
  band cells take ``n_ext`` explicit-Euler Jacobi sweeps of first-order
  upwind differences with pseudo step ``dtau_ext``, S(phi) = phi/sqrt(phi^2+1),
  n from central differences.  The field persists between steps (warm start).
* constrained reinitialisation: phi_tau + S(phi0)(|grad phi|_G - 1) = 0 with
  Godunov's upwind Hamiltonian on fifth-order one-sided derivatives, taken
  with the Hamilton-Jacobi WENO5 weighting of Jiang & Peng (2000) (its linear
  weights give the same fifth-order upwind stencil as the transport; the
  nonlinear weights keep the kinks of a distance function from blowing up),
  smoothness epsilon 1e-6, integrated with TVD-RK3 in pseudo time; cells that have a sign change to any
  lattice neighbour are frozen, which keeps every link's zero crossing, hence
  the discrete zero set, exactly invariant.
* geometry: unweighted least-squares fit of a full quadratic over the 3^D
  stencil (library lstsq), n = g/|g|, kappa = (|g|^2 tr H - g.H.g)/|g|^3
  (= div(grad phi/|grad phi|)).
* Stencil points outside a walled box take the value of the nearest cell in
  the box (clamped index); periodic axes wrap.

Pins (tests/test_oracle_levelset.py): fifth- and third-order convergence on a
periodic sine, rigid-rotation return of a disk, extension constancy along
normals, reinit zero-set invariance and |grad phi| -> 1, circle/sphere
curvature (D-1)/R with O(dx^2) error, exactness of the fit on quadratics.
"""
import itertools

import numpy as np

W5 = np.array([-2.0, 15.0, -60.0, 20.0, 30.0, -3.0]) / 60.0
OFF5 = np.arange(-3, 3)


def _unit(D, a, s):
    e = np.zeros(D, dtype=np.int64)
    e[a] = s
    return e


def d5(geom, phi, cells, a, side):
    """Fifth-order one-sided derivative along axis a at ``cells``.

    side = -1: left-biased (upwind for a positive velocity), offsets -3..+2.
    side = +1: mirror image, offsets +3..-2 with negated weights.
    """
    out = np.zeros(len(cells))
    for wgt, o in zip(W5, OFF5):
        nb = geom.clamp_shift(cells, _unit(geom.D, a, -side * o))
        out += wgt * phi[nb]
    return -side * out


def advect_rhs(geom, phi, ut, cells):
    """L(phi) = -u~ . grad phi with upwind-biased fifth-order derivatives."""
    rhs = np.zeros(len(cells))
    for a in range(geom.D):
        ua = ut[a, cells]
        dm = d5(geom, phi, cells, a, -1)
        dp = d5(geom, phi, cells, a, +1)
        rhs -= ua * np.where(ua >= 0.0, dm, dp)
    return rhs


def rk3(phi, cells, rhs_fn, dt):
    """Shu-Osher TVD-RK3; only ``cells`` change, the rest keep phi."""
    p0 = phi.copy()
    p1 = p0.copy()
    p1[cells] = p0[cells] + dt * rhs_fn(p0)
    p2 = p0.copy()
    p2[cells] = 0.75 * p0[cells] + 0.25 * (p1[cells] + dt * rhs_fn(p1))
    p3 = p0.copy()
    p3[cells] = p0[cells] / 3.0 + (2.0 / 3.0) * (p2[cells] + dt * rhs_fn(p2))
    return p3


def advect(geom, phi, ut, band_cells, dt=1.0):
    """Level-set transport d phi/dt + u~ . grad phi = 0 on the band (Sec. 2.2)."""
    return rk3(phi, band_cells, lambda p: advect_rhs(geom, p, ut, band_cells), dt)


def central_normal(geom, phi, cells):
    """n = grad phi / |grad phi| from central differences (0 where |grad phi| = 0)."""
    g = np.zeros((geom.D, len(cells)))
    for a in range(geom.D):
        g[a] = 0.5 * (phi[geom.clamp_shift(cells, _unit(geom.D, a, 1))]
                      - phi[geom.clamp_shift(cells, _unit(geom.D, a, -1))])
    mag = np.sqrt((g * g).sum(0))
    return np.where(mag > 0.0, g / np.where(mag > 0.0, mag, 1.0), 0.0)


def extend(geom, phi, ut, upd_cells, n_iter, dtau):
    """Eq. hyperbolicExtension: d u~/d tau + S(phi) n . grad u~ = 0.

    First-order upwind in space, explicit Euler in pseudo time, Jacobi sweeps
    over ``upd_cells`` (band cells that are not interface cells).
    """
    ut = ut.copy()
    if len(upd_cells) == 0:
        return ut
    n = central_normal(geom, phi, upd_cells)
    s = phi[upd_cells] / np.sqrt(phi[upd_cells] ** 2 + 1.0)
    v = s[None, :] * n
    lo = [geom.clamp_shift(upd_cells, _unit(geom.D, a, -1)) for a in range(geom.D)]
    hi = [geom.clamp_shift(upd_cells, _unit(geom.D, a, 1)) for a in range(geom.D)]
    for _ in range(n_iter):
        old = ut.copy()
        acc = np.zeros((geom.D, len(upd_cells)))
        for a in range(geom.D):
            back = old[:, upd_cells] - old[:, lo[a]]
            fwd = old[:, hi[a]] - old[:, upd_cells]
            acc += v[a][None, :] * np.where(v[a][None, :] > 0.0, back, fwd)
        ut[:, upd_cells] = old[:, upd_cells] - dtau * acc
    return ut


WENO_EPS = 1e-6


def weno5(geom, phi, cells, a, side):
    """HJ-WENO5 one-sided derivative (Jiang & Peng 2000) along axis a.

    side = -1 uses the differences phi[j] - phi[j-1] around the cell leaning
    left (D^-); side = +1 is the mirror image (D^+).
    """
    e = lambda o: phi[geom.clamp_shift(cells, _unit(geom.D, a, -side * o))]
    p = [e(o) for o in range(-3, 3)]  # p[m] = phi at offset (m-3) on the upwind side
    v = [(-side) * (p[m + 1] - p[m]) for m in range(5)]
    v1, v2, v3, v4, v5 = v
    d1 = v1 / 3.0 - 7.0 * v2 / 6.0 + 11.0 * v3 / 6.0
    d2 = -v2 / 6.0 + 5.0 * v3 / 6.0 + v4 / 3.0
    d3 = v3 / 3.0 + 5.0 * v4 / 6.0 - v5 / 6.0
    s1 = 13.0 / 12.0 * (v1 - 2 * v2 + v3) ** 2 + 0.25 * (v1 - 4 * v2 + 3 * v3) ** 2
    s2 = 13.0 / 12.0 * (v2 - 2 * v3 + v4) ** 2 + 0.25 * (v2 - v4) ** 2
    s3 = 13.0 / 12.0 * (v3 - 2 * v4 + v5) ** 2 + 0.25 * (3 * v3 - 4 * v4 + v5) ** 2
    a1 = 0.1 / (s1 + WENO_EPS) ** 2
    a2 = 0.6 / (s2 + WENO_EPS) ** 2
    a3 = 0.3 / (s3 + WENO_EPS) ** 2
    return (a1 * d1 + a2 * d2 + a3 * d3) / (a1 + a2 + a3)


def reinit_rhs(geom, phi, s0, cells):
    """-S(phi0) (|grad phi|_G - 1) with Godunov's upwind Hamiltonian."""
    g2 = np.zeros(len(cells))
    pos = s0 > 0.0
    for a in range(geom.D):
        dm = weno5(geom, phi, cells, a, -1)
        dp = weno5(geom, phi, cells, a, +1)
        gp = np.maximum(np.maximum(dm, 0.0) ** 2, np.minimum(dp, 0.0) ** 2)
        gn = np.maximum(np.minimum(dm, 0.0) ** 2, np.maximum(dp, 0.0) ** 2)
        g2 += np.where(pos, gp, gn)
    return -s0 * (np.sqrt(g2) - 1.0)


def frozen_cells(geom, lat, phi):
    """Cells whose sign (phi >= 0) differs from a lattice neighbour in the box."""
    gas = phi >= 0.0
    allc = np.arange(geom.N)
    fr = np.zeros(geom.N, dtype=bool)
    for i in range(lat.Q):
        if i == lat.rest:
            continue
        nb, _ = geom.shift(allc, lat.c[i])
        ok = nb >= 0
        fr[ok] |= gas[ok] != gas[nb[ok]]
    return fr


def reinit(geom, lat, phi, band_mask, n_steps, dtau):
    """Constrained reinitialisation (Sec. 2.2, Hartmann et al.); reading above."""
    frozen = frozen_cells(geom, lat, phi)
    cells = np.flatnonzero(band_mask & ~frozen)
    if len(cells) == 0 or n_steps == 0:
        return phi.copy()
    s0 = phi[cells] / np.sqrt(phi[cells] ** 2 + 1.0)
    out = phi
    for _ in range(n_steps):
        out = rk3(out, cells, lambda p: reinit_rhs(geom, p, s0, cells), dtau)
    return out


def _quad_design(D):
    offs = np.array(list(itertools.product(*([(-1, 0, 1)] * D))), dtype=np.float64)
    cols = [np.ones(len(offs))] + [offs[:, a] for a in range(D)]
    cols += [offs[:, a] ** 2 for a in range(D)]
    pairs = [(a, b) for a in range(D) for b in range(a + 1, D)]
    cols += [offs[:, a] * offs[:, b] for a, b in pairs]
    return offs.astype(np.int64), np.stack(cols, 1), pairs


def fit_geometry(geom, phi, cells):
    """n and kappa from a least-squares quadratic over the 3^D stencil (Sec. 2.2).

    Returns (n (D, M), kappa (M,), grad (D, M), hess (D, D, M)).
    """
    D = geom.D
    offs, A, pairs = _quad_design(D)
    cells = np.asarray(cells, dtype=np.int64)
    if len(cells) == 0:
        return np.zeros((D, 0)), np.zeros(0), np.zeros((D, 0)), np.zeros((D, D, 0))
    vals = np.stack([phi[geom.clamp_shift(cells, o)] for o in offs])  # (3^D, M)
    coef, *_ = np.linalg.lstsq(A, vals, rcond=None)
    g = coef[1:1 + D]
    H = np.zeros((D, D, len(cells)))
    for a in range(D):
        H[a, a] = 2.0 * coef[1 + D + a]
    for k, (a, b) in enumerate(pairs):
        H[a, b] = H[b, a] = coef[1 + 2 * D + k]
    g2 = (g * g).sum(0)
    mag = np.sqrt(g2)
    ok = mag > 1e-12
    safe = np.where(ok, mag, 1.0)
    trH = np.trace(H)
    gHg = np.einsum("an,abn,bn->n", g, H, g)
    kappa = np.where(ok, (g2 * trH - gHg) / safe ** 3, 0.0)
    n = np.where(ok[None, :], g / safe[None, :], 0.0)
    return n, kappa, g, H


def classify(phi):
    """Phase per cell: 0 liquid (phi < 0), 1 gas (phi >= 0)."""
    return (phi >= 0.0).astype(np.int8)
