"""Smoothed-indicator observables for the adjoint objective (Sec. 3.2 integrals).

Test infrastructure (like the rest of ``oracle``): only the tests, the smoke
check and the benchmark's CPU baseline use it.

Sec. 3.2 measures the bubble by integrals over the gas region: its volume, its
centroid (the gas-weighted mean position) and its rise velocity (the
gas-weighted mean velocity).  Weighted by the sharp indicator [phi >= 0] these
are piecewise constant in phi, so their derivatives with respect to anything
that moves the interface vanish between cell flips.  The adjoint objective
weights them instead by the smoothed indicator (the reading of the proposed
scope's c21)

    H_eps(phi) = 0                                   phi < -eps
               = 1/2 (1 + phi/eps + sin(pi phi/eps)/pi)   |phi| <= eps
               = 1                                   phi > eps,

with eps given in finest cells (1.5 by default).  The masses stay phase sums:
each cell carries the populations of one phase, so a phase's mass is the sum of
its own cells' densities.  A coarser level's leaf takes phi at its first finest
child, the point the phases are classified at.

Observables in the library's order: liquid mass, gas mass, gas volume, leaf
updates per coarse step, centroid (D), gas velocity (D); volumes in finest
cells.

Pins (tests/test_oracle_objective.py): H_eps's closed-form properties (value
1/2 at the interface, H(phi) + H(-phi) = 1, unit integral of its derivative,
continuity at +-eps), the smoothed volume of a disk and a sphere converging to
pi R^2 and 4/3 pi R^3, the sharp limit eps -> 0, and the adjoint against
central differences in phi and f.
"""
import numpy as np

from .lbm import moments

EPS_DEFAULT = 1.5


def heaviside(phi, eps):
    """H_eps(phi) (smoothed gas indicator)."""
    phi = np.asarray(phi, dtype=np.float64)
    t = np.clip(phi / eps, -1.0, 1.0)
    return np.where(phi > eps, 1.0, np.where(phi < -eps, 0.0, 0.5 * (1.0 + t + np.sin(np.pi * t) / np.pi)))


def dheaviside(phi, eps):
    """d H_eps / d phi."""
    phi = np.asarray(phi, dtype=np.float64)
    inside = np.abs(phi) <= eps
    return np.where(inside, 0.5 / eps * (1.0 + np.cos(np.pi * np.clip(phi / eps, -1.0, 1.0))), 0.0)


def levels_of(sim):
    """Per level of a Sim: leaf mask, phases, grid ratio r, cell centres (finest units) and
    the finest cell each leaf reads phi at."""
    gF = sim.geoms[-1]
    out = []
    for l, g in enumerate(sim.geoms):
        r = 2 ** (sim.L - 1 - l)
        out.append(dict(leaf=sim.masks[l][0].copy(), phase=sim.phase[l].copy(), r=float(r),
                        centers=g.centers(float(r)), corner=gF.flat(g.coord * r), nupd=2.0 ** l))
    return out


def observables(lat, levels, F, phi, eps):
    """The observables with H_eps weights for volume, centroid and velocity."""
    D = lat.D
    mass = np.zeros(2)
    vol, nupd = 0.0, 0.0
    xs, us = np.zeros(D), np.zeros(D)
    for lv, f in zip(levels, F):
        leaf = lv["leaf"]
        v = lv["r"] ** D
        rho, u = moments(lat, f[:, leaf])
        ph = lv["phase"][leaf]
        for s in (0, 1):
            mass[s] += v * rho[ph == s].sum()
        h = heaviside(phi[lv["corner"][leaf]], eps)
        vol += v * h.sum()
        nupd += leaf.sum() * lv["nupd"]
        xs += v * (lv["centers"][:, leaf] * h[None, :]).sum(1)
        us += v * (u * h[None, :]).sum(1)
    return np.concatenate([mass, [vol, nupd], xs / vol, us / vol])


def observables_adjoint(lat, levels, F, phi, eps, a):
    """dJ/dF (per level) and dJ/dphi (finest level) for J = a . observables(F, phi)."""
    D = lat.D
    a = np.asarray(a, dtype=np.float64)
    obs = observables(lat, levels, F, phi, eps)
    V, X, U = obs[2], obs[4:4 + D], obs[4 + D:4 + 2 * D]
    aV, aX, aU = a[2], a[4:4 + D], a[4 + D:4 + 2 * D]
    lphi = np.zeros_like(phi, dtype=np.float64)
    lamF = []
    for lv, f in zip(levels, F):
        leaf = lv["leaf"]
        v = lv["r"] ** D
        lam = np.zeros_like(f)
        rho, u = moments(lat, f[:, leaf])
        ph = lv["phase"][leaf]
        cells = np.flatnonzero(leaf)
        lam[:, cells[ph == 0]] += v * a[0]
        lam[:, cells[ph == 1]] += v * a[1]
        pc = phi[lv["corner"][leaf]]
        h = heaviside(pc, eps)
        # velocity: d u_a / d f_j = (c_ja - u_a) / rho, weight v h / V
        lam[:, cells] += v * h[None, :] * ((lat.cf @ aU)[:, None] - (aU @ u)[None, :]) / rho[None, :] / V
        # phi through H at the cell: volume, centroid (X = sum x h v / V) and velocity (U likewise)
        dh = dheaviside(pc, eps)
        g = v * dh * (aV + (aX @ (lv["centers"][:, leaf] - X[:, None])) / V + (aU @ (u - U[:, None])) / V)
        np.add.at(lphi, lv["corner"][leaf], g)
        lamF.append(lam)
    return lamF, lphi
