"""Lattice Boltzmann core: moments, equilibrium, BGK collision, forcing (Sec. 2.1).

Arrays: populations ``f`` have shape (Q, N) (N cells, flat, x fastest); vectors
(D, N).  Everything float64.

Pins (tests/test_oracle_lbm.py): equilibrium moments (rho, rho u, rho u u + c_s^2
rho I) checked against their closed forms; collision conserves mass exactly and
changes momentum by exactly rho*a; the single-phase Poiseuille and Couette
channels converge to their closed-form profiles, which fixes omega(nu), the
forcing sign and the moving-wall sign.
"""
import numpy as np

from .lattice import CS2


def omega_from_nu(nu):
    """Eq. omega with dt = 1: omega = c_s^2 / (nu + c_s^2 / 2)."""
    return CS2 / (nu + 0.5 * CS2)


def moments(lat, f):
    """Eq. macro: rho = sum_i f_i, u = sum_i c_i f_i / rho (no half-force shift)."""
    rho = f.sum(axis=0)
    j = lat.cf.T @ f
    return rho, j / rho


def equilibrium(lat, rho, u):
    """Eq. feq: w_i rho [1 + c.u/cs2 + (c.u)^2/(2 cs4) - u.u/(2 cs2)]."""
    cu = lat.cf @ u
    usq = (u * u).sum(axis=0)
    return lat.w[:, None] * rho[None, :] * (
        1.0 + cu / CS2 + cu * cu / (2.0 * CS2 * CS2) - usq[None, :] / (2.0 * CS2)
    )


def forcing(lat, rho, accel):
    """Body-force term F_i = w_i rho (c_i . a) / c_s^2.

    The paper prints F_i = -(rho g / c_s^2) w_i c_i . e_z for gravity along -z
    (Sec. 2.1); this is the same term for a general acceleration vector a.
    """
    return lat.w[:, None] * rho[None, :] * (lat.cf @ accel) / CS2


def collide(lat, f, omega, accel):
    """Eq. 1 right-hand side with the BGK operator: f + omega (f^eq - f) + F."""
    rho, u = moments(lat, f)
    return f + omega[None, :] * (equilibrium(lat, rho, u) - f) + forcing(lat, rho, accel)


def strain_rate(lat, f, omega):
    """Strain rate S_ab = -(omega / (2 rho c_s^2)) sum_i c_ia c_ib f^neq_i.

    Standard Chapman-Enskog relation of the BGK scheme (f^neq = f - f^eq);
    used for the stress jump of Eq. Sdecomp.  Returns shape (D, D, N).
    """
    rho, u = moments(lat, f)
    fneq = f - equilibrium(lat, rho, u)
    pi = np.einsum("qa,qb,qn->abn", lat.cf, lat.cf, fneq)
    return -(omega / (2.0 * rho * CS2))[None, None, :] * pi
