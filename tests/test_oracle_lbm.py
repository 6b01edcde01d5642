"""Pins for oracle/lbm.py (Sec. 2.1): equilibrium moments, conservation, closed-form channels."""
import numpy as np
import pytest

from oracle.lattice import CS2, D2Q9, D3Q19
from oracle.lbm import collide, equilibrium, moments, omega_from_nu, strain_rate
from oracle.sim import Sim


@pytest.mark.parametrize("lat", [D2Q9, D3Q19], ids=lambda l: l.name)
def test_equilibrium_moments(lat):
    rng = np.random.default_rng(1)
    N = 50
    rho = 1 + 0.1 * rng.standard_normal(N)
    u = 0.05 * rng.standard_normal((lat.D, N))
    feq = equilibrium(lat, rho, u)
    assert np.allclose(feq.sum(0), rho, rtol=1e-14)
    assert np.allclose(lat.cf.T @ feq, rho * u, atol=1e-15)
    pi = np.einsum("qa,qb,qn->abn", lat.cf, lat.cf, feq)
    want = CS2 * rho[None, None] * np.eye(lat.D)[:, :, None] + rho * np.einsum("an,bn->abn", u, u)
    assert np.allclose(pi, want, atol=1e-14)


@pytest.mark.parametrize("lat", [D2Q9, D3Q19], ids=lambda l: l.name)
def test_collision_conservation(lat):
    rng = np.random.default_rng(2)
    N = 40
    f = lat.w[:, None] * (1 + 0.05 * rng.standard_normal((lat.Q, N)))
    om = np.full(N, 1.3)
    a = 1e-3 * rng.standard_normal((lat.D, N))
    fc = collide(lat, f, om, a)
    rho, u = moments(lat, f)
    assert np.allclose(fc.sum(0), f.sum(0), rtol=1e-14)
    assert np.allclose(lat.cf.T @ fc, rho * u + rho * a, atol=1e-15)


def test_omega_from_nu():
    # tau = 3 nu + 1/2 in lattice units
    assert abs(1 / omega_from_nu(0.1) - 0.8) < 1e-15


def test_strain_rate_of_shear_equilibrium_plus_neq():
    # f^neq = -(w rho / (cs2 omega)) Q:S has strain rate S back (Chapman-Enskog, BGK)
    lat = D2Q9
    om = 1.25
    S = np.array([[0.0, 1e-3], [1e-3, 0.0]])
    rho = np.array([1.0])
    u = np.zeros((2, 1))
    Qi = np.einsum("qa,qb->qab", lat.cf, lat.cf) - CS2 * np.eye(2)[None]
    fneq = -(lat.w * rho[0] / (CS2 * om))[:, None, None] * Qi
    f = equilibrium(lat, rho, u) + np.einsum("qab,ab->q", fneq, S)[:, None]
    got = strain_rate(lat, f, np.array([om]))[:, :, 0]
    assert np.allclose(got, S, atol=1e-16)


def _channel(lat_name, H, nu, G=None, wall_top=None):
    D = 2 if lat_name == "D2Q9" else 3
    base = (2, H) if D == 2 else (2, H, 2)
    periodic = (True, False) if D == 2 else (True, False, True)
    block = (2, H) if D == 2 else (2, H, 2)
    phi0 = -np.ones(int(np.prod(base)))  # all liquid
    wall = np.zeros((2 * D, D))
    if wall_top is not None:
        wall[3, 0] = wall_top
    bf = np.zeros(D)
    if G is not None:
        bf[0] = G
    case = dict(lattice=lat_name, base=base, block=block, periodic=periodic, rho_phys=(1.0, 1.0),
                nu=(nu, nu), body_force=bf, wall_u=wall, phi0=phi0, n_ext=0, reinit_every=0)
    return Sim(case)


def _y_profile(sim, H):
    rho, u = sim.macros()
    g = sim.geoms[-1]
    y = g.coord[1]
    return np.array([u[0, y == j].mean() for j in range(H)])


@pytest.mark.parametrize("lat_name", ["D2Q9", "D3Q19"])
def test_single_phase_poiseuille(lat_name):
    H, nu, G = 16, 1 / 6, 1e-5
    sim = _channel(lat_name, H, nu, G=G)
    sim.step(2500)
    prof = _y_profile(sim, H)
    y = np.arange(H) + 0.5
    exact = G / (2 * nu) * y * (H - y)
    assert np.max(np.abs(prof - exact)) / exact.max() < 5e-3
    # a wrong omega(nu), force sign or wall rule moves this by O(1)
    assert prof.min() > 0


def test_single_phase_couette_moving_wall_sign():
    H, nu, U = 16, 1 / 6, 1e-3
    sim = _channel("D2Q9", H, nu, wall_top=U)
    sim.step(2500)
    prof = _y_profile(sim, H)
    y = np.arange(H) + 0.5
    assert np.max(np.abs(prof - U * y / H)) < 1e-3 * U * 5
    assert prof[-1] > prof[0]


def test_periodic_mass_conservation_exact():
    lat_name = "D2Q9"
    rng = np.random.default_rng(3)
    base = (12, 10)
    case = dict(lattice=lat_name, base=base, block=(4, 5), periodic=(True, True), rho_phys=(1.0, 1.0),
                nu=(0.05, 0.05), phi0=-np.ones(120), n_ext=0, reinit_every=0)
    sim = Sim(case)
    sim.f[0] = sim.f[0] * (1 + 0.01 * rng.standard_normal(sim.f[0].shape))
    m0 = sim.f[0].sum()
    j0 = (D2Q9.cf.T @ sim.f[0]).sum(1)
    sim.step(200)
    assert abs(sim.f[0].sum() - m0) < 1e-12 * m0
    assert np.allclose((D2Q9.cf.T @ sim.f[0]).sum(1), j0, atol=1e-13)
