"""Pins for oracle/cumulant.py (the gas-phase cumulant collision on D3Q27, Sec. 3.2).

* The moment-cumulant recursion against the textbook relations of a few
  central cumulants (order 4 and the order-6 one of a Gaussian, where every
  cumulant above order 2 vanishes: Isserlis' theorem), and a round trip.
* Mass and momentum conservation, the equilibrium (Maxwellian cumulants:
  c_s^2 on the diagonal, zero elsewhere) as a fixed point.
* A decaying shear wave in a periodic box: its amplitude decays at
  nu k^2 with nu = c_s^2 (1 / w1 - 1 / 2), the viscosity the shear rate sets.
* With D3Q27 and BGK in both phases the Sim steps as before; the cumulant
  operator is used only where the case asks for it.
"""
import numpy as np
import pytest

from oracle.cumulant import POS, cumulant_collide, cumulants_from_moments, moments_from_cumulants
from oracle.lattice import CS2, get as get_lattice
from oracle.lbm import equilibrium, moments


def _rand_moments(rng, N=7):
    """Moments of a random positive discrete distribution on {-1, 0, 1}^3, centred."""
    lat = get_lattice("D3Q27")
    f = rng.random((27, N)) + 0.2
    rho, u = moments(lat, f)
    d = lat.cf[None, :, :] - u.T[:, None, :]
    k = np.zeros((27, N))
    for m, r in POS.items():
        w = np.ones((N, 27))
        for a in range(3):
            w *= d[:, :, a] ** m[a]
        k[r] = (w * f.T).sum(1) / rho
    return k


def test_recursion_matches_textbook_relations():
    k = _rand_moments(np.random.default_rng(0))
    c = cumulants_from_moments(k)
    K = lambda *m: k[POS[m]]
    C = lambda *m: c[POS[m]]
    assert np.allclose(C(1, 0, 0), 0, atol=1e-14) and np.allclose(C(1, 1, 0), K(1, 1, 0))
    assert np.allclose(C(2, 1, 0), K(2, 1, 0))  # order 3 equals the central moment
    assert np.allclose(C(2, 2, 0), K(2, 2, 0) - K(2, 0, 0) * K(0, 2, 0) - 2 * K(1, 1, 0) ** 2)
    assert np.allclose(C(2, 1, 1), K(2, 1, 1) - K(2, 0, 0) * K(0, 1, 1) - 2 * K(1, 1, 0) * K(1, 0, 1))
    assert np.allclose(moments_from_cumulants(c), k)


def test_gaussian_cumulants_give_isserlis_moments():
    rng = np.random.default_rng(1)
    A = rng.standard_normal((3, 3))
    S = A @ A.T * 0.1 + np.eye(3) * 0.2
    c = np.zeros((27, 1))
    for (a, b) in ((0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2)):
        m = [0, 0, 0]
        m[a] += 1
        m[b] += 1
        c[POS[tuple(m)]] = S[a, b]
    k = moments_from_cumulants(c)[:, 0]
    sx, sy, sz, sxy, sxz, syz = S[0, 0], S[1, 1], S[2, 2], S[0, 1], S[0, 2], S[1, 2]
    assert np.isclose(k[POS[(2, 2, 0)]], sx * sy + 2 * sxy ** 2)
    assert np.isclose(k[POS[(2, 1, 1)]], sx * syz + 2 * sxy * sxz)
    assert np.isclose(k[POS[(2, 2, 2)]], sx * sy * sz + 2 * sx * syz ** 2 + 2 * sy * sxz ** 2 + 2 * sz * sxy ** 2
                      + 8 * sxy * sxz * syz)
    assert np.isclose(k[POS[(2, 1, 0)]], 0) and np.isclose(k[POS[(2, 2, 1)]], 0)


def test_collision_conserves_mass_momentum_and_keeps_equilibrium():
    lat = get_lattice("D3Q27")
    rng = np.random.default_rng(2)
    N = 11
    rho = 1 + 0.05 * rng.standard_normal(N)
    u = 0.05 * rng.standard_normal((3, N))
    f = equilibrium(lat, rho, u) + 1e-3 * rng.standard_normal((27, N)) * lat.w[:, None]
    fc = cumulant_collide(lat, f, 1.3)
    r0, u0 = moments(lat, f)
    r1, u1 = moments(lat, fc)
    assert np.allclose(r1, r0, rtol=1e-14) and np.allclose(r1 * u1, r0 * u0, atol=1e-15)
    # the Maxwellian's cumulant state (diagonal c_s^2, all others zero) is a fixed point
    c = np.zeros((27, N))
    for m in ((2, 0, 0), (0, 2, 0), (0, 0, 2)):
        c[POS[m]] = CS2
    k = moments_from_cumulants(c)
    from oracle.cumulant import _transform
    T = _transform(lat, u)
    feq = np.linalg.solve(T, (k * rho[None, :]).T[:, :, None])[:, :, 0].T
    assert np.allclose(cumulant_collide(lat, feq, 1.7), feq, rtol=1e-13, atol=1e-15)
    # an unrelaxed shear rate leaves second cumulants, not higher ones, as they were
    f2 = cumulant_collide(lat, f, 0.0)
    assert np.allclose(moments(lat, f2)[0], r0)


@pytest.mark.parametrize("w1", [1.0, 1.6])
def test_shear_wave_decays_at_the_set_viscosity(w1):
    from oracle.sim import Sim
    n = 24
    z = np.arange(n) + 0.5
    U0 = 1e-4
    case = dict(lattice="D3Q27", base=(4, 4, n), block=(4, 4, n), periodic=(True, True, True), rho_phys=(1.0, 1.0),
                nu=(CS2 * (1 / w1 - 0.5),) * 2, phi0=np.full(4 * 4 * n, 1.0), ls_active=False, n_ext=0,
                reinit_every=0, collision=("bgk", "cumulant"))
    sim = Sim(case)
    lat = sim.lat
    k = 2 * np.pi / n
    ux = U0 * np.sin(k * np.repeat(z, 16))
    sim.f[0] = equilibrium(lat, np.ones(16 * n), np.stack([ux, 0 * ux, 0 * ux]))
    T = 200
    sim.step(T)
    _, u = moments(lat, sim.f[0])
    amp = 2 * (u[0] * np.sin(k * np.repeat(z, 16))).mean()
    nu = CS2 * (1 / w1 - 0.5)
    assert abs(np.log(amp / U0) / T + nu * k ** 2) < 0.02 * nu * k ** 2
