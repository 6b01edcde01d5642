"""Pins for oracle/coupling.py (Sec. 2.3, 2.4): link fraction, extrapolation weights, e_min."""
import numpy as np
import pytest

from oracle import coupling
from oracle.grid import LevelGeom
from oracle.lattice import D2Q9, D3Q19


def test_link_fraction_exact_for_linear_phi():
    rng = np.random.default_rng(5)
    for _ in range(100):
        s = rng.uniform(0.01, 0.99)  # interface at fraction s of the link
        slope = rng.uniform(0.2, 3.0) * rng.choice([-1, 1])
        phi_x = -slope * s
        phi_y = slope * (1 - s)
        assert abs(coupling.link_fraction(phi_x, phi_y) - s) < 1e-14


@pytest.mark.parametrize("quad", [True, False])
def test_extrapolation_weights(quad):
    rng = np.random.default_rng(6)
    for q in rng.uniform(0, 1, 50):
        w = coupling.extrapolation_weights(q, quad)
        assert abs(sum(w) - 1) < 1e-14
        # exact for polynomials of degree 2 (quadratic) / 1 (linear) through nodes -q, 1, 2
        for p in range(3 if quad else 2):
            vals = np.array([(-q) ** p, 1.0, 2.0 ** p])
            assert abs(w[0] * vals[0] + w[1] * vals[1] + w[2] * vals[2] - (0.0 ** p)) < 1e-13


def test_printed_third_weight_is_a_typo():
    # the printed set 2/((q+1)(q+2)), 2q/(q+1), 2q/(q+2) sums to 2 at q = 1
    q = 1.0
    assert abs(2 / ((q + 1) * (q + 2)) + 2 * q / (q + 1) + 2 * q / (q + 2) - 2.0) < 1e-15


@pytest.mark.parametrize("lat", [D2Q9, D3Q19], ids=lambda l: l.name)
def test_emin_brute_force(lat):
    D = lat.D
    g = LevelGeom((5,) * D, (False,) * D, (5,) * D)
    xr = int(g.flat(np.full((D, 1), 2))[0])
    rng = np.random.default_rng(7)
    ok = np.ones(g.N, dtype=bool)
    for _ in range(40):
        m = rng.standard_normal(D)
        m /= np.linalg.norm(m)
        e = coupling.choose_emin(lat, g, xr, m, ok)
        cos = [(lat.cf[i] @ m) / lat.norm[i] if i != lat.rest else -9 for i in range(lat.Q)]
        assert e == int(np.argmax(cos))
    # unusable neighbours are skipped
    m = np.zeros(D)
    m[0] = 1.0
    best = coupling.choose_emin(lat, g, xr, m, ok)
    nb, _ = g.shift(np.array([xr]), lat.c[best])
    ok2 = ok.copy()
    ok2[nb[0]] = False
    assert coupling.choose_emin(lat, g, xr, m, ok2) != best


def test_stress_jump_static_and_shear():
    # static: [p] = -sigma kappa_A, Sbar = 0 -> [S] = 0
    nA = np.array([[0.0], [1.0]])
    c = np.array([[1.0], [1.0]])
    z = np.zeros((2, 2, 1))
    v = coupling.stress_jump_cc(c, nA, np.array([0.1]), z, np.array([-0.02 * 0.1]), 0.0,
                                np.array([1.0]), 0.02)
    assert abs(v[0]) < 1e-18
    # pure shear along a flat interface: eta_A S_A = eta_B S_B with Sbar the mean
    etaA, etaB, sA = 0.5, 0.1, 1e-3
    sB = etaA * sA / etaB
    Sbar = np.zeros((2, 2, 1))
    Sbar[0, 1] = Sbar[1, 0] = 0.5 * (sA + sB)
    jump = sB - sA
    got = coupling.stress_jump_cc(c, nA, np.zeros(1), Sbar, np.zeros(1), etaB - etaA,
                                  np.array([0.5 * (etaA + etaB)]), 0.0)
    # c c : [S] = 2 c_x c_y [S]_xy = 2 * jump
    assert abs(got[0] - 2 * jump) < 1e-15
