"""Pins for oracle/lattice.py: exact isotropy identities of the velocity sets (Sec. 2.1)."""
import itertools

import numpy as np
import pytest

from oracle.lattice import CS2, D2Q9, D3Q19, D3Q27


@pytest.mark.parametrize("lat", [D2Q9, D3Q19, D3Q27], ids=lambda l: l.name)
def test_isotropy(lat):
    w, c = lat.w, lat.cf
    D = lat.D
    assert abs(w.sum() - 1.0) < 1e-15
    assert np.allclose(w @ c, 0.0, atol=1e-16)
    m2 = np.einsum("q,qa,qb->ab", w, c, c)
    assert np.allclose(m2, CS2 * np.eye(D), atol=1e-15)
    m3 = np.einsum("q,qa,qb,qc->abc", w, c, c, c)
    assert np.allclose(m3, 0.0, atol=1e-16)
    m4 = np.einsum("q,qa,qb,qc,qd->abcd", w, c, c, c, c)
    I = np.eye(D)
    iso = (np.einsum("ab,cd->abcd", I, I) + np.einsum("ac,bd->abcd", I, I)
           + np.einsum("ad,bc->abcd", I, I)) * CS2 ** 2
    assert np.allclose(m4, iso, atol=1e-15)


@pytest.mark.parametrize("lat", [D2Q9, D3Q19, D3Q27], ids=lambda l: l.name)
def test_opposites_and_counts(lat):
    assert lat.Q == {"D2Q9": 9, "D3Q19": 19, "D3Q27": 27}[lat.name]
    for i in range(lat.Q):
        assert (lat.c[lat.opp[i]] == -lat.c[i]).all()
        assert lat.w[lat.opp[i]] == lat.w[i]
    assert len({tuple(v) for v in lat.c}) == lat.Q


def test_fig1_ordering():
    # Fig. 1a: c0..c3 axis (-x, +x, -y, +y), c4..c7 diagonals, c8 rest
    assert D2Q9.c[0].tolist() == [-1, 0] and D2Q9.c[3].tolist() == [0, 1]
    assert D2Q9.c[6].tolist() == [1, 1] and D2Q9.rest == 8
    # D3Q19 keeps the D3Q27 ordering of Fig. 1b for its 18 moving velocities
    assert (D3Q19.c[:18] == D3Q27.c[:18]).all() and D3Q19.rest == 18
