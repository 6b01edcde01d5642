"""Brute-force pin of the oracle's cut-link enumeration (Sec. 2.3, Sim.cut_links).

A link (x, k) is cut when x carries populations on the finest level and the
cell its incoming population k comes from, x - c_k, is a fluid cell of the
other phase (radiation theorem: the interface crosses the segment between
them).  Phases come from the sign of phi: liquid iff phi < 0, so phi == 0
exactly is gas (Sec. 2.2, Sec. 3.1's "y >= 0 fluid 2").

Every sign pattern (negative, zero, positive) of a 3x3 patch is enumerated for
D2Q9; D3Q19 takes 20 000 random patterns of a 3x3x3 patch.  The patches are
tiled into one box and each patch's centre cell is checked against a plain
loop over the lattice directions written with coordinate tuples; a periodic
and a walled small box are checked at every cell.
"""
import itertools
import types

import numpy as np
import pytest

from oracle import levelset
from oracle.grid import LevelGeom
from oracle.lattice import D2Q9, D3Q19
from oracle.sim import Sim


def _cut_links(lat, geom, phi, fluid):
    fake = types.SimpleNamespace(lat=lat, geoms=[geom])
    return Sim.cut_links(fake, levelset.classify(phi), fluid)


def _brute_cell(lat, dims, periodic, coord, phi_at, fluid_at):
    """Set of incoming directions k cut at the cell ``coord`` (tuple), by definition."""
    D = len(dims)
    out = set()
    if not fluid_at(coord):
        return out
    gas_x = phi_at(coord) >= 0.0
    for k in range(lat.Q):
        ck = tuple(int(v) for v in lat.c[k])
        if all(v == 0 for v in ck):
            continue
        src = []
        inside = True
        for a in range(D):
            s = coord[a] - ck[a]
            if periodic[a]:
                s %= dims[a]
            elif s < 0 or s >= dims[a]:
                inside = False
            src.append(s)
        if not inside:
            continue
        src = tuple(src)
        if fluid_at(src) and (phi_at(src) >= 0.0) != gas_x:
            out.add(k)
    return out


def _tile(patterns, D, per_row):
    """Lay 3^D patches side by side; returns the dims, phi (flat) and each patch centre."""
    n = len(patterns)
    rows = -(-n // per_row)
    if D == 2:
        dims = (3 * per_row, 3 * rows)
    else:
        r2 = int(np.ceil(np.sqrt(rows)))
        dims = (3 * per_row, 3 * r2, 3 * (-(-rows // r2)))
    phi = np.full(dims[::-1], 7.0)
    centres = []
    for p, pat in enumerate(patterns):
        px, rest = p % per_row, p // per_row
        if D == 2:
            org = (3 * px, 3 * rest)
        else:
            r2 = dims[1] // 3
            org = (3 * px, 3 * (rest % r2), 3 * (rest // r2))
        block = np.asarray(pat, float).reshape((3,) * D)  # (z,) y, x order
        sl = tuple(slice(o, o + 3) for o in org[::-1])
        phi[sl] = block
        centres.append(tuple(o + 1 for o in org))
    return dims, phi.reshape(-1), centres


def _check_centres(lat, dims, phi, fluid, centres):
    D = lat.D
    g = LevelGeom(dims, (False,) * D, dims)
    lx, lk = _cut_links(lat, g, phi, fluid)
    got = {}
    for x, k in zip(lx.tolist(), lk.tolist()):
        got.setdefault(x, set()).add(k)
    phi_d = phi.reshape(dims[::-1])
    fl_d = fluid.reshape(dims[::-1])

    def phi_at(c):
        return float(phi_d[c[::-1]])

    def fluid_at(c):
        return bool(fl_d[c[::-1]])

    strides = np.cumprod((1,) + dims[:-1])
    for c in centres:
        flat = int(sum(ci * s for ci, s in zip(c, strides)))
        want = _brute_cell(lat, dims, (False,) * D, c, phi_at, fluid_at)
        assert got.get(flat, set()) == want, (c, got.get(flat), want)


def test_d2q9_every_sign_pattern():
    pats = list(itertools.product((-1.0, 0.0, 1.0), repeat=9))
    dims, phi, centres = _tile(pats, 2, 243)
    _check_centres(D2Q9, dims, phi, np.ones(phi.size, bool), centres)


def test_d2q9_sign_patterns_with_non_fluid_cells():
    rng = np.random.default_rng(21)
    pats = list(itertools.product((-1.0, 0.0, 1.0), repeat=9))
    dims, phi, centres = _tile(pats, 2, 243)
    _check_centres(D2Q9, dims, phi, rng.random(phi.size) > 0.15, centres)


def test_d3q19_random_sign_patterns():
    rng = np.random.default_rng(22)
    pats = rng.choice([-1.0, 0.0, 1.0], size=(20000, 27), p=[0.45, 0.1, 0.45])
    dims, phi, centres = _tile(list(pats), 3, 50)
    fluid = rng.random(phi.size) > 0.1
    _check_centres(D3Q19, dims, phi, fluid, centres)


@pytest.mark.parametrize("lat,dims", [(D2Q9, (5, 4)), (D3Q19, (4, 3, 5))], ids=["D2Q9", "D3Q19"])
@pytest.mark.parametrize("periodic", [True, False])
def test_every_cell_of_a_small_box(lat, dims, periodic):
    D = lat.D
    rng = np.random.default_rng(23)
    per = (periodic,) * D
    g = LevelGeom(dims, per, dims)
    for _ in range(20):
        phi = rng.choice([-2.0, -0.5, 0.0, 0.5, 2.0], size=g.N)
        fluid = rng.random(g.N) > 0.1
        lx, lk = _cut_links(lat, g, phi, fluid)
        got = {}
        for x, k in zip(lx.tolist(), lk.tolist()):
            got.setdefault(x, set()).add(k)
        phi_d = phi.reshape(dims[::-1])
        fl_d = fluid.reshape(dims[::-1])
        for flat in range(g.N):
            c = tuple(int(v) for v in g.coord[:, flat])
            want = _brute_cell(lat, dims, per, c, lambda cc: float(phi_d[cc[::-1]]),
                               lambda cc: bool(fl_d[cc[::-1]]))
            assert got.get(flat, set()) == want, (c, got.get(flat), want)


@pytest.mark.parametrize("plant", [("-lat.c[k]", "lat.c[k]"), ("phase[src[ok]] != phase[cells[ok]]",
                                                                "phase[src[ok]] == phase[cells[ok]]")],
                         ids=["source_on_the_wrong_side", "same_phase_links"])
def test_brute_force_detects_a_planted_mistake(monkeypatch, plant):
    from tests.test_oracle_refill import _mutant
    monkeypatch.setattr(Sim, "cut_links", _mutant(Sim.cut_links, *plant))
    rng = np.random.default_rng(24)
    pats = rng.choice([-1.0, 0.0, 1.0], size=(200, 9))
    dims, phi, centres = _tile(list(pats), 2, 20)
    with pytest.raises(AssertionError):
        _check_centres(D2Q9, dims, phi, np.ones(phi.size, bool), centres)
