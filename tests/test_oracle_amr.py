"""Pins for oracle/amr.py (Sec. 2.1 last paragraph, 2.6, 3.2.2): grading, masks,
transfer operators, and a two-level single-phase Poiseuille against its closed form."""
import itertools

import numpy as np
import pytest

from oracle import amr
from oracle.grid import LevelGeom
from oracle.lattice import D2Q9, D3Q19
from oracle.lbm import equilibrium, moments
from oracle.sim import Sim


def _geoms(base, L, block, periodic):
    return [LevelGeom(tuple(b * 2 ** l for b in base), periodic, block) for l in range(L)]


@pytest.mark.parametrize("L", [2, 3])
def test_grading_invariants_brute_force(L):
    rng = np.random.default_rng(8)
    for trial in range(20):
        geoms = _geoms((16, 12), L, (4, 4), (bool(trial % 2), False))
        want = [rng.random(g.NB) < 0.15 for g in geoms[:-1]]
        st = amr.grade(geoms, want)
        for l, g in enumerate(geoms):
            for b in range(g.NB):
                if l > 0:
                    par = amr.block_parent(geoms[l - 1], g, b)
                    assert (st[l][b] != amr.INACTIVE) == (st[l - 1][par] == amr.REFINED)
                if st[l][b] == amr.REFINED:
                    for nb in g.block_neighbors(b):
                        assert st[l][nb] != amr.INACTIVE
            if l < L - 1:
                # every tagged block whose parent chain is refined is refined
                act = st[l] != amr.INACTIVE
                assert np.all(st[l][want[l] & act] == amr.REFINED)


def test_masks_brute_force():
    geoms = _geoms((8, 8), 2, (4, 4), (False, False))
    st = amr.grade(geoms, [np.array([True, False, False, False])])
    for l, g in enumerate(geoms):
        leaf, cov, rl, gh = amr.level_masks(g, D2Q9, st[l])
        for x in range(g.N):
            nbs = [g.shift(np.array([x]), D2Q9.c[i])[0][0] for i in range(8)]
            s = st[l][g.block_of[x]]
            near_leaf = any(n >= 0 and st[l][g.block_of[n]] == amr.LEAF for n in nbs)
            assert leaf[x] == (s == amr.LEAF)
            assert rl[x] == (s == amr.REFINED and near_leaf)
            assert gh[x] == (s == amr.INACTIVE and near_leaf)


@pytest.mark.parametrize("lat", [D2Q9, D3Q19], ids=lambda l: l.name)
def test_transfer_operators_exact_on_equilibrium_and_linear_fields(lat):
    D = lat.D
    base = (4,) * D
    geoms = _geoms(base, 2, (2,) * D, (True,) * D)
    gc, gf = geoms
    rng = np.random.default_rng(9)
    rho = 1.0 + 0.01 * rng.standard_normal()
    u = 0.01 * rng.standard_normal((D, 1))
    feq = equilibrium(lat, np.full(gc.N, rho), np.repeat(u, gc.N, 1))
    usable = np.ones(gc.N, dtype=bool)
    cells = np.arange(gf.N)
    fi = amr.interpolate_coarse(lat, gc, gf, feq, usable, cells)
    assert np.allclose(amr.rescale_neq(lat, fi, np.full(gf.N, 0.7)), feq[:, :1], atol=1e-15)
    # linear-in-space populations are reproduced at fine centres (interior, central gradients)
    gc2, gf2 = _geoms((6,) * D, 2, (2,) * D, (False,) * D)
    xc = gc2.centers()
    coef = rng.standard_normal((lat.Q, D))
    F = coef @ xc + 1.0
    inner = np.flatnonzero(((gf2.coord >= 2) & (gf2.coord < 10)).all(0))
    fi2 = amr.interpolate_coarse(lat, gc2, gf2, F, np.ones(gc2.N, dtype=bool), inner)
    want = coef @ gf2.centers(0.5)[:, inner] + 1.0
    assert np.allclose(fi2, want, atol=1e-12)
    # restriction of a fine equilibrium is that equilibrium
    rl = np.arange(gc.N)
    ch = amr.child_cells(gc, gf, rl)
    feqf = equilibrium(lat, np.full(gf.N, rho), np.repeat(u, gf.N, 1))
    mean = feqf[:, ch].mean(axis=1)
    assert np.allclose(amr.rescale_neq(lat, mean, np.full(gc.N, 1.6)), feq, atol=1e-15)


def _two_level_poiseuille_error(Hc, steps, nu=0.5, G=2e-6):
    H = 2 * Hc  # finest cells
    yf = np.arange(H) + 0.5
    phi = np.repeat(-(0.5 + np.abs(yf - H / 2)), 8)  # all liquid, fine band round the centre line
    case = dict(lattice="D2Q9", base=(4, Hc), n_levels=2, block=(2, Hc // 4), periodic=(True, False),
                rho_phys=(1.0, 1.0), nu=(nu, nu), body_force=(G, 0.0), phi0=phi,
                refine_dist=[Hc / 2 - 2], sensor="signed", ls_active=False)
    sim = Sim(case)
    assert (sim.status[0] == amr.REFINED).any() and (sim.status[0] == amr.LEAF).any()
    sim.step(steps)
    umax = G / (2 * nu) * (H / 2) ** 2
    err = 0.0
    for l, g in enumerate(sim.geoms):
        leaf = sim.masks[l][0]
        rho, u = moments(D2Q9, sim.f[l][:, leaf])
        y = g.centers(2 ** (1 - l))[1, leaf]
        err = max(err, np.abs(u[0] - G / (2 * nu) * y * (H - y)).max() / umax)
    return err


@pytest.mark.slow
def test_two_level_single_phase_poiseuille_converges():
    """Closed form on a two-level grid; the level coupling converges with resolution
    (about 1.7% at 32 finest cells, 0.7% at 64: the ghost interpolation is one-sided
    next to the fine region).  A wrong f^neq rescaling or force scaling does not converge."""
    e1 = _two_level_poiseuille_error(16, 1500)
    e2 = _two_level_poiseuille_error(32, 4000)
    assert e1 < 0.025 and e2 < 0.01, (e1, e2)
    assert e1 / e2 > 2.0, (e1, e2)


def test_two_level_couette_linear_profile_exact():
    Hc = 16
    H = 2 * Hc
    yf = np.arange(H) + 0.5
    phi = np.repeat(-(0.5 + np.abs(yf - H / 2)), 8)
    U = 1e-3
    wall = np.zeros((4, 2))
    wall[3, 0] = U
    case = dict(lattice="D2Q9", base=(4, Hc), n_levels=2, block=(2, 4), periodic=(True, False),
                rho_phys=(1.0, 1.0), nu=(1 / 6, 1 / 6), wall_u=wall, phi0=phi,
                refine_dist=[6.0], sensor="signed", ls_active=False)
    sim = Sim(case)
    sim.step(3000)
    for l, g in enumerate(sim.geoms):
        leaf = sim.masks[l][0]
        rho, u = moments(D2Q9, sim.f[l][:, leaf])
        y = g.centers(2 ** (1 - l))[1, leaf]
        assert np.abs(u[0] - U * y / H).max() < 5e-4 * U
