"""Block refinement and Dupuis-Chopard level coupling (Sec. 2.1 last paragraph, Sec. 2.6, Sec. 3.2.2).

Levels l = 0..L-1 halve the cell size (2:1).  Every level is a dense box of
base * 2^l cells; a block of level l is INACTIVE (its parent is not refined),
LEAF (it carries the solution) or REFINED (covered by 2^D blocks of level l+1).

Readings (the paper names the method and gives no formulas):

* Sensor (Sec. 2.6, Sec. 3.2.2): a level-l block is tagged for refinement when
  a finest-level cell under it satisfies the level's criterion: the symmetric
  band |phi| <= d_l, or the paper's signed sensor read as phi >= -d_l (its text
  says d_ref = 0 refines the gas, phi > 0, while its formula as printed refines
  phi <= d_ref; the text and Fig. 10a are followed).  Untagged blocks coarsen.
* Grading: a refined block's 3^D neighbours must be active, enforced from the
  finest level down; refinement of a block implies refinement of its parent.
* Time stepping: acoustic scaling dt ~ dx, so nu_l = nu_fine / 2^(L-1-l)
  (tau_f - 1/2 = 2 (tau_c - 1/2)) and lattice accelerations a_l = a_fine * 2^(L-1-l).
* Coarse-to-fine (ghost ring of the fine level, the fine cells just outside
  its active blocks): linear interpolation of the coarse pre-collision
  populations at the fine cell centre (offset +-1/4 coarse cell per axis,
  central gradients where both coarse neighbours are leaves, one-sided where
  only one is, none otherwise), linear in time (t and t+1/2), then
  f = f^eq + (tau_f / (2 tau_c)) f^neq and a fine-level collision.
* Fine-to-coarse (covered coarse cells that a coarse leaf streams from):
  mean of the 2^D children's pre-collision populations with
  f^neq scaled by 2 tau_c / tau_f.
* Regrid: new fine blocks are filled by the coarse-to-fine interpolation
  (without collision); coarsened blocks' parents by the fine-to-coarse mean.

Pins: tests/test_oracle_amr.py (grading and masks by brute force, equilibrium
and linear fields reproduced exactly by the transfer operators, single-phase
two-level Poiseuille against its closed form).
"""
import numpy as np

from .lbm import equilibrium, moments

INACTIVE, LEAF, REFINED = 0, 1, 2


def child_cells(gc, gf, cells):
    """Flat indices (2^D, M) of the fine children of coarse ``cells``."""
    D = gc.D
    out = []
    for s in np.ndindex(*([2] * D)):
        co = 2 * gc.coord[:, cells] + np.array(s)[:, None]
        out.append(gf.flat(co))
    return np.stack(out)


def parent_cells(gc, gf, cells):
    return gc.flat(gf.coord[:, cells] // 2)


def block_parent(gc, gf, bf):
    return gc.flat_block(gf.block_coord(np.asarray(bf)) // 2)


def sensor(geoms, phi, dists, mode):
    """Per level l < L-1, a boolean per block: tagged for refinement."""
    L = len(geoms)
    gF = geoms[-1]
    want = []
    for l in range(L - 1):
        g = geoms[l]
        r = 2 ** (L - 1 - l)
        blk = g.flat_block((gF.coord // r) // np.array(g.block)[:, None])
        if mode == "signed":
            crit = phi >= -dists[l]
        else:
            crit = np.abs(phi) <= dists[l]
        w = np.zeros(g.NB, dtype=bool)
        np.logical_or.at(w, blk, crit)
        want.append(w)
    return want


def grade(geoms, want):
    """Enforce nesting and 2:1 balance; returns the status arrays per level."""
    L = len(geoms)
    want = [w.copy() for w in want]
    for l in range(L - 2, 0, -1):
        g = geoms[l]
        gc = geoms[l - 1]
        for b in np.flatnonzero(want[l]):
            for nb in g.block_neighbors(int(b)):
                want[l - 1][block_parent(gc, g, nb)] = True
            want[l - 1][block_parent(gc, g, int(b))] = True
    status = []
    for l in range(L):
        g = geoms[l]
        if l == 0:
            act = np.ones(g.NB, dtype=bool)
        else:
            par = block_parent(geoms[l - 1], g, np.arange(g.NB))
            act = status[l - 1][par] == REFINED
        st = np.where(act, LEAF, INACTIVE).astype(np.int8)
        if l < L - 1:
            st = np.where(act & want[l], REFINED, st).astype(np.int8)
        status.append(st)
    return status


def level_masks(geom, lat, status):
    """Cell masks: leaf, covered, rlayer (covered cells a leaf streams from), ghost."""
    st = status[geom.block_of]
    leaf = st == LEAF
    covered = st == REFINED
    active = st != INACTIVE
    allc = np.arange(geom.N)
    near_leaf = np.zeros(geom.N, dtype=bool)
    for i in range(lat.Q):
        if i == lat.rest:
            continue
        nb, _ = geom.shift(allc, lat.c[i])
        ok = nb >= 0
        near_leaf[ok] |= leaf[nb[ok]]
    rlayer = covered & near_leaf
    ghost = (~active) & near_leaf
    return leaf, covered, rlayer, ghost


def interpolate_coarse(lat, gc, gf, F, usable, fine_cells):
    """Linear interpolation of coarse populations F at fine cell centres."""
    par = parent_cells(gc, gf, fine_cells)
    out = F[:, par].copy()
    for a in range(gc.D):
        e = np.zeros(gc.D, dtype=np.int64)
        e[a] = 1
        s = gf.coord[a, fine_cells] % 2
        delta = (s - 0.5) / 2.0
        up, _ = gc.shift(par, e)
        dn, _ = gc.shift(par, -e)
        upok = up >= 0
        upok[upok] = usable[up[upok]]
        dnok = dn >= 0
        dnok[dnok] = usable[dn[dnok]]
        fu = F[:, np.where(upok, up, 0)]
        fd = F[:, np.where(dnok, dn, 0)]
        fp = F[:, par]
        grad = np.where(upok & dnok, 0.5 * (fu - fd),
                        np.where(upok, fu - fp, np.where(dnok, fp - fd, 0.0)))
        out += delta[None, :] * grad
    return out


def rescale_neq(lat, f, factor):
    """f -> f^eq(rho, u) + factor * (f - f^eq), factor per column."""
    rho, u = moments(lat, f)
    feq = equilibrium(lat, rho, u)
    return feq + factor[None, :] * (f - feq)
