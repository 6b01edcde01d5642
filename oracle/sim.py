"""One coarse time step of the coupled level-set LB method (Sec. 2), multi-level.

State: per level the PRE-collision populations f_l(t) (Eq. 1 left-hand side
after streaming), each cell holding the populations of its own phase; the
finest-level level set phi and the persistent extension velocity u~.

Order of one finest-level step t -> t+1 (the paper prints no order; this one
is the reading used by both implementations):
  1. moments, strain rate at t; n, kappa at t on interface cells;
  2. BGK collision with forcing on every leaf cell (phase parameters);
  3. streaming: same-phase links pull, walls take half-way bounce-back with
     the moving-wall term, cut links take Eq. bb with Eq. bb_cc;
  4. level set: u~ on interface cells from u_I(t), extension, TVD-RK3
     advection, constrained reinitialisation every ``reinit_every`` steps;
  5. phases at t+1; cells whose phase flipped are refilled (Sec. 2.4).
Coarser levels run collision + streaming only (the interface lives on the
finest level, Sec. 2.5) inside the Dupuis-Chopard recursion described in
``amr``.  A coarse step advances the finest level 2^(L-1) times.

Parity is pinned by the closed-form flows in tests/test_oracle_flows.py and
tests/test_oracle_amr.py, the cut-link enumeration by brute force
(tests/test_oracle_cut_links.py) and the refill by exact reproduction of
fields built to satisfy the interface conditions
(tests/test_oracle_refill.py); the step order itself is a reading (parity
unpinned beyond those checks).
"""
import numpy as np

from . import amr, coupling, levelset
from .grid import LevelGeom
from .lattice import CS2, get as get_lattice
from .lbm import collide, equilibrium, forcing, moments, omega_from_nu, strain_rate

DEFAULTS = dict(
    n_levels=1, sigma=0.0, body_force=None, gravity=None, x_ref=None, wall_u=None, p_gas0=0.0,
    n_ext=8, dtau_ext=0.5, reinit_every=1, n_reinit=1, dtau_reinit=0.3,
    refine_dist=None, sensor="band", regrid_every=0, ls_active=True, slip=None,
    collision=("bgk", "bgk"),
)


class Sim:
    """FP64 oracle simulation of one case (lattice units of the finest level)."""

    def __init__(self, case):
        c = dict(DEFAULTS)
        c.update(case)
        self.case = c
        self.lat = get_lattice(c["lattice"])
        lat = self.lat
        D = lat.D
        self.D = D
        self.L = int(c["n_levels"])
        base = tuple(int(b) for b in c["base"])
        self.periodic = tuple(bool(p) for p in c["periodic"])
        self.slip = tuple(bool(s) for s in (c["slip"] or (False,) * D))
        # collision operator per phase (liquid, gas): BGK, or the cumulant model on D3Q27
        self.collision = tuple(str(k) for k in c["collision"])
        assert all(k in ("bgk", "cumulant") for k in self.collision)
        assert "cumulant" not in self.collision or c["lattice"] == "D3Q27", "cumulant collision needs D3Q27"
        self.geoms = [LevelGeom(tuple(b * 2 ** l for b in base), self.periodic, c["block"], self.slip)
                      for l in range(self.L)]
        gF = self.geoms[-1]
        self.rho_phys = np.asarray(c["rho_phys"], dtype=np.float64)
        self.nu = np.asarray(c["nu"], dtype=np.float64)
        zero = np.zeros(D)
        self.body_force = np.asarray(c["body_force"] if c["body_force"] is not None else zero, float)
        self.gravity = np.asarray(c["gravity"] if c["gravity"] is not None else zero, float)
        self.sigma = float(c["sigma"])
        wu = c["wall_u"]
        self.wall_u = np.zeros((2 * D, D)) if wu is None else np.asarray(wu, float).reshape(2 * D, D)
        self.prm = dict(rho_phys=self.rho_phys, nu=self.nu, sigma=self.sigma)
        phi0 = np.asarray(c["phi0"], dtype=np.float64).reshape(-1)
        assert phi0.size == gF.N
        self.phi = phi0.copy()
        self.ut = np.zeros((D, gF.N))
        self.fine_steps = 0
        self.steps = 0
        self.stats = dict(refill_fail=0, coarse_cut=0, flipped=0)
        if self.L > 1:
            self.status = amr.grade(self.geoms, amr.sensor(self.geoms, self.phi, self._dists(), c["sensor"]))
        else:
            self.status = [np.full(gF.NB, amr.LEAF, dtype=np.int8)]
        self._build_masks()
        x_ref = np.asarray(c["x_ref"] if c["x_ref"] is not None else zero, float)
        self.f = []
        for l, g in enumerate(self.geoms):
            r = 2.0 ** (self.L - 1 - l)
            xc = g.centers(r)
            drho = -(self.gravity[:, None] * (xc - x_ref[:, None])).sum(0) / CS2
            drho = drho + np.where(self.phase[l] == 1, float(c["p_gas0"]) / (self.rho_phys[1] * CS2), 0.0)
            self.f.append(equilibrium(lat, 1.0 + drho, np.zeros((D, g.N))))
        self.ghost = [None] * self.L

    # ------------------------------------------------------------------ setup
    def _dists(self):
        d = self.case["refine_dist"]
        if d is None:
            d = [8.0] * (self.L - 1)
        return [float(x) for x in d]

    def _build_masks(self):
        self.masks = [amr.level_masks(g, self.lat, st) for g, st in zip(self.geoms, self.status)]
        gF = self.geoms[-1]
        self.phase = []
        for l, g in enumerate(self.geoms):
            r = 2 ** (self.L - 1 - l)
            corner = gF.flat(g.coord * r)
            self.phase.append(levelset.classify(self.phi[corner]))

    def level_params(self, l, phase):
        """omega and acceleration per cell of level l from the cell phases."""
        r = 2.0 ** (self.L - 1 - l)
        nu = self.nu[phase] / r
        om = omega_from_nu(nu)
        acc = (self.gravity[:, None] + self.body_force[:, None] / self.rho_phys[phase][None, :]) * r
        return om, acc

    def collide(self, f, om, acc, phase):
        """Post-collision populations with each cell's phase operator and forcing (Eq. 1)."""
        out = collide(self.lat, f, om, acc)
        for p in (0, 1):
            m = phase == p
            if self.collision[p] == "cumulant" and m.any():
                from .cumulant import cumulant_collide
                out[:, m] = cumulant_collide(self.lat, f[:, m], om[m]) + forcing(self.lat, f[:, m].sum(0), acc[:, m])
        return out

    def tau(self, l, phase):
        return 1.0 / self.level_params(l, phase)[0]

    # ------------------------------------------------------------ interface
    def cut_links(self, phase, fluid):
        """All (x, k) with x fluid on the finest level and x - c_k of the other phase.

        Pinned by brute force over every sign pattern of a 3x3 patch (D2Q9) and
        random 3x3x3 patterns (D3Q19), tests/test_oracle_cut_links.py."""
        lat = self.lat
        gF = self.geoms[-1]
        xs, ks = [], []
        cells = np.flatnonzero(fluid)
        for k in range(lat.Q):
            if k == lat.rest:
                continue
            src, _ = gF.shift(cells, -lat.c[k])
            ok = src >= 0
            ok[ok] = fluid[src[ok]] & (phase[src[ok]] != phase[cells[ok]])
            xs.append(cells[ok])
            ks.append(np.full(ok.sum(), k))
        return np.concatenate(xs), np.concatenate(ks)

    def band_mask(self, iface_mask):
        """Narrow band: blocks with an interface cell plus their 3^D neighbours, on active blocks."""
        gF = self.geoms[-1]
        hot = np.zeros(gF.NB, dtype=bool)
        hot[np.unique(gF.block_of[iface_mask])] = True
        band = np.zeros(gF.NB, dtype=bool)
        for b in np.flatnonzero(hot):
            band[gF.block_neighbors(int(b))] = True
        band &= self.status[-1] != amr.INACTIVE
        return band[gF.block_of]

    # ------------------------------------------------------------ stepping
    def step(self, n=1):
        for _ in range(n):
            self._advance(0)
            self.steps += 1
            re = int(self.case["regrid_every"])
            if self.L > 1 and re > 0 and self.steps % re == 0:
                self.regrid()

    def _advance(self, l):
        lat = self.lat
        g = self.geoms[l]
        leaf, covered, rlayer, ghost = self.masks[l]
        finest = l == self.L - 1
        if l < self.L - 1:
            self._restrict(l)
        f_old = self.f[l].copy()
        ph = self.phase[l]
        om, acc = self.level_params(l, ph)
        coll = np.flatnonzero(leaf | rlayer)
        fc = np.zeros_like(self.f[l])
        fc[:, coll] = self.collide(self.f[l][:, coll], om[coll], acc[:, coll], ph[coll])
        if finest:
            fluid = leaf
            rho, u = moments(lat, self.f[l])
            S = strain_rate(lat, self.f[l], om)
            lx, lk = self.cut_links(ph, fluid)
            iface = np.zeros(g.N, dtype=bool)
            iface[lx] = True
            icells = np.flatnonzero(iface)
            nvec = np.zeros((self.D, g.N))
            kap = np.zeros(g.N)
            nv, kv, _, _ = levelset.fit_geometry(g, self.phi, icells)
            nvec[:, icells] = nv
            kap[icells] = kv
        f_new = self.f[l].copy()
        cells = np.flatnonzero(leaf)
        gh = self.ghost[l]
        for k in range(lat.Q):
            i = lat.opp[k]
            src, face, flip = g.pull(cells, lat.c[k])
            wall = src < 0
            val = np.empty(len(cells))
            if wall.any():
                ci = lat.cf[i]
                du = self.wall_u[face[wall]] @ ci
                val[wall] = fc[i, cells[wall]] - (2.0 * lat.w[i] / CS2) * du
            inn = ~wall
            s = src[inn]
            ks = lat.mirror[k, flip[inn]]  # the population's direction at its source
            from_ghost = ghost[s]
            v = fc[ks, s]
            if gh is not None:
                v = np.where(from_ghost, gh[ks, s], v)
            if k != lat.rest:
                cut = (~from_ghost) & (ph[s] != ph[cells[inn]])
                refl = cut & (flip[inn] != 0)  # reflected at a slip wall into the other phase
                if refl.any():
                    v = v.copy()
                    v[refl] = fc[i, cells[inn][refl]]
                    cut &= ~refl
                if cut.any():
                    if finest:
                        v = v.copy()
                        v[cut] = coupling.interface_values(
                            lat, g, cells[inn][cut], np.full(cut.sum(), k), fc, ph, fluid,
                            self.phi, rho, u, S, nvec, kap, self.prm)
                    else:
                        self.stats["coarse_cut"] += int(cut.sum())
                        v = v.copy()
                        v[cut] = fc[i, cells[inn][cut]]
            val[inn] = v
            f_new[k, cells] = val
        if finest:
            if self.case["ls_active"]:
                self._levelset_and_refill(f_new, lx, lk, iface, u)
            self.fine_steps += 1
        self.f[l] = f_new
        if l < self.L - 1:
            self.ghost[l + 1] = self._ghost(l, f_old)
            self._advance(l + 1)
            self.ghost[l + 1] = self._ghost(l, 0.5 * (f_old + f_new))
            self._advance(l + 1)

    def _levelset_and_refill(self, f_new, lx, lk, iface, u):
        lat = self.lat
        gF = self.geoms[-1]
        leaf = self.masks[-1][0]
        ph_old = self.phase[-1]
        band = self.band_mask(iface)
        acc, cnt = coupling.interface_velocity_per_cell(lat, gF, lx, lk, ph_old, self.phi, u, gF.N)
        ic = cnt > 0
        self.ut[:, ic] = acc[:, ic] / cnt[ic][None, :]
        upd = np.flatnonzero(band & ~iface)
        self.ut = levelset.extend(gF, self.phi, self.ut, upd, int(self.case["n_ext"]),
                                  float(self.case["dtau_ext"]))
        bcells = np.flatnonzero(band)
        phi = levelset.advect(gF, self.phi, self.ut, bcells)
        re = int(self.case["reinit_every"])
        if re > 0 and (self.fine_steps + 1) % re == 0:
            phi = levelset.reinit(gF, lat, phi, band, int(self.case["n_reinit"]),
                                  float(self.case["dtau_reinit"]))
        self.phi = phi
        ph_new = levelset.classify(phi)
        flipped = np.flatnonzero(leaf & (ph_new != ph_old))
        if len(flipped):
            nv, kv, _, _ = levelset.fit_geometry(gF, phi, flipped)
            nvec = np.zeros((self.D, gF.N))
            kap = np.zeros(gF.N)
            nvec[:, flipped] = nv
            kap[flipped] = kv
            self.stats["refill_fail"] += coupling.refill(
                lat, gF, f_new, flipped, ph_old, ph_new, leaf, phi, nvec, kap, self.prm)
            self.stats["flipped"] += len(flipped)
        self.phase[-1] = ph_new

    # ------------------------------------------------------------ level coupling
    def _restrict(self, l):
        """Covered coarse cells that a leaf streams from get the children's mean."""
        lat = self.lat
        gc, gf = self.geoms[l], self.geoms[l + 1]
        rl = np.flatnonzero(self.masks[l][2])
        if len(rl) == 0:
            return
        ch = amr.child_cells(gc, gf, rl)
        mean = self.f[l + 1][:, ch].mean(axis=1)
        ph = self.phase[l][rl]
        fac = 2.0 * self.tau(l, ph) / self.tau(l + 1, ph)
        self.f[l][:, rl] = amr.rescale_neq(lat, mean, fac)

    def _ghost(self, l, F):
        """Post-collision populations of the ghost ring of level l+1 from coarse F."""
        lat = self.lat
        gc, gf = self.geoms[l], self.geoms[l + 1]
        ghost = self.masks[l + 1][3]
        gcells = np.flatnonzero(ghost)
        out = np.zeros((lat.Q, gf.N))
        if len(gcells) == 0:
            return out
        usable = self.masks[l][0]
        fi = amr.interpolate_coarse(lat, gc, gf, F, usable, gcells)
        ph = self.phase[l][amr.parent_cells(gc, gf, gcells)]
        fac = self.tau(l + 1, ph) / (2.0 * self.tau(l, ph))
        fi = amr.rescale_neq(lat, fi, fac)
        om, acc = self.level_params(l + 1, ph)
        out[:, gcells] = self.collide(fi, om, acc, ph)
        return out

    def regrid(self):
        """Sensor + grading, then fill new blocks / coarsened parents (Sec. 2.6)."""
        lat = self.lat
        old = self.status
        new = amr.grade(self.geoms, amr.sensor(self.geoms, self.phi, self._dists(), self.case["sensor"]))
        L = self.L
        for l in range(L - 2, -1, -1):
            gc, gf = self.geoms[l], self.geoms[l + 1]
            coars = np.flatnonzero((old[l] == amr.REFINED) & (new[l] != amr.REFINED))
            if len(coars):
                cells = np.flatnonzero(np.isin(gc.block_of, coars))
                ch = amr.child_cells(gc, gf, cells)
                mean = self.f[l + 1][:, ch].mean(axis=1)
                ph = self.phase[l][cells]
                fac = 2.0 * self.tau(l, ph) / self.tau(l + 1, ph)
                self.f[l][:, cells] = amr.rescale_neq(lat, mean, fac)
        for l in range(0, L - 1):
            gc, gf = self.geoms[l], self.geoms[l + 1]
            par = amr.block_parent(gc, gf, np.arange(gf.NB))
            newblk = np.flatnonzero((new[l][par] == amr.REFINED) & (old[l][par] != amr.REFINED))
            if len(newblk):
                cells = np.flatnonzero(np.isin(gf.block_of, newblk))
                usable = (old[l][gc.block_of] == amr.LEAF) | (new[l][gc.block_of] == amr.LEAF)
                fi = amr.interpolate_coarse(lat, gc, gf, self.f[l], usable, cells)
                ph = self.phase[l][amr.parent_cells(gc, gf, cells)]
                fac = self.tau(l + 1, ph) / (2.0 * self.tau(l, ph))
                self.f[l + 1][:, cells] = amr.rescale_neq(lat, fi, fac)
        self.status = new
        keep_fine_phase = self.phase[-1]
        self._build_masks()
        self.phase[-1] = keep_fine_phase

    # ------------------------------------------------------------ observables
    def macros(self, l=None):
        l = self.L - 1 if l is None else l
        return moments(self.lat, self.f[l])

    def observables(self):
        """Mass per phase, gas volume, centroid and rise velocity (Sec. 3.2) in finest units."""
        D = self.D
        mass = np.zeros(2)
        vol = 0.0
        xs = np.zeros(D)
        us = np.zeros(D)
        for l, g in enumerate(self.geoms):
            leaf = self.masks[l][0]
            r = 2 ** (self.L - 1 - l)
            v = float(r ** D)
            rho, u = moments(self.lat, self.f[l][:, leaf])
            ph = self.phase[l][leaf]
            for p in (0, 1):
                mass[p] += v * rho[ph == p].sum()
            gas = ph == 1
            vol += v * gas.sum()
            xs += v * g.centers(r)[:, leaf][:, gas].sum(1)
            us += v * u[:, gas].sum(1)
        cen = xs / vol if vol > 0 else np.full(D, np.nan)
        ub = us / vol if vol > 0 else np.full(D, np.nan)
        return dict(mass=mass, volume=vol, centroid=cen, velocity=ub)
