"""Discrete adjoint of the oracle's multi-level (block AMR) step with a frozen interface.

Test infrastructure (like the rest of ``oracle``): only the tests, the smoke
check and the benchmark's CPU baseline use it.

The paper has no adjoint; this module extends the frozen-interface adjoint of
oracle/adjoint.py to the block-refined grids of Sec. 2.1 (last paragraph) and
Sec. 2.6.  With the level set and the block layout held fixed (no advection,
no regrid), one coarse step is a smooth map of the per-level populations
(f_0, ..., f_{L-1}), made of, in the recursive order of the forward oracle:

* restriction: the covered coarse cells that a coarse leaf streams from get
  the mean of their 2^D children, non-equilibrium part scaled by
  2 tau_c / tau_f;
* the level's sub-step: BGK collision on leaves and restriction-layer cells,
  push streaming into leaves with half-way bounce-back at walls, plain
  bounce-back on coarse cut links, the interface treatment of Eq. bb,
  Eq. bb_cc and Eq. Sdecomp on the finest level, and pulls from the ghost
  ring of the level;
* twice per coarse sub-step, the ghost ring of the next finer level:
  coarse populations at t and at t + 1/2 (the mean of old and new),
  linearly interpolated in space, non-equilibrium part scaled by
  tau_f / (2 tau_c), then collided with the fine level's parameters;
  each followed by a sub-step of the finer level.

The relaxation times depend on the viscosities, so the two rescale factors
carry parameter derivatives of their own.  ``AMRFrozenStep.step_adjoint``
applies the transpose of this map by reversing the recursion: the second
fine sub-step first, the ghost transfer of t + 1/2 splitting its adjoint
between the old and new coarse states, the first fine sub-step, the ghost
transfer of t, the coarse sub-step, and last the restriction, whose adjoint
goes to the fine state the restriction read.  Pins in
tests/test_oracle_adjoint_amr.py: the step against the forward oracle, the
dot-product identity <J v, w> = <v, J^T w> of one coarse step with J v from
central differences, every parameter derivative and window gradients
against central differences of the objective in float64.
"""
import numpy as np

from . import amr
from . import objective as indicator
from .adjoint import NPARAM, FrozenStep, params_of  # noqa: F401  (params_of re-exported)
from .lattice import CS2
from .lbm import collide, equilibrium, moments, omega_from_nu


# --------------------------------------------------------------------------- building blocks
def feq_T(lat, f, lam):
    """d/df of <lam, f^eq(rho(f), u(f))> per cell (the chain rule through the moments)."""
    rho, u = moments(lat, f)
    feq = equilibrium(lat, rho, u)
    cu = lat.cf @ u
    out = np.repeat((lam * feq).sum(0)[None, :] / rho[None, :], lat.Q, 0)  # d f^eq / d rho, d rho / d f_j = 1
    for a in range(lat.D):
        # d f^eq_q / d u_a = w_q rho (c_qa / cs2 + (c_q . u) c_qa / cs2^2 - u_a / cs2)
        d = lat.w[:, None] * rho[None, :] * (lat.cf[:, a][:, None] / CS2 + cu * lat.cf[:, a][:, None] / CS2 ** 2
                                             - u[a][None, :] / CS2)
        B = (lam * d).sum(0)
        out += B[None, :] * (lat.cf[:, a][:, None] - u[a][None, :]) / rho[None, :]  # d u_a / d f_j
    return out


def collide_T(lat, f, om, acc, lc):
    """Transpose of f -> f + om (f^eq - f) + w rho (c . acc) / cs2 applied to lc:
    (lam_f, dJ/d om per cell, dJ/d acc (D, N))."""
    rho, u = moments(lat, f)
    feq = equilibrium(lat, rho, u)
    lam = (1.0 - om)[None, :] * lc + feq_T(lat, f, om[None, :] * lc)
    lam += (lc * lat.w[:, None] * (lat.cf @ acc)).sum(0)[None, :] / CS2  # the forcing's rho
    l_om = (lc * (feq - f)).sum(0)
    l_acc = np.einsum("qn,qa->an", lc * lat.w[:, None] * rho[None, :], lat.cf) / CS2
    return lam, l_om, l_acc


def rescale_T(lat, f, fac, lam):
    """Transpose of f -> f^eq + fac (f - f^eq): (lam_f, dJ/d fac per cell)."""
    rho, u = moments(lat, f)
    feq = equilibrium(lat, rho, u)
    out = fac[None, :] * lam + feq_T(lat, f, (1.0 - fac)[None, :] * lam)
    return out, (lam * (f - feq)).sum(0)


def interpolate_T(gc, gf, usable, fine_cells, lam, Nc):
    """Transpose of amr.interpolate_coarse: adjoint (Q, Nc) of the coarse field
    from the adjoint ``lam`` (Q, len(fine_cells)) of the interpolated values."""
    par = amr.parent_cells(gc, gf, fine_cells)
    Q = lam.shape[0]
    out = np.zeros((Q, Nc))
    for q in range(Q):
        np.add.at(out[q], par, lam[q])
    for a in range(gc.D):
        e = np.zeros(gc.D, dtype=np.int64)
        e[a] = 1
        delta = (gf.coord[a, fine_cells] % 2 - 0.5) / 2.0
        up, _ = gc.shift(par, e)
        dn, _ = gc.shift(par, -e)
        upok = up >= 0
        upok[upok] = usable[up[upok]]
        dnok = dn >= 0
        dnok[dnok] = usable[dn[dnok]]
        both = upok & dnok
        only_up = upok & ~dnok
        only_dn = dnok & ~upok
        # grad = 0.5 (F_up - F_dn) | F_up - F_par | F_par - F_dn | 0
        w_up = np.where(both, 0.5, np.where(only_up, 1.0, 0.0)) * delta
        w_dn = np.where(both, -0.5, np.where(only_dn, -1.0, 0.0)) * delta
        w_par = np.where(only_up, -1.0, np.where(only_dn, 1.0, 0.0)) * delta
        for q in range(Q):
            np.add.at(out[q], up[upok], (w_up * lam[q])[upok])
            np.add.at(out[q], dn[dnok], (w_dn * lam[q])[dnok])
            np.add.at(out[q], par, w_par * lam[q])
    return out


# --------------------------------------------------------------------------- coarse levels
class CoarseLevel:
    """Sub-step of a level l < L-1 with a frozen interface: BGK collision with
    forcing on leaves and restriction-layer cells, push streaming into leaves
    with half-way bounce-back at walls (moving lid), plain bounce-back where the
    source lies in the other phase, and the ghost ring's values where the
    source is a ghost cell.  Parameters scale with the level as in the forward
    oracle (acoustic scaling: nu / r, acceleration * r, r = 2^(L-1-l))."""

    def __init__(self, sim, l):
        self.l = l
        self.lat = lat = sim.lat
        self.g = g = sim.geoms[l]
        self.leaf, self.covered, self.rlayer, self.ghostm = (m.copy() for m in sim.masks[l])
        self.coll = self.leaf | self.rlayer
        self.phase = sim.phase[l].copy()
        self.r = 2.0 ** (sim.L - 1 - l)
        self.gravity, self.body_force, self.wall_u = sim.gravity.copy(), sim.body_force.copy(), sim.wall_u.copy()
        cells = np.arange(g.N)
        self.src, self.same, self.fg, self.cut, self.wall = [], [], [], [], []
        for k in range(lat.Q):
            src, face, flip = g.pull(cells, lat.c[k])  # reflected at slip walls
            ok = (src >= 0) & self.leaf
            s = np.where(ok, src, 0)
            fg = ok & self.ghostm[s]
            cut = ok & ~fg & (self.phase[s] != self.phase) & (k != lat.rest)
            self.src.append((src, face, lat.mirror[k, flip]))
            self.fg.append(fg)
            self.cut.append(cut)
            self.same.append(ok & ~fg & ~cut)
            self.wall.append((src < 0) & self.leaf)

    def cell_params(self, p):
        ph, r = self.phase, self.r
        om = omega_from_nu(p[3:5][ph] / r)
        acc = (self.gravity[:, None] + self.body_force[:, None] / p[1:3][ph][None, :]) * r
        return om, acc

    def step(self, f, p, gh):
        lat = self.lat
        om, acc = self.cell_params(p)
        c = self.coll
        fc = np.zeros_like(f)
        fc[:, c] = collide(lat, f[:, c], om[c], acc[:, c])
        fn = f.copy()
        for k in range(lat.Q):
            i = lat.opp[k]
            src, face, ks = self.src[k]
            same, fg, cut, wall = self.same[k], self.fg[k], self.cut[k], self.wall[k]
            fn[k, same] = fc[ks[same], src[same]]
            if fg.any():
                fn[k, fg] = gh[ks[fg], src[fg]]
            if cut.any():
                fn[k, cut] = fc[i, cut]
            if wall.any():
                fn[k, wall] = fc[i, wall] - (2 * lat.w[i] / CS2) * (self.wall_u[face[wall]] @ lat.cf[i])
        return fn

    def step_adjoint(self, f, p, lam_next, lam_gh):
        """(lam_n, dJ/dp); accumulates the ghost ring's adjoint into lam_gh."""
        lat = self.lat
        om, acc = self.cell_params(p)
        lc = np.zeros_like(f)
        for k in range(lat.Q):
            i = lat.opp[k]
            src, _, ks = self.src[k]
            same, fg, cut, wall = self.same[k], self.fg[k], self.cut[k], self.wall[k]
            np.add.at(lc, (ks[same], src[same]), lam_next[k, same])
            np.add.at(lam_gh, (ks[fg], src[fg]), lam_next[k, fg])
            lc[i, cut] += lam_next[k, cut]
            lc[i, wall] += lam_next[k, wall]
        c = self.coll
        lam = np.zeros_like(f)
        lam[:, c], l_om, l_acc = collide_T(lat, f[:, c], om[c], acc[:, c], lc[:, c])
        lam[:, ~self.leaf] += lam_next[:, ~self.leaf]  # non-leaf cells keep their values
        dp = np.zeros(NPARAM)
        ph = self.phase[c]
        rp, nu = p[1:3], p[3:5]
        for s in (0, 1):
            m = ph == s
            om_s = omega_from_nu(nu[s] / self.r)
            dp[3 + s] += l_om[m].sum() * (-om_s * om_s / CS2) / self.r
            dp[1 + s] += (l_acc[:, m].sum(1) * (-self.body_force * self.r / rp[s] ** 2)).sum()
        return lam, dp


# --------------------------------------------------------------------------- the coarse step
def _tau(nu, r):
    """tau of a level with grid ratio r to the finest level, and d tau / d nu."""
    return 1.0 / omega_from_nu(nu / r), 1.0 / (r * CS2)


class AMRFrozenStep:
    """One coarse step of a multi-level Sim with the level set and blocks held fixed."""

    def __init__(self, sim, phi=None, eps=None):
        """``eps``: None for the sharp gas indicator in the observables, else the width of
        the smoothed indicator H_eps (oracle/objective.py)."""
        self.eps = eps
        self.sim = sim
        self.lat = sim.lat
        self.L = L = sim.L
        self.D = sim.D
        self.geoms = sim.geoms
        self.fine = FrozenStep(sim, phi)
        self.levels = [CoarseLevel(sim, l) for l in range(L - 1)] + [self.fine]
        self.leaf = [sim.masks[l][0].copy() for l in range(L)]
        self.phase = [sim.phase[l].copy() for l in range(L)]
        self.r = [2.0 ** (L - 1 - l) for l in range(L)]
        self.tr = []
        for l in range(L - 1):
            gc, gf = sim.geoms[l], sim.geoms[l + 1]
            rl = np.flatnonzero(sim.masks[l][2])
            gcells = np.flatnonzero(sim.masks[l + 1][3])
            par = amr.parent_cells(gc, gf, gcells) if len(gcells) else np.zeros(0, dtype=np.int64)
            self.tr.append(dict(rl=rl, ch=amr.child_cells(gc, gf, rl), ph_r=self.phase[l][rl],
                                gcells=gcells, ph_g=self.phase[l][par], usable=self.leaf[l].copy()))

    # ---------------------------------------------------------------- transfers
    def _fac_r(self, l, ph, p):
        """2 tau_c / tau_f per restricted cell and its derivative in nu[ph]."""
        tc, dc = _tau(p[3:5][ph], self.r[l])
        tf, df = _tau(p[3:5][ph], self.r[l + 1])
        return 2.0 * tc / tf, 2.0 * (dc * tf - tc * df) / (tf * tf)

    def _fac_g(self, l, ph, p):
        """tau_f / (2 tau_c) per ghost cell and its derivative in nu[ph]."""
        tc, dc = _tau(p[3:5][ph], self.r[l])
        tf, df = _tau(p[3:5][ph], self.r[l + 1])
        return tf / (2.0 * tc), (df * tc - tf * dc) / (2.0 * tc * tc)

    def _ghost_params(self, l, ph, p):
        r = self.r[l + 1]
        om = omega_from_nu(p[3:5][ph] / r)
        acc = (self.sim.gravity[:, None] + self.sim.body_force[:, None] / p[1:3][ph][None, :]) * r
        return om, acc

    def _restrict(self, l, Ff, p):
        t = self.tr[l]
        mean = Ff[:, t["ch"]].mean(axis=1)
        fac, _ = self._fac_r(l, t["ph_r"], p)
        return amr.rescale_neq(self.lat, mean, fac)

    def _restrict_T(self, l, Ff, p, lam_rl, dp):
        t = self.tr[l]
        ch, ph = t["ch"], t["ph_r"]
        nch = ch.shape[0]
        mean = Ff[:, ch].mean(axis=1)
        fac, dfac = self._fac_r(l, ph, p)
        lm, l_fac = rescale_T(self.lat, mean, fac, lam_rl)
        for s in (0, 1):
            dp[3 + s] += (l_fac * dfac)[ph == s].sum()
        out = np.zeros_like(Ff)
        for j in range(nch):
            out[:, ch[j]] += lm / nch  # the children of distinct cells are distinct
        return out

    def _ghost(self, l, F, p):
        t = self.tr[l]
        lat = self.lat
        gf = self.geoms[l + 1]
        out = np.zeros((lat.Q, gf.N))
        gcells = t["gcells"]
        if len(gcells) == 0:
            return out
        fi = amr.interpolate_coarse(lat, self.geoms[l], gf, F, t["usable"], gcells)
        fac, _ = self._fac_g(l, t["ph_g"], p)
        fr = amr.rescale_neq(lat, fi, fac)
        om, acc = self._ghost_params(l, t["ph_g"], p)
        out[:, gcells] = collide(lat, fr, om, acc)
        return out

    def _ghost_T(self, l, F, p, lam_gh, dp):
        """Adjoint of the coarse field F from the ghost ring's adjoint lam_gh."""
        t = self.tr[l]
        lat = self.lat
        gc, gf = self.geoms[l], self.geoms[l + 1]
        gcells, ph = t["gcells"], t["ph_g"]
        if len(gcells) == 0:
            return np.zeros_like(F)
        fi = amr.interpolate_coarse(lat, gc, gf, F, t["usable"], gcells)
        fac, dfac = self._fac_g(l, ph, p)
        fr = amr.rescale_neq(lat, fi, fac)
        om, acc = self._ghost_params(l, ph, p)
        lr, l_om, l_acc = collide_T(lat, fr, om, acc, lam_gh[:, gcells])
        li, l_fac = rescale_T(lat, fi, fac, lr)
        rp, nu = p[1:3], p[3:5]
        r = self.r[l + 1]
        for s in (0, 1):
            m = ph == s
            om_s = omega_from_nu(nu[s] / r)
            dp[3 + s] += l_om[m].sum() * (-om_s * om_s / CS2) / r + (l_fac * dfac)[m].sum()
            dp[1 + s] += (l_acc[:, m].sum(1) * (-self.sim.body_force * r / rp[s] ** 2)).sum()
        return interpolate_T(gc, gf, t["usable"], gcells, li, gc.N)

    # ---------------------------------------------------------------- forward
    def _advance(self, l, F, p, gh, rec):
        last = l == self.L - 1
        if not last:
            rec["fine_in"] = F[l + 1].copy()
            rl = self.tr[l]["rl"]
            if len(rl):
                F[l][:, rl] = self._restrict(l, F[l + 1], p)
        f_old = F[l].copy()
        rec["f_old"], rec["gh"] = f_old, gh
        F[l] = self._level_step(l, f_old, p, gh, rec)
        if not last:
            rec["f_new"] = F[l].copy()
            rec["kids"] = []
            for src in (f_old, 0.5 * (f_old + F[l])):
                kid = {}
                self._advance(l + 1, F, p, self._ghost(l, src, p), kid)
                rec["kids"].append(kid)

    def _level_step(self, l, f_old, p, gh, rec):
        return self.levels[l].step(f_old, p, gh)

    def _level_step_T(self, l, f_old, p, lam_new, lam_gh, geo, rec):
        if l == self.L - 1:
            return self.fine.step_adjoint(f_old, p, lam_new, geo, lam_gh)
        return self.levels[l].step_adjoint(f_old, p, lam_new, lam_gh)

    def step(self, F, p, rec=None):
        """The per-level populations after one coarse step."""
        F = [f.copy() for f in F]
        self._advance(0, F, p, None, {} if rec is None else rec)
        return F

    # ---------------------------------------------------------------- adjoint
    def _advance_T(self, l, lamF, p, rec, dp, geo):
        """Reverse of _advance(l): lamF[l:] go from the adjoints of the states after
        the call to those before it; returns the adjoint of the ghost values gh."""
        Q = self.lat.Q
        last = l == self.L - 1
        lam_new = lamF[l].copy()
        lam_old_extra = np.zeros_like(lam_new)
        f_old = rec["f_old"]
        if not last:
            mid = 0.5 * (f_old + rec["f_new"])
            lg = self._advance_T(l + 1, lamF, p, rec["kids"][1], dp, geo)
            lm = self._ghost_T(l, mid, p, lg, dp)
            lam_new += 0.5 * lm
            lam_old_extra += 0.5 * lm
            lg = self._advance_T(l + 1, lamF, p, rec["kids"][0], dp, geo)
            lam_old_extra += self._ghost_T(l, f_old, p, lg, dp)
        lam_gh = np.zeros((Q, self.geoms[l].N))
        lam_old, d = self._level_step_T(l, f_old, p, lam_new, lam_gh, geo, rec)
        dp += d
        lam_old += lam_old_extra
        if not last:
            rl = self.tr[l]["rl"]
            if len(rl):
                lam_rl = lam_old[:, rl].copy()
                lam_old[:, rl] = 0.0  # the restriction overwrote these values
                lamF[l + 1] += self._restrict_T(l, rec["fine_in"], p, lam_rl, dp)
        lamF[l] = lam_old
        return lam_gh

    def step_adjoint(self, F, p, lamF, geo=None):
        """(lam_n, dJ/dp): the transpose of one coarse step's Jacobian at F applied
        to the per-level adjoints lamF.  ``geo`` as in FrozenStep.step_adjoint
        (the finest level's frozen geometry)."""
        rec = {}
        self.step(F, p, rec)
        lam = [x.copy() for x in lamF]
        dp = np.zeros(NPARAM)
        self._advance_T(0, lam, p, rec, dp, geo)
        return lam, dp

    # ---------------------------------------------------------------- observables
    def observables(self, F, phi=None):
        """liquid mass, gas mass, gas volume, leaf updates per coarse step, centroid (D),
        gas velocity (D); sums over the leaves of all levels in finest-cell units."""
        if self.eps is not None:
            phi = self.fine.phi if phi is None else phi
            return indicator.observables(self.lat, indicator.levels_of(self.sim), F, phi, self.eps)
        D = self.D
        mass = np.zeros(2)
        vol, nupd = 0.0, 0.0
        xs, us = np.zeros(D), np.zeros(D)
        for l, g in enumerate(self.geoms):
            leaf, r = self.leaf[l], self.r[l]
            v = r ** D
            rho, u = moments(self.lat, F[l][:, leaf])
            ph = self.phase[l][leaf]
            for s in (0, 1):
                mass[s] += v * rho[ph == s].sum()
            gas = ph == 1
            vol += v * gas.sum()
            nupd += leaf.sum() * 2.0 ** l
            xs += v * g.centers(r)[:, leaf][:, gas].sum(1)
            us += v * u[:, gas].sum(1)
        return np.concatenate([mass, [vol, nupd], xs / vol, us / vol])

    def observables_phi_adjoint(self, F, a, phi=None):
        """dJ/dphi (finest level) of J = a . observables at fixed populations."""
        if self.eps is None:
            return np.zeros(self.geoms[-1].N)
        phi = self.fine.phi if phi is None else phi
        return indicator.observables_adjoint(self.lat, indicator.levels_of(self.sim), F, phi, self.eps, a)[1]

    def observables_adjoint(self, F, a, phi=None):
        if self.eps is not None:
            phi = self.fine.phi if phi is None else phi
            return indicator.observables_adjoint(self.lat, indicator.levels_of(self.sim), F, phi, self.eps, a)[0]
        D = self.D
        a = np.asarray(a, dtype=np.float64)
        vol = sum((self.r[l] ** D) * (self.leaf[l] & (self.phase[l] == 1)).sum() for l in range(self.L))
        au = a[4 + D:4 + 2 * D]
        out = []
        for l in range(self.L):
            lat = self.lat
            v = self.r[l] ** D
            rho, u = moments(lat, F[l])
            lam = np.zeros_like(F[l])
            liq = self.leaf[l] & (self.phase[l] == 0)
            gas = self.leaf[l] & (self.phase[l] == 1)
            lam[:, liq] += v * a[0]
            lam[:, gas] += v * a[1]
            lam[:, gas] += v * ((lat.cf @ au)[:, None] - (au @ u[:, gas])[None, :]) / rho[gas][None, :] / vol
            out.append(lam)
        return out

    def geometry_to_phi(self, geo):
        return self.fine.geometry_to_phi(geo)


# --------------------------------------------------------------------------- moving level set
class AMRMovingStep(AMRFrozenStep):
    """One coarse step of a multi-level Sim with the finest level's level set transported.

    The state is (per-level populations, phi, u~); phi and u~ live on the finest level and
    advance in each of its 2^(L-1) sub-steps (oracle/adjoint_ls.py's MovingStep, with the
    ghost-ring values an input).  As there, the window must keep every discrete decision:
    no cell changes phase (so refill is the identity and the coarse levels' phases, fixed at
    the last regrid, stay valid), the band, frozen cells, upwind sides and Godunov branches
    stay those of the forward steps; blocks do not regrid.  The reverse recursion is the
    frozen one with the finest sub-step's transpose replaced by MovingStep's, which carries
    the adjoints of phi and u~ from sub-step to sub-step."""

    def __init__(self, sim, eps=None):
        super().__init__(sim, eps=eps)
        from .adjoint_ls import MovingStep
        self.moving = MovingStep(sim)

    def _level_step(self, l, f_old, p, gh, rec):
        if l < self.L - 1:
            return self.levels[l].step(f_old, p, gh)
        rec["ls"] = (self._ls[0], self._ls[1])
        f1, phi1, ut1 = self.moving.step((f_old, self._ls[0], self._ls[1]), p, gh)
        self._ls = [phi1, ut1]
        return f1

    def _level_step_T(self, l, f_old, p, lam_new, lam_gh, geo, rec):
        if l < self.L - 1:
            return self.levels[l].step_adjoint(f_old, p, lam_new, lam_gh)
        phi, ut = rec["ls"]
        (lf, lphi, lut), d = self.moving.step_adjoint((f_old, phi, ut), p, (lam_new, self._lls[0], self._lls[1]),
                                                      lam_gh)
        self._lls = [lphi, lut]
        return lf, d

    def step(self, S, p, rec=None):
        """(per-level populations, phi, u~) after one coarse step."""
        F = [f.copy() for f in S[0]]
        self._ls = [S[1].copy(), S[2].copy()]
        self._advance(0, F, p, None, {} if rec is None else rec)
        return (F, self._ls[0], self._ls[1])

    def step_adjoint(self, S, p, LAM, geo=None):
        """Adjoints of (populations, phi, u~) at the step's start, and dJ/dp."""
        rec = {}
        self.step(S, p, rec)
        lam = [x.copy() for x in LAM[0]]
        self._lls = [LAM[1].copy(), LAM[2].copy()]
        dp = np.zeros(NPARAM)
        self._advance_T(0, lam, p, rec, dp, None)
        return (lam, self._lls[0], self._lls[1]), dp

    def observables(self, S):
        return AMRFrozenStep.observables(self, S[0], S[1])

    def observables_adjoint(self, S, a):
        N = self.geoms[-1].N
        return (AMRFrozenStep.observables_adjoint(self, S[0], a, S[1]),
                AMRFrozenStep.observables_phi_adjoint(self, S[0], a, S[1]), np.zeros((self.D, N)))


# --------------------------------------------------------------------------- windows
def trajectory(step, F0, p, nsteps):
    if isinstance(F0, tuple):  # (populations, phi, u~): steps return new arrays
        out = [F0]
        for _ in range(nsteps):
            out.append(step.step(out[-1], p))
        return out
    out = [[f.copy() for f in F0]]
    for _ in range(nsteps):
        out.append(step.step(out[-1], p))
    return out


def objective(step, F0, p, nsteps, a):
    return float(np.asarray(a) @ step.observables(trajectory(step, F0, p, nsteps)[-1]))


def gradients(step, F0, p, nsteps, a, want_phi=False):
    """J = a . observables(F_N), dJ/dp and dJ/dF_0 (per level), plus dJ/dphi of
    the finest level's frozen level set with ``want_phi``."""
    a = np.asarray(a, dtype=np.float64)
    tr = trajectory(step, F0, p, nsteps)
    J = float(a @ step.observables(tr[-1]))
    lam = step.observables_adjoint(tr[-1], a)
    dp = np.zeros(NPARAM)
    N = step.geoms[-1].N
    geo = dict(phi=np.zeros(N), n=np.zeros((step.D, N)), kappa=np.zeros(N)) if want_phi else None
    for n in range(nsteps - 1, -1, -1):
        lam, d = step.step_adjoint(tr[n], p, lam, geo)
        dp += d
    if want_phi:
        return J, dp, lam, step.geometry_to_phi(geo) + step.observables_phi_adjoint(tr[-1], a)
    return J, dp, lam
