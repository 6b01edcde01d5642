"""Discrete adjoint of the oracle's single-level step with a MOVING level set.

Test infrastructure (like the rest of ``oracle``).

The paper has no adjoint; this module extends ``adjoint.FrozenStep`` to the
full step of Sec. 2 with the level set transported: the state is
(f, phi, u~) and one step maps it through

  1. the lattice Boltzmann step with the interface geometry (q, n, kappa) of
     phi_n (``adjoint.FrozenStep`` built on phi_n);
  2. u~ on interface cells = mean of u_I = (1 - q) u(x) + q u(y) over their
     cut links, u from the pre-collision moments of f_n;
  3. ``n_ext`` Jacobi sweeps of the first-order upwind extension on the other
     band cells (Eq. hyperbolicExtension), velocity S(phi) n(phi);
  4. TVD-RK3 transport of phi with the upwind-biased fifth-order stencil;
  5. one constrained HJ-WENO5 reinitialisation pseudo step (TVD-RK3).

What stays fixed is what the paper's method decides discretely: phases, cut
links, band, the upwind side of every stencil (sign of the velocity, of
S(phi0), Godunov's branch), the frozen cells of the reinitialisation, and
refill (windows without flipped cells; ``MovingStep.step`` raises if a cell
flips).  On such windows the map is smooth and ``step_adjoint`` applies the
transpose of its Jacobian, written out pass by pass in the forward's order
reversed.  Pins (tests/test_oracle_adjoint_ls.py): MovingStep.step equals
Sim.step; the one-step dot-product identity for each state component and
every parameter; central differences of a window objective in every
parameter, in f_0, phi_0 and u~_0.
"""
import numpy as np

from .adjoint import NPARAM, FrozenStep, params_of
from .coupling import interface_velocity_per_cell
from .lattice import CS2
from .lbm import moments
from .levelset import OFF5, W5, WENO_EPS, _unit, advect, extend, frozen_cells, reinit

__all__ = ["MovingStep", "NPARAM", "params_of", "gradients", "objective"]


# --------------------------------------------------------------------------- WENO5 gradient
def _weno5_grad(v):
    """HJ-WENO5 value and its partial derivatives in the five differences v (5, M)."""
    v1, v2, v3, v4, v5 = v
    e = [np.array([1 / 3, -7 / 6, 11 / 6, 0, 0]), np.array([0, -1 / 6, 5 / 6, 1 / 3, 0]),
         np.array([0, 0, 1 / 3, 5 / 6, -1 / 6])]
    b = [np.array([1, -2, 1, 0, 0.0]), np.array([0, 1, -2, 1, 0.0]), np.array([0, 0, 1, -2, 1.0])]
    c = [np.array([1, -4, 3, 0, 0.0]), np.array([0, 1, 0, -1, 0.0]), np.array([0, 0, 3, -4, 1.0])]
    gam = [0.1, 0.6, 0.3]
    d, s, a, da = [], [], [], []
    for k in range(3):
        dk = e[k] @ v
        bv, cv = b[k] @ v, c[k] @ v
        sk = 13.0 / 12.0 * bv ** 2 + 0.25 * cv ** 2
        dsk = 13.0 / 6.0 * bv[None, :] * b[k][:, None] + 0.5 * cv[None, :] * c[k][:, None]  # (5, M)
        ak = gam[k] / (sk + WENO_EPS) ** 2
        dak = -2.0 * gam[k] / (sk + WENO_EPS) ** 3 * dsk
        d.append(dk), s.append(sk), a.append(ak), da.append(dak)
    A = a[0] + a[1] + a[2]
    val = (a[0] * d[0] + a[1] * d[1] + a[2] * d[2]) / A
    grad = np.zeros_like(v)
    for k in range(3):
        grad += (a[k] / A)[None, :] * e[k][:, None] + ((d[k] - val) / A)[None, :] * da[k]
    return val, grad


# --------------------------------------------------------------------------- linear stencils
def _d5_table(geom, cells, a, side):
    """Neighbour indices and coefficients of d5 (levelset.d5) at cells: d5 = sum coef phi[nb]."""
    nbs, cfs = [], []
    for wgt, o in zip(W5, OFF5):
        nbs.append(geom.clamp_shift(cells, _unit(geom.D, a, -side * o)))
        cfs.append(-side * wgt)
    return nbs, cfs


def _rk3_adjoint(lam3, cells, stages, dt, rhs_T):
    """Transpose of levelset.rk3 (Shu-Osher TVD-RK3 on ``cells``; other cells keep p0).

    stages: (p0, p1, p2); rhs_T(p, mu) adds, for the stage value p, the transpose
    of the right-hand side's Jacobian applied to mu (values on cells) and returns
    it as a full-length array.  Returns the adjoint of p0."""
    p0, p1, p2 = stages
    lp0 = lam3.copy()
    mu3 = lam3[cells]
    lp0[cells] = mu3 / 3.0
    lp2 = np.zeros_like(lam3)
    lp2[cells] += 2.0 / 3.0 * mu3
    lp2 += rhs_T(p2, 2.0 / 3.0 * dt * mu3)
    mu2 = lp2[cells].copy()
    off = np.ones(len(lam3), dtype=bool)
    off[cells] = False
    lp0[off] += lp2[off]
    lp0[cells] += 0.75 * mu2
    lp1 = np.zeros_like(lam3)
    lp1[cells] += 0.25 * mu2
    lp1 += rhs_T(p1, 0.25 * dt * mu2)
    mu1 = lp1[cells].copy()
    lp0[off] += lp1[off]
    lp0[cells] += mu1
    lp0 += rhs_T(p0, dt * mu1)
    return lp0


def _rk3_stages(p0, cells, rhs, dt):
    p1 = p0.copy()
    p1[cells] = p0[cells] + dt * rhs(p0)
    p2 = p0.copy()
    p2[cells] = 0.75 * p0[cells] + 0.25 * (p1[cells] + dt * rhs(p1))
    p3 = p0.copy()
    p3[cells] = p0[cells] / 3.0 + (2.0 / 3.0) * (p2[cells] + dt * rhs(p2))
    return (p0, p1, p2), p3


# --------------------------------------------------------------------------- the moving step
class MovingStep:
    """Step and transposed step of the finest level of a Sim with the level set transported
    (the whole step on a single-level grid; on a multi-level grid one finest sub-step, whose
    ghost-ring values are an input, see oracle/adjoint_amr.py)."""

    def __init__(self, sim, eps=None):
        """``eps``: None for the sharp gas indicator in the observables, else the width of
        the smoothed indicator H_eps (oracle/objective.py), which makes volume, centroid and
        velocity depend on phi."""
        c = sim.case
        assert c["ls_active"], "the level set must be live"
        self.eps = eps
        assert int(c["reinit_every"]) in (0, 1), "reinitialisation every step or never"
        self.sim = sim
        self.g = g = sim.geoms[-1]
        self.lat = lat = sim.lat
        self.D = lat.D
        self.phase = sim.phase[-1].copy()
        self.leaf = sim.masks[-1][0].copy()
        self.lx, self.lk = sim.cut_links(self.phase, self.leaf)
        iface = np.zeros(g.N, dtype=bool)
        iface[self.lx] = True
        self.iface = iface
        self.band = sim.band_mask(iface)
        self.bcells = np.flatnonzero(self.band)
        self.upd = np.flatnonzero(self.band & ~iface)
        self.n_ext, self.dtau_ext = int(c["n_ext"]), float(c["dtau_ext"])
        self.reinit_on = int(c["reinit_every"]) == 1 and int(c["n_reinit"]) > 0
        self.n_reinit, self.dtau_reinit = int(c["n_reinit"]), float(c["dtau_reinit"])
        self.frozen = frozen_cells(g, lat, sim.phi)
        self.rcells = np.flatnonzero(self.band & ~self.frozen)
        # link partners of the interface velocity
        i = lat.opp[self.lk]
        self.ly, _ = g.shift(self.lx, lat.c[i].T)
        cnt = np.zeros(g.N)
        np.add.at(cnt, self.lx, 1.0)
        self.cnt = cnt

    def frozen_step(self, phi):
        return FrozenStep(self.sim, phi)

    # ------------------------------------------------------------------ forward
    def _forward_ls(self, f, phi, ut):
        """Level-set part of the step with every intermediate (from phi_n, u(f_n), u~_n)."""
        g, lat = self.g, self.lat
        rho, u = moments(lat, f)
        acc, cnt = interface_velocity_per_cell(lat, g, self.lx, self.lk, self.phase, phi, u, g.N)
        ut0 = ut.copy()
        ic = cnt > 0
        ut0[:, ic] = acc[:, ic] / cnt[ic]
        sweeps = [ut0]
        for _ in range(self.n_ext):
            sweeps.append(extend(g, phi, sweeps[-1], self.upd, 1, self.dtau_ext))
        ut1 = sweeps[-1]
        from .levelset import advect_rhs
        adv_st, ps = _rk3_stages(phi, self.bcells, lambda p: advect_rhs(g, p, ut1, self.bcells), 1.0)
        rein = []
        phi1 = ps
        if self.reinit_on:
            fr = frozen_cells(g, lat, ps)
            if not np.array_equal(fr, self.frozen):
                raise ValueError("the frozen cells of the reinitialisation changed")
            from .levelset import reinit_rhs
            s0 = ps[self.rcells] / np.sqrt(ps[self.rcells] ** 2 + 1.0)
            for _ in range(self.n_reinit):
                st, phi1 = _rk3_stages(phi1, self.rcells, lambda p: reinit_rhs(g, p, s0, self.rcells),
                                       self.dtau_reinit)
                rein.append(st)
        return dict(rho=rho, u=u, ut0=ut0, sweeps=sweeps, ut1=ut1, adv=adv_st, ps=ps, rein=rein, phi1=phi1)

    def step(self, state, p, gh=None):
        f, phi, ut = state
        f1 = self.frozen_step(phi).step(f, p, gh)
        F = self._forward_ls(f, phi, ut)
        if not np.array_equal(F["phi1"][self.leaf] >= 0, phi[self.leaf] >= 0):
            raise ValueError("a cell changed phase: the window must be free of flips")
        return (f1, F["phi1"], F["ut1"])

    def observables(self, state):
        return FrozenStep(self.sim, state[1], self.eps).observables(state[0])

    # ------------------------------------------------------------------ transposes of the passes
    def _reinit_T(self, lam, F):
        """Adjoint of the constrained reinitialisation: (adjoint of phi*, including S(phi*))."""
        g, D = self.g, self.D
        cells = self.rcells
        ps = F["ps"]
        s0 = ps[cells] / np.sqrt(ps[cells] ** 2 + 1.0)
        pos = s0 > 0.0
        l_s0 = np.zeros(len(cells))

        def rhs_T(p, mu):
            nonlocal l_s0
            out = np.zeros(g.N)
            g2 = np.zeros(len(cells))
            parts = []
            for a in range(D):
                for side in (-1, 1):
                    pts = [g.clamp_shift(cells, _unit(D, a, -side * o)) for o in range(-3, 3)]
                    v = np.stack([(-side) * (p[pts[m + 1]] - p[pts[m]]) for m in range(5)])
                    val, grad = _weno5_grad(v)
                    parts.append((a, side, pts, val, grad))
            dgs = []
            for a in range(D):
                _, _, _, dm, _ = parts[2 * a]
                _, _, _, dpv, _ = parts[2 * a + 1]
                gp_m, gp_p = np.maximum(dm, 0.0) ** 2, np.minimum(dpv, 0.0) ** 2
                gn_m, gn_p = np.minimum(dm, 0.0) ** 2, np.maximum(dpv, 0.0) ** 2
                use_m = np.where(pos, gp_m >= gp_p, gn_m >= gn_p)
                ga = np.where(pos, np.maximum(gp_m, gp_p), np.maximum(gn_m, gn_p))
                g2 += ga
                # d ga / d dm and d ga / d dp on the selected branch
                d_dm = np.where(use_m, 2.0 * np.where(pos, np.maximum(dm, 0.0), np.minimum(dm, 0.0)), 0.0)
                d_dp = np.where(use_m, 0.0, 2.0 * np.where(pos, np.minimum(dpv, 0.0), np.maximum(dpv, 0.0)))
                dgs.append((d_dm, d_dp))
            sq = np.sqrt(g2)
            l_s0 += mu * (-(sq - 1.0))
            l_g2 = mu * np.where(sq > 0.0, -s0 / (2.0 * np.where(sq > 0.0, sq, 1.0)), 0.0)
            for a in range(D):
                for j, side in enumerate((-1, 1)):
                    _, _, pts, val, grad = parts[2 * a + j]
                    lw = l_g2 * dgs[a][j]
                    for m in range(5):  # v_m = -side (p[m+1] - p[m])
                        np.add.at(out, pts[m + 1], lw * grad[m] * (-side))
                        np.add.at(out, pts[m], lw * grad[m] * side)
            return out

        lps = lam
        for st in reversed(F["rein"]):
            lps = _rk3_adjoint(lps, cells, st, self.dtau_reinit, rhs_T)
        lps = lps.copy()
        lps[cells] += l_s0 / (ps[cells] ** 2 + 1.0) ** 1.5
        return lps

    def _advect_T(self, lam, F):
        """Adjoint of the TVD-RK3 transport: (adjoint of phi_n, adjoint of u~)."""
        g, D = self.g, self.D
        cells = self.bcells
        ut1 = F["ut1"]
        l_ut = np.zeros((D, g.N))
        tabs = []
        for a in range(D):
            ua = ut1[a, cells]
            tm, tp = _d5_table(g, cells, a, -1), _d5_table(g, cells, a, +1)
            use_m = ua >= 0.0
            nbs = [np.where(use_m, m, q) for m, q in zip(tm[0], tp[0])]
            cfs = [np.where(use_m, cm, cq) for cm, cq in zip(tm[1], tp[1])]
            tabs.append((ua, nbs, cfs))

        def rhs_T(p, mu):
            out = np.zeros(g.N)
            for a, (ua, nbs, cfs) in enumerate(tabs):
                dval = np.zeros(len(cells))
                for nb, cf in zip(nbs, cfs):
                    dval += cf * p[nb]
                    np.add.at(out, nb, -ua * cf * mu)  # L = -sum_a u~_a d_a(p)
                np.add.at(l_ut[a], cells, -mu * dval)
            return out

        lphi = _rk3_adjoint(lam, cells, F["adv"], 1.0, rhs_T)
        return lphi, l_ut

    def _extend_T(self, lam_ut, phi, F):
        """Adjoint of the n_ext Jacobi sweeps: (adjoint of the initial u~, adjoint of phi via S(phi) n)."""
        g, D = self.g, self.D
        cells = self.upd
        lphi = np.zeros(g.N)
        if len(cells) == 0 or self.n_ext == 0:
            return lam_ut.copy(), lphi
        lo = [g.clamp_shift(cells, _unit(D, a, -1)) for a in range(D)]
        hi = [g.clamp_shift(cells, _unit(D, a, 1)) for a in range(D)]
        gr = np.stack([0.5 * (phi[hi[a]] - phi[lo[a]]) for a in range(D)])
        mag = np.sqrt((gr * gr).sum(0))
        okg = mag > 0.0
        nh = np.where(okg, gr / np.where(okg, mag, 1.0), 0.0)
        s = phi[cells] / np.sqrt(phi[cells] ** 2 + 1.0)
        v = s[None, :] * nh
        dt = self.dtau_ext
        lv = np.zeros((D, len(cells)))
        lam = lam_ut.copy()
        for k in range(self.n_ext - 1, -1, -1):
            old = F["sweeps"][k]
            lc = lam[:, cells].copy()
            for a in range(D):
                pos = v[a] > 0.0
                diff = np.where(pos[None, :], old[:, cells] - old[:, lo[a]], old[:, hi[a]] - old[:, cells])
                lv[a] += (lc * (-dt * diff)).sum(0)
                # new[c] = old[c] - dt v (pos: old[c] - old[lo]; else old[hi] - old[c])
                lam[:, cells] += lc * np.where(pos, -dt * v[a], dt * v[a])[None, :]
                for b in range(D):
                    np.add.at(lam[b], lo[a], np.where(pos, dt * v[a], 0.0) * lc[b])
                    np.add.at(lam[b], hi[a], np.where(pos, 0.0, -dt * v[a]) * lc[b])
        # v = s(phi) n(phi), s = phi / sqrt(phi^2 + 1), n = g / |g|, g_a = (phi[hi] - phi[lo]) / 2
        ls = (lv * nh).sum(0)
        lnh = s[None, :] * lv
        lg = np.where(okg[None, :], (lnh - nh * (nh * lnh).sum(0)) / np.where(okg, mag, 1.0), 0.0)
        np.add.at(lphi, cells, ls / (phi[cells] ** 2 + 1.0) ** 1.5)
        for a in range(D):
            np.add.at(lphi, hi[a], 0.5 * lg[a])
            np.add.at(lphi, lo[a], -0.5 * lg[a])
        return lam, lphi

    def _ext_init_T(self, lam_ut0, f, phi, F):
        """Adjoint of u~ on interface cells = mean u_I over cut links: (adjoint of u~_n,
        adjoint of f_n via the moments, adjoint of phi via q)."""
        lat, g = self.lat, self.g
        x, y = self.lx, self.ly
        u, rho = F["u"], F["rho"]
        lut = lam_ut0.copy()
        lut[:, self.iface] = 0.0
        luI = lam_ut0[:, x] / self.cnt[x][None, :]
        px, py = phi[x], phi[y]
        q = px / (px - py)
        lu = np.zeros_like(u)
        for a in range(self.D):
            np.add.at(lu[a], x, (1.0 - q) * luI[a])
            np.add.at(lu[a], y, q * luI[a])
        lq = (luI * (u[:, y] - u[:, x])).sum(0)
        lphi = np.zeros(g.N)
        np.add.at(lphi, x, lq * (-py) / (px - py) ** 2)
        np.add.at(lphi, y, lq * px / (px - py) ** 2)
        cmu = lat.cf[:, :, None] - u[None, :, :]
        lf = np.einsum("an,jan->jn", lu, cmu) / rho[None, :]
        return lut, lf, lphi

    # ------------------------------------------------------------------ the transposed step
    def step_adjoint(self, state, p, lam, lam_gh=None):
        """Adjoints of (f_n, phi_n, u~_n) and dJ/dp from those of (f_{n+1}, phi_{n+1}, u~_{n+1});
        with ``lam_gh`` also accumulates the adjoint of the ghost-ring values."""
        f, phi, ut = state
        lf1, lphi1, lut1 = lam
        F = self._forward_ls(f, phi, ut)
        lps = self._reinit_T(lphi1, F) if self.reinit_on else lphi1
        lphi, lut_adv = self._advect_T(lps, F)
        lut_ext, lphi_ext = self._extend_T(lut1 + lut_adv, phi, F)
        lut, lf_init, lphi_init = self._ext_init_T(lut_ext, f, phi, F)
        st = self.frozen_step(phi)
        N = self.g.N
        geo = dict(phi=np.zeros(N), n=np.zeros((self.D, N)), kappa=np.zeros(N))
        lf, dp = st.step_adjoint(f, p, lf1, geo, lam_gh)
        lphi = lphi + lphi_ext + lphi_init + st.geometry_to_phi(geo)
        return (lf + lf_init, lphi, lut), dp

    def observables_adjoint(self, state, a):
        f, phi, ut = state
        st = FrozenStep(self.sim, phi, self.eps)
        return (st.observables_adjoint(f, a), st.observables_phi_adjoint(f, a), np.zeros((self.D, self.g.N)))


def trajectory(step, s0, p, nsteps):
    out = [s0]
    for _ in range(nsteps):
        out.append(step.step(out[-1], p))
    return out


def objective(step, s0, p, nsteps, a):
    return float(np.asarray(a) @ step.observables(trajectory(step, s0, p, nsteps)[-1]))


def gradients(step, s0, p, nsteps, a):
    """J = a . observables(f_N) and (dJ/dp, dJ/d(f_0, phi_0, u~_0))."""
    a = np.asarray(a, dtype=np.float64)
    tr = trajectory(step, s0, p, nsteps)
    J = float(a @ step.observables(tr[-1]))
    lam = step.observables_adjoint(tr[-1], a)
    dp = np.zeros(NPARAM)
    for n in range(nsteps - 1, -1, -1):
        lam, d = step.step_adjoint(tr[n], p, lam)
        dp += d
    return J, dp, lam
