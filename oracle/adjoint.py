"""Discrete adjoint of the oracle's single-level step with a frozen interface.

Test infrastructure (like the rest of ``oracle``): only the tests, the smoke
check and the benchmark's CPU baseline use it.

The paper has no adjoint; this module defines the one the library computes.
With the level set held fixed over a window of steps (no advection, no
reinitialisation, no refill; the phases, cut links, q, n and kappa are
constants), one step is a smooth map f_n -> f_{n+1}(f_n; p) of the
pre-collision populations (Sec. 2.1 and 2.3):

  moments and strain rate of f_n -> BGK collision with forcing ->
  push streaming with half-way bounce-back at walls and, on cut links,
  the interpolated bounce-back of Eq. bb with the momentum term of Eq. bb_cc
  and the stress jump of Eq. Sdecomp.

The parameters are p = (sigma, rho_0, rho_1, nu_0, nu_1): surface tension,
physical densities and kinematic viscosities of liquid (0) and gas (1).  The
objective is a weighted sum a . obs of the observables of Sec. 3.2 after the
last step, in the order the library reports them: liquid mass, gas mass, gas
volume, leaf count, gas centroid (D), gas velocity (D).

``FrozenStep.step_adjoint`` applies the transpose of the step's Jacobian to
an adjoint population field (the chain rule written out by hand, link by
link and cell by cell) and returns the parameter partials; ``gradients``
runs the reverse sweep over a stored trajectory.  The level set
itself is a further input: phi sets the link fractions q (radiation
theorem) and, through the least-squares quadratic fit (Sec. 2.2), the
interface cells' normal and curvature; ``gradients(..., want_phi=True)``
also returns dJ/dphi, valid while no perturbation changes a sign of phi.
Pins in tests/test_oracle_adjoint.py: every parameter derivative and
directional derivatives in phi against central finite differences of the
forward map in float64, and the dot-product identity
<J v, w> = <v, J^T w> of one step with J v from central differences, on
cases that exercise every bounce-back branch.
"""
import numpy as np

from .lattice import CS2
from .lbm import equilibrium, moments, omega_from_nu, strain_rate
from . import objective as indicator
from .levelset import fit_geometry

NPARAM = 5  # sigma, rho_0, rho_1, nu_0, nu_1


def params_of(sim):
    """The parameter vector p of a Sim."""
    return np.array([sim.sigma, sim.rho_phys[0], sim.rho_phys[1], sim.nu[0], sim.nu[1]], dtype=np.float64)


class FrozenStep:
    """The smooth step of the finest level of a Sim whose level set is held fixed.

    On a single-level grid this is the whole step.  On a multi-level grid it is
    one finest-level sub-step: leaves that stream from the ghost ring take the
    ring's post-collision values ``gh`` (an input here, built from the coarser
    level by oracle/adjoint_amr.py), and ``step_adjoint`` returns their adjoint.
    """

    def __init__(self, sim, phi=None, eps=None):
        """``phi`` replaces the Sim's level set (same signs: the masks are the Sim's).
        ``eps``: None for the sharp gas indicator in the observables, else the width of
        the smoothed indicator H_eps (oracle/objective.py)."""
        assert sim.collision == ("bgk", "bgk"), "the adjoint transposes the BGK collision"
        self.eps = eps
        self.sim = sim
        self.lat = lat = sim.lat
        self.g = g = sim.geoms[-1]
        self.D, self.Q = lat.D, lat.Q
        self.phase = sim.phase[-1].copy()
        self.leaf = sim.masks[-1][0].copy()
        self.ghostm = sim.masks[-1][3].copy()
        self.phi = (sim.phi if phi is None else np.asarray(phi, dtype=np.float64)).copy()
        assert np.array_equal(self.phi >= 0, sim.phi >= 0), "phi must keep the Sim's signs"
        self.gravity = sim.gravity.copy()
        self.body_force = sim.body_force.copy()
        self.wall_u = sim.wall_u.copy()
        # cut links (x, k): x - c_k lies in the other phase; i = opp(k) points from x to y = x + c_i
        x, k = sim.cut_links(self.phase, self.leaf)
        i = lat.opp[k]
        y, _ = g.shift(x, lat.c[i].T)
        self.x, self.k, self.i, self.y = x, k, i, y
        self.q = self.phi[x] / (self.phi[x] - self.phi[y])  # radiation theorem, Sec. 2.3
        self.A = self.phase[x]
        self.B = 1 - self.A
        back, _ = g.shift(x, -lat.c[i].T)
        ok = back >= 0
        ok[ok] = self.leaf[back[ok]] & (self.phase[back[ok]] == self.A[ok])
        self.back, self.ok = back, ok
        icells = np.unique(x)
        nvec = np.zeros((self.D, g.N))
        kap = np.zeros(g.N)
        nv, kv, _, _ = fit_geometry(g, self.phi, icells)
        nvec[:, icells] = nv
        kap[icells] = kv
        self.icells, self.nvec, self.kap = icells, nvec, kap
        q = self.q
        m = (1 - q) * nvec[:, x] + q * nvec[:, y]
        nm = np.sqrt((m * m).sum(0))
        n = np.where(nm > 0, m / np.where(nm > 0, nm, 1.0), 0.0)
        self.nhat, self.nm = n, nm
        sgn = np.where(self.A == 0, 1.0, -1.0)  # n points into the gas; n_A from A into B
        self.sgn = sgn
        self.nA = sgn * n
        self.kA = sgn * ((1 - q) * kap[x] + q * kap[y])
        self.ci = lat.cf[i].T
        cells = np.arange(g.N)
        # pull sources: (src, face, direction at the source), reflected at slip walls
        self.src = []
        for kk in range(lat.Q):
            src, face, flip = g.pull(cells, lat.c[kk])
            self.src.append((src, face, lat.mirror[kk, flip]))
        self.cut = np.zeros((lat.Q, g.N), dtype=bool)
        self.cut[k, x] = True
        # leaves whose source x - c_k is a ghost-ring cell (none on a single level)
        self.from_ghost = np.zeros((lat.Q, g.N), dtype=bool)
        # links reflected at a slip wall whose source lies in the other phase: plain bounce-back
        self.rcut = np.zeros((lat.Q, g.N), dtype=bool)
        for kk in range(lat.Q):
            src, _, ks = self.src[kk]
            ok = (src >= 0) & self.leaf
            ok[ok] = self.ghostm[src[ok]]
            self.from_ghost[kk] = ok
            r = (src >= 0) & self.leaf & (ks != kk) & ~ok
            r[r] = self.phase[src[r]] != self.phase[r]
            self.rcut[kk] = r
        self.gas = self.leaf & (self.phase == 1)
        self.centers = g.centers(1.0)

    # ---------------------------------------------------------------- parameters
    def cell_params(self, p):
        """omega and acceleration per cell for the parameter vector p."""
        ph = self.phase
        rp, nu = p[1:3], p[3:5]
        om = omega_from_nu(nu[ph])
        acc = self.gravity[:, None] + self.body_force[:, None] / rp[ph][None, :]
        return om, acc

    # ---------------------------------------------------------------- forward
    def _link_pieces(self, rho, u, S, p):
        q, A, B, x, y = self.q, self.A, self.B, self.x, self.y
        rp, nu = p[1:3], p[3:5]
        etaA, etaB = rp[A] * nu[A], rp[B] * nu[B]
        eb = 0.5 * (etaA + etaB)
        je = etaB - etaA
        jp = CS2 * (rp[B] * (rho[y] - 1.0) - rp[A] * (rho[x] - 1.0))
        Sbar = 0.5 * (S[:, :, x] + S[:, :, y])
        nA, ci = self.nA, self.ci
        v = np.einsum("abn,bn->an", Sbar, nA)
        Snn = (nA * v).sum(0)
        cn = (ci * nA).sum(0)
        cvt = (ci * v).sum(0) - Snn * cn
        r = je / eb
        alpha = (jp + p[0] * self.kA) / (2.0 * eb) - r * Snn
        ccS = alpha * cn * cn - 2.0 * r * cn * cvt  # c_i c_i : [S]
        uI = (1 - q) * u[:, x] + q * u[:, y]
        wi = self.lat.w[self.i]
        df = -(2.0 * wi / CS2) * ((ci * uI).sum(0) - q * (1 - q) * ccS)  # Eq. bb_cc
        return dict(eb=eb, je=je, jp=jp, Snn=Snn, cn=cn, cvt=cvt, r=r, alpha=alpha, df=df, ccS=ccS, v=v,
                    Sbar=Sbar)

    def step(self, f, p, gh=None):
        """f_{n+1} from the pre-collision populations f_n (and the ghost ring's values gh)."""
        lat = self.lat
        om, acc = self.cell_params(p)
        rho, u = moments(lat, f)
        S = strain_rate(lat, f, om)
        fc = f + om[None, :] * (equilibrium(lat, rho, u) - f) \
            + lat.w[:, None] * rho[None, :] * (lat.cf @ acc) / CS2
        fn = f.copy()
        for k in range(lat.Q):
            i = lat.opp[k]
            src, face, ks = self.src[k]
            wall = (src < 0) & self.leaf
            fg, rc = self.from_ghost[k], self.rcut[k]
            same = (src >= 0) & ~self.cut[k] & self.leaf & ~fg & ~rc
            fn[k, same] = fc[ks[same], src[same]]
            if fg.any():
                fn[k, fg] = gh[ks[fg], src[fg]]
            if rc.any():
                fn[k, rc] = fc[i, rc]
            if wall.any():
                fn[k, wall] = fc[i, wall] - (2 * lat.w[i] / CS2) * (self.wall_u[face[wall]] @ lat.cf[i])
        P = self._link_pieces(rho, u, S, p)
        x, k, i, q = self.x, self.k, self.i, self.q
        fi, fk = fc[i, x], fc[k, x]
        fb = np.where(self.ok, fc[i, np.where(self.ok, self.back, 0)], 0.0)
        df = P["df"]
        fn[k, x] = np.where(q >= 0.5, fi / (2 * q) + (2 * q - 1) / (2 * q) * fk + df / (2 * q),
                            np.where(self.ok, 2 * q * fi + (1 - 2 * q) * fb + df, fi + df))  # Eq. bb
        return fn

    def observables(self, f):
        """liquid mass, gas mass, gas volume, leaf count, centroid (D), gas velocity (D)."""
        if self.eps is not None:
            return indicator.observables(self.lat, indicator.levels_of(self.sim), [f], self.phi, self.eps)
        rho, u = moments(self.lat, f)
        leaf, gas = self.leaf, self.gas
        vol = float(gas.sum())
        return np.concatenate([[rho[leaf & (self.phase == 0)].sum(), rho[gas].sum(), vol, float(leaf.sum())],
                               self.centers[:, gas].sum(1) / vol, u[:, gas].sum(1) / vol])

    # ---------------------------------------------------------------- adjoint
    def observables_phi_adjoint(self, f, a):
        """dJ/dphi of J = a . observables(f) at fixed f: zero with the sharp indicator, the
        H_eps' terms with the smoothed one."""
        if self.eps is None:
            return np.zeros(self.g.N)
        return indicator.observables_adjoint(self.lat, indicator.levels_of(self.sim), [f], self.phi, self.eps, a)[1]

    def observables_adjoint(self, f, a):
        """dJ/df for J = a . observables(f)."""
        if self.eps is not None:
            return indicator.observables_adjoint(self.lat, indicator.levels_of(self.sim), [f], self.phi,
                                                 self.eps, a)[0][0]
        lat = self.lat
        rho, u = moments(lat, f)
        D = self.D
        lam = np.zeros_like(f)
        lam[:, self.leaf & (self.phase == 0)] += a[0]
        lam[:, self.gas] += a[1]
        vol = float(self.gas.sum())
        au = np.asarray(a[4 + D:4 + 2 * D], dtype=np.float64)
        g = self.gas
        # d u_a / d f_j = (c_ja - u_a) / rho
        lam[:, g] += ((lat.cf @ au)[:, None] - (au @ u[:, g])[None, :]) / rho[g][None, :] / vol
        return lam

    def step_adjoint(self, f, p, lam_next, geo=None, lam_gh=None):
        """(lam_n, dJ/dp): the transpose of the step's Jacobian applied to lam_next.

        With ``geo`` (dict of arrays phi (N,), n (D, N), kappa (N,)), also
        accumulates the adjoints of the frozen geometry: of phi through the link
        fractions q, and of the interface cells' normal and curvature.  With
        ``lam_gh`` ((Q, N)), accumulates the adjoint of the ghost-ring values."""
        lat, g = self.lat, self.g
        D, Q, N = self.D, self.Q, g.N
        om, acc = self.cell_params(p)
        rho, u = moments(lat, f)
        feq = equilibrium(lat, rho, u)
        S = strain_rate(lat, f, om)
        dp = np.zeros(NPARAM)
        # ---- streaming: transpose of the push and of the wall bounce-back
        lc = np.zeros_like(f)
        for k in range(Q):
            i = lat.opp[k]
            src, _, ks = self.src[k]
            fg, rc = self.from_ghost[k], self.rcut[k]
            same = (src >= 0) & ~self.cut[k] & self.leaf & ~fg & ~rc
            np.add.at(lc, (ks[same], src[same]), lam_next[k, same])
            if fg.any():
                np.add.at(lam_gh, (ks[fg], src[fg]), lam_next[k, fg])
            lc[i, rc] += lam_next[k, rc]
            wall = (src < 0) & self.leaf
            lc[i, wall] += lam_next[k, wall]
        # ---- cut links: transpose of Eq. bb
        x, k, i, q, y, A, B = self.x, self.k, self.i, self.q, self.y, self.A, self.B
        lam = lam_next[k, x]
        hi = q >= 0.5
        ok = self.ok & ~hi
        np.add.at(lc, (i, x), np.where(hi, 1 / (2 * q), np.where(ok, 2 * q, 1.0)) * lam)
        np.add.at(lc, (k, x), np.where(hi, (2 * q - 1) / (2 * q), 0.0) * lam)
        np.add.at(lc, (i[ok], self.back[ok]), (1 - 2 * q[ok]) * lam[ok])
        l_df = np.where(hi, 1 / (2 * q), 1.0) * lam
        # ---- Eq. bb_cc: df = -(2 w_i / cs2) (c_i . u_I - q (1 - q) c_i c_i : [S])
        P = self._link_pieces(rho, u, S, p)
        wi = lat.w[i]
        ci, nA = self.ci, self.nA
        l_uI = -(2 * wi / CS2) * l_df * ci
        l_ccS = (2 * wi / CS2) * q * (1 - q) * l_df
        lam_u = np.zeros((D, N))
        for a in range(D):
            np.add.at(lam_u[a], x, (1 - q) * l_uI[a])
            np.add.at(lam_u[a], y, q * l_uI[a])
        cn, cvt, Snn, r, eb, je = P["cn"], P["cvt"], P["Snn"], P["r"], P["eb"], P["je"]
        l_alpha = l_ccS * cn * cn
        l_cvt = -2 * r * cn * l_ccS
        l_r = -2 * cn * cvt * l_ccS - Snn * l_alpha
        l_jp = l_alpha / (2 * eb)
        l_eb = -l_alpha * (P["jp"] + p[0] * self.kA) / (2 * eb * eb) - l_r * je / (eb * eb)
        l_je = l_r / eb
        l_etaA = 0.5 * l_eb - l_je
        l_etaB = 0.5 * l_eb + l_je
        dp[0] += (l_alpha * self.kA / (2 * eb)).sum()
        rp, nu = p[1:3], p[3:5]
        for ph in (0, 1):
            mA, mB = A == ph, B == ph
            l_eta = l_etaA[mA].sum() + l_etaB[mB].sum()
            dp[1 + ph] += l_eta * nu[ph]
            dp[3 + ph] += l_eta * rp[ph]
            dp[1 + ph] += CS2 * ((l_jp * (rho[y] - 1.0))[mB].sum() - (l_jp * (rho[x] - 1.0))[mA].sum())
        lam_rho = np.zeros(N)
        np.add.at(lam_rho, y, CS2 * rp[B] * l_jp)
        np.add.at(lam_rho, x, -CS2 * rp[A] * l_jp)
        if geo is not None:
            self._geometry_adjoint(f, p, om, rho, u, lam, hi, ok, l_df, l_ccS, P, geo)
        # Snn = n.Sbar.n and c.v_t = c.Sbar.n - Snn (c.n)
        l_Snn = -r * l_alpha - cn * l_cvt
        l_Sbar = np.einsum("an,bn->abn", ci, nA) * l_cvt + np.einsum("an,bn->abn", nA, nA) * l_Snn
        lam_S = np.zeros((D, D, N))
        for a in range(D):
            for b in range(D):
                np.add.at(lam_S[a, b], x, 0.5 * l_Sbar[a, b])
                np.add.at(lam_S[a, b], y, 0.5 * l_Sbar[a, b])
        # ---- collision: fc = f + omega (feq(rho, u) - f) + w rho (c . acc) / cs2
        cu = lat.cf @ u
        lam_n = (1 - om)[None, :] * lc
        lam_n += ((om[None, :] * feq / rho[None, :] + lat.w[:, None] * (lat.cf @ acc) / CS2) * lc).sum(0)[None, :]
        Bv = np.zeros((D, N))
        for a in range(D):
            dfeq = lat.w[:, None] * rho[None, :] * (lat.cf[:, a][:, None] / CS2 + cu * lat.cf[:, a][:, None] / CS2 ** 2
                                                    - u[a][None, :] / CS2)
            Bv[a] = om * (dfeq * lc).sum(0)
        # moments: d rho / d f_j = 1, d u_a / d f_j = (c_ja - u_a) / rho
        cmu = lat.cf[:, :, None] - u[None, :, :]
        lam_n += np.einsum("an,jan->jn", Bv + lam_u, cmu) / rho[None, :]
        lam_n += lam_rho[None, :]
        # strain rate S_ab = kk Pi_ab, kk = -omega / (2 rho cs2), Pi_ab = sum_q c_qa c_qb (f_q - feq_q)
        kk = -om / (2 * rho * CS2)
        Pi = np.einsum("qa,qb,qn->abn", lat.cf, lat.cf, f - feq)
        eye = np.eye(D)
        for a in range(D):
            for b in range(D):
                dPi = ((lat.cf[:, a] * lat.cf[:, b])[:, None] - (CS2 * eye[a, b] - u[a] * u[b])[None, :]
                       - lat.cf[:, a][:, None] * u[b][None, :] - u[a][None, :] * lat.cf[:, b][:, None])
                lam_n += (lam_S[a, b] * kk)[None, :] * (dPi - Pi[a, b][None, :] / rho[None, :])
        # parameter partials of the collision: omega(nu), acc(rho), and S through omega
        l_om = (lc * (feq - f)).sum(0) + (lam_S * S).sum((0, 1)) / om
        l_acc = np.einsum("qn,qa->an", lc * lat.w[:, None] * rho[None, :], lat.cf) / CS2
        for ph in (0, 1):
            m = self.leaf & (self.phase == ph)
            om_p = omega_from_nu(nu[ph])
            dp[3 + ph] += l_om[m].sum() * (-om_p * om_p / CS2)  # d omega / d nu
            dp[1 + ph] += (l_acc[:, m].sum(1) * (-self.body_force / rp[ph] ** 2)).sum()
        lam_n[:, ~self.leaf] = lam_next[:, ~self.leaf]
        return lam_n, dp


    def _geometry_adjoint(self, f, p, om, rho, u, lam, hi, ok, l_df, l_ccS, P, geo):
        """Per link: the adjoints of q (explicit in Eq. bb and through u_I, q(1-q), the
        interpolated n and kappa) and of the link's n_A, kappa_A; n_A, kappa_A go on
        to the interface cells' n and kappa, q to phi(x) and phi(y)."""
        lat = self.lat
        x, k, i, y, q = self.x, self.k, self.i, self.y, self.q
        _, acc = self.cell_params(p)
        from .lbm import equilibrium as feq_of
        fc = f + om[None, :] * (feq_of(lat, rho, u) - f) + lat.w[:, None] * rho[None, :] * (lat.cf @ acc) / CS2
        fi, fk = fc[i, x], fc[k, x]
        fb = np.where(self.ok, fc[i, np.where(self.ok, self.back, 0)], 0.0)
        df = P["df"]
        w6 = 2 * lat.w[i] / CS2
        ci = self.ci
        # explicit q in the Bouzidi branches (df held fixed)
        l_q = lam * np.where(hi, (-fi + fk - df) / (2 * q * q), np.where(ok, 2 * fi - 2 * fb, 0.0))
        # df = -w6 (c.u_I - q (1 - q) ccS): u_I and the factor q (1 - q)
        l_q += l_df * (-w6) * (ci * (u[:, y] - u[:, x])).sum(0)
        l_q += l_df * w6 * (1 - 2 * q) * P["ccS"]
        # ccS(n_A, kappa_A) = alpha cn^2 - 2 r cn cvt, alpha = (jp + sigma kappa_A) / (2 eb) - r Snn
        cn, cvt, r, alpha, v, Snn, Sbar = P["cn"], P["cvt"], P["r"], P["alpha"], P["v"], P["Snn"], P["Sbar"]
        Sc = np.einsum("abn,bn->an", Sbar, ci)
        d_cvt = Sc - 2 * cn * v - Snn * ci  # d cvt / d n_A
        l_nA = l_ccS * (cn * cn * (-2 * r * v) + (2 * alpha * cn - 2 * r * cvt) * ci - 2 * r * cn * d_cvt)
        l_kA = l_ccS * cn * cn * p[0] / (2 * P["eb"])
        # n_A = sgn m / |m|, m = (1 - q) n_x + q n_y;  kappa_A = sgn ((1 - q) kappa_x + q kappa_y)
        nh, nm, sgn = self.nhat, self.nm, self.sgn
        safe = np.where(nm > 0, nm, 1.0)
        l_nh = sgn * l_nA
        l_m = np.where(nm > 0, (l_nh - nh * (nh * l_nh).sum(0)) / safe, 0.0)
        nx, ny = self.nvec[:, x], self.nvec[:, y]
        l_q += (l_m * (ny - nx)).sum(0)
        kx, ky = self.kap[x], self.kap[y]
        l_q += sgn * (ky - kx) * l_kA
        for a in range(self.D):
            np.add.at(geo["n"][a], x, (1 - q) * l_m[a])
            np.add.at(geo["n"][a], y, q * l_m[a])
        np.add.at(geo["kappa"], x, sgn * (1 - q) * l_kA)
        np.add.at(geo["kappa"], y, sgn * q * l_kA)
        # q = phi_x / (phi_x - phi_y)
        px, py = self.phi[x], self.phi[y]
        den = (px - py) ** 2
        np.add.at(geo["phi"], x, l_q * (-py) / den)
        np.add.at(geo["phi"], y, l_q * px / den)

    def geometry_to_phi(self, geo):
        """dJ/dphi: geo["phi"] plus the transpose of the least-squares fit (Sec. 2.2)
        applied to the interface cells' normal and curvature adjoints."""
        from .levelset import _quad_design
        g = self.g
        D = self.D
        offs, A, pairs = _quad_design(D)
        Pinv = np.linalg.pinv(A)  # coef = Pinv vals
        cells = self.icells
        vals = np.stack([self.phi[g.clamp_shift(cells, o)] for o in offs])
        coef = Pinv @ vals
        gr = coef[1:1 + D]
        H = np.zeros((D, D, len(cells)))
        for a in range(D):
            H[a, a] = 2.0 * coef[1 + D + a]
        for kk, (a, b) in enumerate(pairs):
            H[a, b] = H[b, a] = coef[1 + 2 * D + kk]
        g2 = (gr * gr).sum(0)
        mag = np.sqrt(g2)
        okc = mag > 1e-12
        safe = np.where(okc, mag, 1.0)
        n = gr / safe
        trH = np.trace(H)
        Hg = np.einsum("abn,bn->an", H, gr)
        kap = (g2 * trH - (gr * Hg).sum(0)) / safe ** 3
        ln = geo["n"][:, cells]
        lk = geo["kappa"][cells]
        # n = g / |g|;  kappa = (|g|^2 tr H - g.H.g) / |g|^3
        l_g = (ln - n * (n * ln).sum(0)) / safe
        l_g += lk * ((2 * gr * trH - 2 * Hg) / safe ** 3 - 3 * kap * gr / safe ** 2)
        l_H = lk * (g2[None, None, :] * np.eye(D)[:, :, None] - gr[:, None, :] * gr[None, :, :]) / safe ** 3
        l_coef = np.zeros_like(coef)
        l_coef[1:1 + D] = l_g
        for a in range(D):
            l_coef[1 + D + a] = 2.0 * l_H[a, a]
        for kk, (a, b) in enumerate(pairs):
            l_coef[1 + 2 * D + kk] = l_H[a, b] + l_H[b, a]
        l_coef[:, ~okc] = 0.0
        l_vals = Pinv.T @ l_coef
        out = geo["phi"].copy()
        for j, o in enumerate(offs):
            np.add.at(out, g.clamp_shift(cells, o), l_vals[j])
        return out


def trajectory(step, f0, p, nsteps):
    fs = [f0]
    for _ in range(nsteps):
        fs.append(step.step(fs[-1], p))
    return fs


def objective(step, f0, p, nsteps, a):
    return float(np.asarray(a) @ step.observables(trajectory(step, f0, p, nsteps)[-1]))


def gradients(step, f0, p, nsteps, a, want_phi=False):
    """J = a . observables(f_N) and its adjoint gradients: (J, dJ/dp, dJ/df_0),
    plus dJ/dphi (the frozen level set) with ``want_phi``."""
    a = np.asarray(a, dtype=np.float64)
    fs = trajectory(step, f0, p, nsteps)
    J = float(a @ step.observables(fs[-1]))
    lam = step.observables_adjoint(fs[-1], a)
    dp = np.zeros(NPARAM)
    N = step.g.N
    geo = dict(phi=np.zeros(N), n=np.zeros((step.D, N)), kappa=np.zeros(N)) if want_phi else None
    for n in range(nsteps - 1, -1, -1):
        lam, d = step.step_adjoint(fs[n], p, lam, geo)
        dp += d
    if want_phi:
        return J, dp, lam, step.geometry_to_phi(geo) + step.observables_phi_adjoint(fs[-1], a)
    return J, dp, lam
