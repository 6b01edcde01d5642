"""Interface coupling (Sec. 2.3) and refill of newly activated cells (Sec. 2.4).

Conventions used throughout.  A link is named by the cell x and the INCOMING
direction k whose source x - c_k lies in the other phase; i = opp(k) is the
direction from x towards the interface, so x + c_i is the other-phase node of
Eq. bb.  Phase A is x's phase, B the other one; [X] = X_B - X_A; n_A is the
unit normal pointing from A into B and kappa_A = div n_A.

Readings (where the passages are garbled or silent):

* Eq. bb, q >= 1/2 branch: the second population is the opposite one at the
  same node, f_k^c(x) (linear Bouzidi); the printed x - c_i would not be a
  linear interpolation.  When the q < 1/2 branch needs x - c_i but that node is
  not a fluid node of phase A, the link falls back to half-way bounce-back
  f_k = f_i^c(x) + df (the q = 1/2 case of both branches).
* Momentum term (Eq. bb_cc and the moving-wall term below Eq. bb): the paper
  writes the term for the direction the populations arrive from; for i
  pointing towards the boundary the sign that reproduces the Couette profile is
  df = -(2 w_i / c_s^2) (c_i . u_B), with no density factor (the paper has none).
* Eq. bb_cc's stress term: Lambda_i = c_i (x) c_i.  Linear interpolation of the
  velocity along the link misses the interface value by q(1-q) c_i.[grad u].c_i
  when the gradient jumps; subtracting that is exactly the printed term with
  this Lambda, so df = -(2 w_i/c_s^2)(c_i.u_I - q(1-q) c_i c_i : [S]).
* Eq. Sdecomp: [S]:nn = ([p] + sigma kappa_A)/(2 eta_bar) - ([eta]/eta_bar) Sbar:nn,
  [S]:n t = -([eta]/eta_bar) Sbar:n t, tangential-tangential part zero.  The
  printed factor 2 on sigma kappa is dropped because kappa = div n is the sum of
  the principal curvatures; the static drop then carries p_in - p_out =
  sigma kappa (sigma / R in 2D).  Sbar = (S_A(x) + S_B(x + c_i))/2.
* Two LB solvers each at rest density 1: physical density rho_k enters through
  eta_k = rho_k nu_k and p_k = rho_k c_s^2 (rho_hat - 1) (gauge pressure).
* u_I = (1-q) u_A(x) + q u_B(x + c_i); n and kappa linearly interpolated along
  the link from the two nodes' least-squares values, n renormalised.
* Refill (Sec. 2.4): e_min = the non-rest direction, among those whose
  neighbour is a valid node of the new phase, that maximises (e_i.m)/|e_i|
  with m the unit normal pointing into the new phase (ties: lowest index);
  q = phi(x_r)/(phi(x_r) - phi(x_r - e_min)) when x_r - e_min lies in the other
  phase, else 1/2.  Extrapolation weights are the Lagrange weights of the nodes
  -q (interface), 1 and 2 evaluated at 0: 2/((q+1)(q+2)), 2q/(q+1), -q/(q+2)
  (the printed third weight 2q/(q+2) does not sum to one); with no valid second
  node, the linear pair 1/(1+q), q/(1+q).  u_Gamma is x_r's own old-phase
  velocity; rho_Gamma carries the old phase's pressure plus the Laplace jump,
  p_new = p_old + sigma kappa_new.  f^neq is copied from x_r + e_min.

Pins: tests/test_oracle_coupling.py (weights exact on quadratics and summing to
one, q exact for linear phi, e_min brute force); tests/test_oracle_refill.py
(the composed refill: new-phase density and velocity polynomials along e_min
that meet the interface conditions at Gamma are reproduced exactly for any q
on both branches, a static drop's flipped cells land on their new phase's
pressure either way, a planted moment-free f^neq at x_r + e_min is copied
exactly, no usable neighbour gives the rest state, and planted mistakes fail);
the two-layer Poiseuille / Couette closed forms and the static-drop Laplace
jump in tests/test_oracle_flows.py.
"""
import numpy as np

from .lattice import CS2
from .lbm import equilibrium, moments


def link_fraction(phi_x, phi_y):
    """Radiation theorem (Sec. 2.3): q = phi(x) / (phi(x) - phi(x + e_i))."""
    return phi_x / (phi_x - phi_y)


def stress_jump_cc(c_i, nA, kA, Sbar, jp, jeta, eta_bar, sigma):
    """c_i c_i : [S] with [S] built from Eq. Sdecomp (reading in the header)."""
    Snn = np.einsum("an,abn,bn->n", nA, Sbar, nA)
    v = np.einsum("abn,bn->an", Sbar, nA)
    vt = v - (nA * v).sum(0)[None, :] * nA
    alpha = (jp + sigma * kA) / (2.0 * eta_bar) - (jeta / eta_bar) * Snn
    cn = (c_i * nA).sum(0)
    cvt = (c_i * vt).sum(0)
    return alpha * cn * cn - 2.0 * (jeta / eta_bar) * cn * cvt


def interface_values(lat, geom, x, k, fc, phase, fluid, phi, rho, u, S, nvec, kappa, prm):
    """Missing populations f_k(x, t+1) on cut links (Eq. bb with Eq. bb_cc).

    x, k: arrays of link cells and incoming directions.  fc: post-collision
    populations at t; rho, u, S: that step's pre-collision moments and strain
    rate; fluid: cells that carry populations of their phase at this level.
    """
    if len(x) == 0:
        return np.zeros(0)
    i = lat.opp[k]
    ci = lat.cf[i].T  # (D, M)
    y, _ = geom.shift(x, lat.c[i].T)
    q = link_fraction(phi[x], phi[y])
    A = phase[x]
    B = 1 - A
    uI = (1.0 - q) * u[:, x] + q * u[:, y]
    n = (1.0 - q) * nvec[:, x] + q * nvec[:, y]
    nm = np.sqrt((n * n).sum(0))
    n = np.where(nm > 0.0, n / np.where(nm > 0.0, nm, 1.0), 0.0)
    kap = (1.0 - q) * kappa[x] + q * kappa[y]
    sgn = np.where(A == 0, 1.0, -1.0)  # n points to gas; n_A points from A into B
    nA = sgn * n
    kA = sgn * kap
    rp = np.asarray(prm["rho_phys"], dtype=np.float64)
    nu = np.asarray(prm["nu"], dtype=np.float64)
    etaA = rp[A] * nu[A]
    etaB = rp[B] * nu[B]
    eta_bar = 0.5 * (etaA + etaB)
    jeta = etaB - etaA
    jp = rp[B] * CS2 * (rho[y] - 1.0) - rp[A] * CS2 * (rho[x] - 1.0)
    Sbar = 0.5 * (S[:, :, x] + S[:, :, y])
    ccS = stress_jump_cc(ci, nA, kA, Sbar, jp, jeta, eta_bar, prm["sigma"])
    df = -(2.0 * lat.w[i] / CS2) * ((ci * uI).sum(0) - q * (1.0 - q) * ccS)
    back, _ = geom.shift(x, -lat.c[i].T)
    back_ok = back >= 0
    back_ok[back_ok] = fluid[back[back_ok]] & (phase[back[back_ok]] == A[back_ok])
    fi = fc[i, x]
    fk = fc[k, x]
    fb = np.where(back_ok, fc[i, np.where(back_ok, back, 0)], 0.0)
    low = 2.0 * q * fi + (1.0 - 2.0 * q) * fb + df
    high = fi / (2.0 * q) + (2.0 * q - 1.0) / (2.0 * q) * fk + df / (2.0 * q)
    half = fi + df
    return np.where(q >= 0.5, high, np.where(back_ok, low, half))


def interface_velocity_per_cell(lat, geom, cells_links_x, k, phase, phi, u, ncell):
    """Mean over each interface cell's cut links of u_I (extension data)."""
    D = geom.D
    if len(cells_links_x) == 0:
        return np.zeros((D, ncell)), np.zeros(ncell)
    i = lat.opp[k]
    y, _ = geom.shift(cells_links_x, lat.c[i].T)
    q = link_fraction(phi[cells_links_x], phi[y])
    uI = (1.0 - q) * u[:, cells_links_x] + q * u[:, y]
    acc = np.zeros((D, ncell))
    cnt = np.zeros(ncell)
    for a in range(D):
        np.add.at(acc[a], cells_links_x, uI[a])
    np.add.at(cnt, cells_links_x, 1.0)
    return acc, cnt


def extrapolation_weights(q, quadratic):
    """Lagrange weights of nodes (-q, 1, 2) [or (-q, 1)] evaluated at 0 (Sec. 2.4)."""
    if quadratic:
        return 2.0 / ((q + 1.0) * (q + 2.0)), 2.0 * q / (q + 1.0), -q / (q + 2.0)
    return 1.0 / (1.0 + q), q / (1.0 + q), 0.0


def choose_emin(lat, geom, xr, m, ok_new):
    """e_min for one refilled cell: argmax over usable directions of e.m/|e|."""
    best = -1
    best_val = -np.inf
    for i in range(lat.Q):
        if i == lat.rest:
            continue
        nb, _ = geom.shift(np.array([xr]), lat.c[i])
        if nb[0] < 0 or not ok_new[nb[0]]:
            continue
        val = float(lat.cf[i] @ m) / lat.norm[i]
        if val > best_val:
            best_val = val
            best = i
    return best


def refill(lat, geom, f_new, cells, phase_old, phase_new, fluid, phi_new, nvec, kappa, prm):
    """Initialise cells that changed phase (Sec. 2.4).

    f_new holds the streamed populations at t+1 (old phase for the flipped
    cells).  Modified in place; returns the number of cells that found no
    usable neighbour (set to rest equilibrium).
    """
    rp = np.asarray(prm["rho_phys"], dtype=np.float64)
    n_fail = 0
    rho_all = f_new.sum(0)
    for xr in cells:
        Pn = int(phase_new[xr])
        Po = int(phase_old[xr])
        ok_new = fluid & (phase_new == Pn) & (phase_old == Pn)
        sg = 1.0 if Pn == 0 else -1.0  # kappa of the new phase: kappa_new = sg*kappa
        m = -nvec[:, xr] if Pn == 0 else nvec[:, xr]
        e = choose_emin(lat, geom, xr, m, ok_new)
        if e < 0:
            f_new[:, xr] = lat.w
            n_fail += 1
            continue
        ce = lat.c[e]
        b, _ = geom.shift(np.array([xr]), -ce)
        if b[0] >= 0 and phase_new[b[0]] != Pn:
            q = phi_new[xr] / (phi_new[xr] - phi_new[b[0]])
        else:
            q = 0.5
        a1, _ = geom.shift(np.array([xr]), ce)
        a2, _ = geom.shift(np.array([xr]), 2 * ce)
        quad = bool(a2[0] >= 0 and ok_new[a2[0]])
        w0, w1, w2 = extrapolation_weights(q, quad)
        r_old, u_old = moments(lat, f_new[:, [xr]])
        p_gamma = rp[Po] * CS2 * (r_old[0] - 1.0) + prm["sigma"] * sg * kappa[xr]
        rho_g = 1.0 + p_gamma / (rp[Pn] * CS2)
        u_g = u_old[:, 0]
        r1, u1 = moments(lat, f_new[:, [a1[0]]])
        rho_r = w0 * rho_g + w1 * r1[0]
        u_r = w0 * u_g + w1 * u1[:, 0]
        if quad:
            r2, u2 = moments(lat, f_new[:, [a2[0]]])
            rho_r += w2 * r2[0]
            u_r += w2 * u2[:, 0]
        fneq = f_new[:, a1[0]] - equilibrium(lat, r1, u1)[:, 0]
        f_new[:, xr] = equilibrium(lat, np.array([rho_r]), u_r[:, None])[:, 0] + fneq
    del rho_all
    return n_fail
