"""Cumulant collision on D3Q27, the paper's gas-phase operator in 3D (Sec. 3.2, which
names the cumulant model of Geier et al. 2015 without printing it).

Test infrastructure (like the rest of ``oracle``): only the tests, the smoke
check and the benchmark's CPU baseline use it.

Definition, per cell, written from the cumulant idea itself (no listing):
* central moments per unit mass of the 27 velocities,
    k_m = (1/rho) sum_i prod_a (c_ia - u_a)^(m_a) f_i,   m in {0, 1, 2}^3;
* cumulants c_m of the distribution f / rho from them by the moment-cumulant
  recursion obtained by differentiating log of the moment generating function
  once along the first axis a with m_a > 0:
    k_m = sum over j <= m - e_a of binom(m - e_a, j) c_(j + e_a) k_(m - e_a - j)
  (multi-index binomials are products over the axes); with central moments the
  first cumulants vanish and c = k at orders 2 and 3;
* relaxation: the off-diagonal second cumulants and the differences of the
  diagonal ones with the shear rate w1 (nu = c_s^2 (1/w1 - 1/2)), the trace of
  the second cumulants towards its equilibrium 3 c_s^2 with the bulk rate w2,
  every cumulant of order n >= 3 towards zero with the rate w[n];
* back: moments from the relaxed cumulants by the same recursion, then the 27
  populations from the 27 central moments times rho (a 27 x 27 linear system
  per cell).
Readings: the paper gives no rates; w2 and all higher rates default to 1 (their
usual choice); forcing is added after the collision exactly as for BGK.

Pins: tests/test_oracle_cumulant.py (recursion against the textbook
fourth-order relations and a round trip, conservation of mass and momentum,
the equilibrium as a fixed point, the shear-wave decay rate against
nu = c_s^2 (1/w1 - 1/2)).
"""
from itertools import product

import numpy as np

from .lattice import CS2

MIDX = [m for m in product(range(3), repeat=3)]  # multi-indices (m_x, m_y, m_z), each 0..2
POS = {m: n for n, m in enumerate(MIDX)}
ORDER = np.array([sum(m) for m in MIDX])


def _binom(n, k):
    out = 1
    for a, b in zip(n, k):
        out *= {(0, 0): 1, (1, 0): 1, (1, 1): 1, (2, 0): 1, (2, 1): 2, (2, 2): 1}[(a, b)]
    return out


def _below(m):
    return [j for j in MIDX if all(x <= y for x, y in zip(j, m))]


def _recursion_terms(m):
    """(coefficient, cumulant index, moment index) of k_m = sum coef c_. k_. (first axis a)."""
    a = next(i for i in range(3) if m[i] > 0)
    mm = tuple(m[i] - (i == a) for i in range(3))
    out = []
    for j in _below(mm):
        cj = tuple(j[i] + (i == a) for i in range(3))
        rest = tuple(mm[i] - j[i] for i in range(3))
        out.append((_binom(mm, j), cj, rest))
    return out


def cumulants_from_moments(k):
    """k: (27, N) moments per unit mass (k_000 = 1) -> cumulants (27, N) (c_000 = 0)."""
    c = np.zeros_like(k)
    for m in sorted(MIDX, key=sum):
        if sum(m) == 0:
            continue
        acc = k[POS[m]].copy()
        for coef, cj, rest in _recursion_terms(m):
            if cj == m:  # the term with j = m - e_a: c_m k_0, k_0 = 1
                continue
            acc -= coef * c[POS[cj]] * k[POS[rest]]
        c[POS[m]] = acc
    return c


def moments_from_cumulants(c):
    """Inverse of cumulants_from_moments (k_000 = 1)."""
    k = np.zeros_like(c)
    k[POS[(0, 0, 0)]] = 1.0
    for m in sorted(MIDX, key=sum):
        if sum(m) == 0:
            continue
        acc = np.zeros(c.shape[1:])
        for coef, cj, rest in _recursion_terms(m):
            acc = acc + coef * c[POS[cj]] * k[POS[rest]]
        k[POS[m]] = acc
    return k


def _transform(lat, u):
    """T[n, m, i] = prod_a (c_ia - u_a)^(m_a) for every cell n."""
    d = lat.cf[None, :, :] - u.T[:, None, :]  # (N, Q, 3)
    T = np.ones((u.shape[1], 27, lat.Q))
    for r, m in enumerate(MIDX):
        for a in range(3):
            if m[a]:
                T[:, r, :] *= d[:, :, a] ** m[a]
    return T


def cumulant_collide(lat, f, w1, w2=1.0, w_high=(1.0, 1.0, 1.0, 1.0)):
    """Post-collision populations (no forcing); w1 per cell, w_high the rates of orders 3..6."""
    assert lat.Q == 27, "the cumulant operator is defined on D3Q27"
    rho = f.sum(0)
    u = (lat.cf.T @ f) / rho
    T = _transform(lat, u)
    k = np.einsum("nmi,in->mn", T, f) / rho[None, :]
    c = cumulants_from_moments(k)
    cs = c.copy()
    w1 = np.broadcast_to(np.asarray(w1, dtype=np.float64), rho.shape)
    xx, yy, zz = POS[(2, 0, 0)], POS[(0, 2, 0)], POS[(0, 0, 2)]
    for m in ((1, 1, 0), (1, 0, 1), (0, 1, 1)):
        cs[POS[m]] = (1.0 - w1) * c[POS[m]]
    dxy = (1.0 - w1) * (c[xx] - c[yy])
    dxz = (1.0 - w1) * (c[xx] - c[zz])
    tr = c[xx] + c[yy] + c[zz]
    tr = tr + w2 * (3.0 * CS2 - tr)
    cs[xx] = (tr + dxy + dxz) / 3.0
    cs[yy] = cs[xx] - dxy
    cs[zz] = cs[xx] - dxz
    for r, m in enumerate(MIDX):
        if ORDER[r] >= 3:
            cs[r] = (1.0 - w_high[ORDER[r] - 3]) * c[r]
    ks = moments_from_cumulants(cs)
    return np.linalg.solve(T, (ks * rho[None, :]).T[:, :, None])[:, :, 0].T
