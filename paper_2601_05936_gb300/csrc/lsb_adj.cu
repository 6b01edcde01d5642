// Discrete adjoint of the frozen-interface step (the paper has no adjoint; the
// forward step is Sec. 2.1 and 2.3).  With the level set held fixed, one
// finest-level step maps the pre-collision populations f_n to f_{n+1} through
// BGK collision with forcing (Eq. 1, feq, omega), push streaming with
// half-way wall bounce-back, and the interpolated bounce-back of Eq. bb with
// the momentum term of Eq. bb_cc and the stress jump of Eq. Sdecomp on cut
// links.  The kernels here apply the transpose of that map's Jacobian to an
// adjoint population field lambda_{n+1} (same layout as f) and accumulate the
// partial derivatives with respect to the case parameters:
//
//   k_adj_seed      lambda_N = dJ/df_N for J = a . observables (Sec. 3.2)
//   k_adj_links     per cut link: transpose of Eq. bb (coefficients of the
//                   parked post-collision values go to the link buffer, the
//                   back-neighbour coefficient is added in place), and of
//                   Eq. bb_cc / Sdecomp down to the pre-collision moments and
//                   strain rate of both link cells (macro adjoint, atomics)
//                   and to sigma, the densities and the dynamic viscosities
//   k_adj_collide   per cell: transpose of the push (a gather), plus the
//                   link-buffer terms, then of the collision and the moments;
//                   omega and acceleration partials
//   k_adj_macro     per interface cell: the moment and strain-rate adjoints
//                   of the cut links carried to the populations
//   k_adj_geometry  once per sweep, when dJ/dphi is asked for: the interface
//                   cells' normal and curvature adjoints through the
//                   least-squares fit to phi (the link fractions' part is
//                   added by k_adj_links)
//
// Precision: lambda and the Jacobians in FP32 (the forward arithmetic), every
// parameter partial summed in FP64.
#include "lsb_kernels.h"

namespace lsb {

namespace {

constexpr int kShCases = 64;  // cases whose link partials a CTA sums in shared memory

// Index of the symmetric pair (a, b) in the strain-rate storage of the
// forward kernels: 2D xx, xy, yy; 3D xx, xy, xz, yy, yz, zz.
template <int D>
__device__ __forceinline__ int sym(int a, int b) {
  const int lo = a < b ? a : b, hi = a < b ? b : a;
  if (D == 2) return lo + hi;
  return lo == 0 ? hi : (lo == 1 ? 2 + hi : 5);
}

// Moments and strain rate S_ab = -(omega / (2 rho c_s^2)) sum_i c_ia c_ib (f_i - feq_i)
// of one cell, S in the symmetric storage order above.
template <int Q>
__device__ __forceinline__ void moments_strain(const float *f, float om, float &drho, float u[3], float *S) {
  using LT = Lat<Q>;
  constexpr int D = LT::D;
  lb_moments<Q>(f, drho, u);
  const float usq = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
  float P[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const float fn = f[i] - feq_dev<Q>(i, drho, u, usq);
    const float c[3] = {(float)LT::cx(i), (float)LT::cy(i), (float)LT::cz(i)};
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
      for (int b = a; b < D; ++b) P[sym<D>(a, b)] += c[a] * c[b] * fn;
  }
  const float s = -1.5f * om / (1.0f + drho);
#pragma unroll
  for (int k = 0; k < D * (D + 1) / 2; ++k) S[k] = s * P[k];
}

}  // namespace

// ------------------------------------------------------------------ seed
// lambda_N[j] at a leaf cell of volume v (finest cells): a_mass[phase] v, plus in
// the gas v sum_a a_u[a] (c_ja - u_a) / (rho V_gas), the derivative of the gas
// velocity observable sum(v u) / V_gas.  obs holds the raw sums of
// k_observables (entry 2 of each case: V_gas).
template <int Q>
// eps > 0: the smoothed-indicator objective (k_observables with eps): the velocity
// weights carry H_eps of phi at the leaf's first finest child, and lphi (finest-level
// adjoint of phi, or NULL) receives the direct term vol H_eps' (a_V + a_X.(x - X)/V +
// a_U.(u - U)/V).  obs holds the raw sums (volume, sum x h vol, sum u h vol).
__global__ void k_adj_seed(Ctx C, BlockShape S, const int *list, int nlist, const float *F, float *lam,
                           const double *wobs, const double *obs, int stride, float eps, float *lphi) {
  using LT = Lat<Q>;
  constexpr int D = LT::D;
  for (int w = blockIdx.x; w < nlist; w += gridDim.x) {
    int x, y, z;
    const LevelDev &L = blk_cell(C, S, list[w], threadIdx.x, x, y, z);
    if (x >= L.n[0] || y >= L.n[1] || z >= L.n[2]) continue;
    const long long c = cidx(L, x, y, z);
    const uint8_t tg = C.tag[L.cell_off + c];
    if (!(tg & TAG_LEAF)) continue;
    const long long N = L.ncell;
    const float *Fl = F + L.cell_off * Q;
    float *lm = lam + L.cell_off * Q;
    const double *a = wobs + (long long)L.case_id * stride;
    const double V = obs[(long long)L.case_id * stride + 2];
    float vol = 1.f;
    for (int k = 0; k < D; ++k) vol *= (float)L.scale;
    const int gas = tg & TAG_GAS;
    float f[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) f[i] = Fl[i * N + c];
    float drho, u[3];
    lb_moments<Q>(f, drho, u);
    const float base = vol * (float)a[gas];
    float au[3] = {0.f, 0.f, 0.f}, auu = 0.f;
    float h = gas ? 1.f : 0.f;
    long long pc = -1;
    if (eps > 0.f) {
      pc = corner_phi_index(C, L, x, y, z);
      h = smooth_h(C.phi[pc], eps);
    }
    if (h != 0.f && V > 0.0) {
      const float s = vol * h / ((1.0f + drho) * (float)V);
      for (int k = 0; k < D; ++k) {
        au[k] = s * (float)a[4 + D + k];
        auu += au[k] * u[k];
      }
    }
    if (eps > 0.f && lphi && V > 0.0) {
      const float dh = smooth_dh(C.phi[pc], eps);
      if (dh != 0.f) {
        const double *o = obs + (long long)L.case_id * stride;
        const int crd[3] = {x, y, z};
        double t = a[2];
        for (int k = 0; k < D; ++k) {
          const double xk = ((double)crd[k] + 0.5) * L.scale;
          t += a[4 + k] * (xk - o[4 + k] / V) / V + a[4 + D + k] * ((double)u[k] - o[4 + D + k] / V) / V;
        }
        lphi[pc] += (float)((double)(vol * dh) * t);  // one leaf per finest cell: no other writer
      }
    }
#pragma unroll
    for (int i = 0; i < Q; ++i)
      lm[i * N + c] = base + au[0] * LT::cx(i) + au[1] * LT::cy(i) + au[2] * LT::cz(i) - auu;
  }
}

// ------------------------------------------------------------------ cut links
// One thread per interface cell x (phase A); for each cut link (x, k), i = opp(k)
// points to y = x + c_i (phase B).  The forward value was
//   q >= 1/2:          fi / 2q + (2q - 1)/2q fk + df / 2q
//   q < 1/2, back ok:  2q fi + (1 - 2q) fb + df
//   otherwise:         fi + df
// with fi, fk the post-collision populations of x parked in the link buffer and
// fb the value streamed into (x, i) from the back neighbour x - c_i.  The link
// buffer receives the coefficients of fi and fk times lambda; the fb term is added
// to lambda_{n+1}(x, i), which only the gather of the back neighbour reads
// ((x, i) is not a cut link when the back neighbour is in phase A, and only this
// thread writes it).  df's adjoint goes to the moments and strain rate of x and y.
//
// grad per case (NG_ADJ doubles): [0] sigma, [1, 2] rho_phys through [p],
// [3, 4] eta, [5, 6] the kinematic viscosity per phase through the relaxation
// rates and times of every level (d omega_l / d nu = -3 omega_l^2 / r_l with
// r_l = 2^(L-1-l)), [7 .. 12] the finest level's lattice acceleration per phase
// (level l uses r_l times it).
template <int Q>
__global__ void k_adj_links(Ctx C, int glevel, const float *__restrict__ F, float *lamN, float *LA, float *MA,
                            double *grad, int ncase, GeoAdj G) {
  using LT = Lat<Q>;
  constexpr int D = LT::D;
  constexpr int NS = D * (D + 1) / 2;
  __shared__ double sg[kShCases * 5];
  const bool shared_sum = ncase <= kShCases;
  for (int k = threadIdx.x; k < kShCases * 5; k += blockDim.x) sg[k] = 0.0;
  __syncthreads();
  const int n = min(C.counters[glevel * NCOUNT + 1], (int)C.list_cap);
  const int2 *lst = C.iface_list + (long long)glevel * C.list_cap;
  const long long NF = C.nfine;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
    const int2 it = lst[e];
    const LevelDev &L = C.lds[it.x];
    const long long c = it.y;
    int x, y, z;
    cell_xyz(L, c, x, y, z);
    const long long fo = L.fine_off;
    const uint32_t cm = C.cmask[fo + c];
    const int cb = C.cbase[fo + c];
    const uint8_t tg = C.tag[L.cell_off + c];
    const int A = tg & TAG_GAS;
    const int Bp = 1 - A;
    const long long N = L.ncell;
    const float *Fl = F + L.cell_off * Q;
    float *lam = lamN + L.cell_off * Q;
    float f[Q];
#pragma unroll
    for (int j = 0; j < Q; ++j) f[j] = Fl[j * N + c];
    float rA, uA[3], SA[6];
    moments_strain<Q>(f, L.omega[A], rA, uA, SA);
    const float phx = C.phi[fo + c];
    float nx[3] = {0.f, 0.f, 0.f};
    for (int a = 0; a < D; ++a) nx[a] = C.nvec[a * NF + fo + c];
    const float kx = C.kappa[fo + c];
    const float etaA = L.eta[A], etaB = L.eta[Bp];
    const float eb = 0.5f * (etaA + etaB);
    const float je = etaB - etaA;
    const float r = je / eb;
    const float sgn = (A == 0) ? 1.0f : -1.0f;
    // macro adjoint of x, summed over its links: rho, u[D], S[NS]
    float mx[1 + 3 + 6];
    for (int m = 0; m < 1 + D + NS; ++m) mx[m] = 0.f;
    double gs = 0.0, grp[2] = {0.0, 0.0}, get[2] = {0.0, 0.0};
    for (int k = 0; k < Q; ++k) {
      if (!(cm & (1u << k))) continue;
      const int i = LT::opp(k);
      const long long li = cb + __popc(cm & ((1u << k) - 1u));
      if (li >= C.link_cap) continue;
      const float lml = lam[k * N + c];
      int yx = x + LT::cx(i), yy = y + LT::cy(i), yz = z + LT::cz(i);
      wrap(L, 0, yx); wrap(L, 1, yy); if (D == 3) wrap(L, 2, yz);
      const long long cy_ = cidx(L, yx, yy, yz);
      const float phy = C.phi[fo + cy_];
      const float q = phx / (phx - phy);
      // Bouzidi branch coefficients
      bool hi = q >= 0.5f, ok = false;
      if (!hi) {
        int bx = x - LT::cx(i), by = y - LT::cy(i), bz = z - LT::cz(i);
        ok = wrap(L, 0, bx) && wrap(L, 1, by) && (D == 2 || wrap(L, 2, bz));
        if (ok) {
          const uint8_t tb = C.tag[L.cell_off + cidx(L, bx, by, bz)];
          ok = (tb & TAG_LEAF) && ((tb & TAG_GAS) == A);
        }
      }
      const float c_fi = hi ? 0.5f / q : (ok ? 2.0f * q : 1.0f);
      const float c_fk = hi ? (2.0f * q - 1.0f) / (2.0f * q) : 0.0f;
      const float c_df = hi ? 0.5f / q : 1.0f;
      LA[2 * li] = c_fi * lml;
      LA[2 * li + 1] = c_fk * lml;
      if (!hi && ok) lam[i * N + c] += (1.0f - 2.0f * q) * lml;
      const float ldf = c_df * lml;
      if (ldf == 0.0f) continue;
      // forward pieces of Eq. bb_cc at this link
      float fy[Q];
#pragma unroll
      for (int j = 0; j < Q; ++j) fy[j] = Fl[j * N + cy_];
      float rB, uB[3], SB[6];
      moments_strain<Q>(fy, L.omega[Bp], rB, uB, SB);
      float nv[3] = {0.f, 0.f, 0.f}, nn = 0.f;
      for (int a = 0; a < D; ++a) {
        nv[a] = (1.0f - q) * nx[a] + q * C.nvec[a * NF + fo + cy_];
        nn += nv[a] * nv[a];
      }
      nn = sqrtf(nn);
      for (int a = 0; a < D; ++a) nv[a] = nn > 0.f ? sgn * nv[a] / nn : 0.f;
      const float kap = sgn * ((1.0f - q) * kx + q * C.kappa[fo + cy_]);
      float Sb[6];
      for (int s = 0; s < NS; ++s) Sb[s] = 0.5f * (SA[s] + SB[s]);
      const float jp = CS2 * (L.rho_phys[Bp] * rB - L.rho_phys[A] * rA);
      const float ci[3] = {(float)LT::cx(i), (float)LT::cy(i), (float)LT::cz(i)};
      float v[3] = {0.f, 0.f, 0.f}, Snn = 0.f, cn = 0.f, cv = 0.f;
      for (int a = 0; a < D; ++a) {
        for (int b = 0; b < D; ++b) v[a] += Sb[sym<D>(a, b)] * nv[b];
        Snn += nv[a] * v[a];
        cn += ci[a] * nv[a];
        cv += ci[a] * v[a];
      }
      const float cvt = cv - Snn * cn;
      // transpose of df = -6 w_i (c_i . u_I - q (1 - q) ccS), ccS = alpha cn^2 - 2 r cn cvt,
      // alpha = (jp + sigma kappa) / (2 eb) - r Snn, r = je / eb
      const float w6 = 6.0f * LT::w(i);
      const float luI = -w6 * ldf;  // times c_i
      const float lccS = w6 * q * (1.0f - q) * ldf;
      const float la = lccS * cn * cn;
      const float lcvt = -2.0f * r * cn * lccS;
      const float lr = -2.0f * cn * cvt * lccS - Snn * la;
      const float ljp = la / (2.0f * eb);
      const float leb = -la * (jp + L.sigma * kap) / (2.0f * eb * eb) - lr * je / (eb * eb);
      const float lje = lr / eb;
      gs += (double)(la * kap / (2.0f * eb));
      grp[Bp] += (double)(ljp * CS2 * rB);
      grp[A] -= (double)(ljp * CS2 * rA);
      get[A] += (double)(0.5f * leb - lje);
      get[Bp] += (double)(0.5f * leb + lje);
      const float lSnn = -r * la - cn * lcvt;
      if (G.phi) {
        // adjoint of the frozen geometry: q (explicit in Eq. bb, in u_I, in q (1 - q)
        // and in the interpolated n, kappa), the link's n_A and kappa_A
        const float om = L.omega[A];
        const float acA = LT::cx(i) * L.acc[A][0] + LT::cy(i) * L.acc[A][1] + LT::cz(i) * L.acc[A][2];
        const float usA = uA[0] * uA[0] + uA[1] * uA[1] + uA[2] * uA[2];
        // post-collision f_i, f_k of x (Eq. 1) and the forward df
        float f_i = 0.f, f_k = 0.f;  // select without dynamic register indexing
#pragma unroll
        for (int j = 0; j < Q; ++j) {
          f_i = j == i ? f[j] : f_i;
          f_k = j == k ? f[j] : f_k;
        }
        const float fi = f_i + om * (feq_dev<Q>(i, rA, uA, usA) - f_i) + 3.0f * LT::w(i) * (1.0f + rA) * acA;
        const float fk = f_k + om * (feq_dev<Q>(k, rA, uA, usA) - f_k) - 3.0f * LT::w(k) * (1.0f + rA) * acA;
        const float ccS = cn * cn * ((jp + L.sigma * kap) / (2.0f * eb) - r * Snn) - 2.0f * r * cn * cvt;
        float cuI = 0.f, cdu = 0.f;
        for (int a = 0; a < D; ++a) {
          cuI += ci[a] * ((1.0f - q) * uA[a] + q * uB[a]);
          cdu += ci[a] * (uB[a] - uA[a]);
        }
        const float df = -w6 * (cuI - q * (1.0f - q) * ccS);
        float lq = 0.f;
        if (hi) {
          lq = lml * (-fi + fk - df) / (2.0f * q * q);
        } else if (ok) {
          int bx = x - LT::cx(i), by = y - LT::cy(i), bz = z - LT::cz(i);
          wrap(L, 0, bx); wrap(L, 1, by); if (D == 3) wrap(L, 2, bz);
          const long long cbk = cidx(L, bx, by, bz);
          float fbv[Q];
#pragma unroll
          for (int j = 0; j < Q; ++j) fbv[j] = Fl[j * N + cbk];
          float rb, ub[3];
          lb_moments<Q>(fbv, rb, ub);
          const float usb = ub[0] * ub[0] + ub[1] * ub[1] + ub[2] * ub[2];
          const float fb_i = Fl[(long long)i * N + cbk];
          const float fb = fb_i + om * (feq_dev<Q>(i, rb, ub, usb) - fb_i) + 3.0f * LT::w(i) * (1.0f + rb) * acA;
          lq = lml * (2.0f * fi - 2.0f * fb);
        }
        lq += ldf * (-w6) * cdu + ldf * w6 * (1.0f - 2.0f * q) * ccS;
        // d ccS / d n_A = cn^2 (-2 r v) + (2 alpha cn - 2 r cvt) c - 2 r cn (Sbar c - 2 cn v - Snn c)
        const float alpha = (jp + L.sigma * kap) / (2.0f * eb) - r * Snn;
        float lnA[3] = {0.f, 0.f, 0.f};
        for (int a = 0; a < D; ++a) {
          float Sc = 0.f;
          for (int b = 0; b < D; ++b) Sc += Sb[sym<D>(a, b)] * ci[b];
          lnA[a] = lccS * (-2.0f * r * cn * cn * v[a] + (2.0f * alpha * cn - 2.0f * r * cvt) * ci[a] -
                           2.0f * r * cn * (Sc - 2.0f * cn * v[a] - Snn * ci[a]));
        }
        const float lkA = lccS * cn * cn * L.sigma / (2.0f * eb);
        // n_A = sgn m / |m|, m = (1 - q) n_x + q n_y; kappa_A = sgn ((1 - q) kappa_x + q kappa_y)
        const long long my = fo + cy_;
        if (nn > 0.f) {
          float nh[3], dot = 0.f;
          for (int a = 0; a < D; ++a) {
            nh[a] = sgn * nv[a];  // m / |m|
            dot += nh[a] * sgn * lnA[a];
          }
          for (int a = 0; a < D; ++a) {
            const float lm = (sgn * lnA[a] - nh[a] * dot) / nn;
            lq += lm * (C.nvec[a * NF + my] - nx[a]);
            atomicAdd(G.n + a * NF + fo + c, (1.0f - q) * lm);
            atomicAdd(G.n + a * NF + my, q * lm);
          }
        }
        const float ky = C.kappa[my];
        lq += sgn * (ky - kx) * lkA;
        atomicAdd(G.kappa + fo + c, sgn * (1.0f - q) * lkA);
        atomicAdd(G.kappa + my, sgn * q * lkA);
        // q = phi_x / (phi_x - phi_y)
        const float den = (phx - phy) * (phx - phy);
        atomicAdd(G.phi + fo + c, -lq * phy / den);
        atomicAdd(G.phi + my, lq * phx / den);
      }
      // macro adjoint: rho through [p], u through u_I, S through Sbar (half to each cell)
      const long long my = fo + cy_;
      mx[0] -= CS2 * L.rho_phys[A] * ljp;
      atomicAdd(MA + my, CS2 * L.rho_phys[Bp] * ljp);
      for (int a = 0; a < D; ++a) {
        mx[1 + a] += (1.0f - q) * luI * ci[a];
        atomicAdd(MA + (1 + a) * NF + my, q * luI * ci[a]);
      }
      for (int a = 0; a < D; ++a)
        for (int b = a; b < D; ++b) {
          // sum of the (a, b) and (b, a) entries of ci n^T lcvt + n n^T lSnn
          const float t = a == b ? ci[a] * nv[a] * lcvt + nv[a] * nv[a] * lSnn
                                 : (ci[a] * nv[b] + ci[b] * nv[a]) * lcvt + 2.0f * nv[a] * nv[b] * lSnn;
          const int s = sym<D>(a, b);
          mx[1 + D + s] += 0.5f * t;
          atomicAdd(MA + (1 + D + s) * NF + my, 0.5f * t);
        }
    }
    for (int m = 0; m < 1 + D + NS; ++m)
      if (mx[m] != 0.f) atomicAdd(MA + m * NF + fo + c, mx[m]);
    const double vals[5] = {gs, grp[0], grp[1], get[0], get[1]};
    for (int k = 0; k < 5; ++k) {
      if (vals[k] == 0.0) continue;
      if (shared_sum) atomicAdd(sg + L.case_id * 5 + k, vals[k]);
      else atomicAdd(grad + (long long)L.case_id * NG_ADJ + k, vals[k]);
    }
  }
  __syncthreads();
  if (shared_sum)
    for (int k = threadIdx.x; k < ncase * 5; k += blockDim.x)
      if (sg[k] != 0.0) atomicAdd(grad + (long long)(k / 5) * NG_ADJ + (k % 5), sg[k]);
}

#ifndef LSB_ADJ_MINB
#define LSB_ADJ_MINB 2  // CTAs of 512 threads per SM the adjoint collision is built for (64 registers,
                        // some spills: 0.354 -> 0.371 of measured HBM against one CTA at 128)
#endif
// ------------------------------------------------------------------ streaming + collision
// One thread per leaf cell.  lambda_c (adjoint of the post-collision values) is
// the transpose of the forward push: population i of x went to x + c_i, to
// (x, opp(i)) at a wall, or to the link buffer across the interface.  Then the
// transpose of the collision f + omega (feq(rho, u) - f) + 3 w rho (c . acc),
// of the moments (d rho / d f_j = 1, d u_a / d f_j = (c_ja - u_a) / rho) and of
// the strain rate S = k Pi, k = -omega / (2 rho c_s^2),
// Pi_ab = sum c_a c_b (f - feq), with dPi_ab / df_j = c_ja c_jb - c_s^2 d_ab
// + u_a u_b - c_ja u_b - u_a c_jb.
template <int Q>
__global__ void __launch_bounds__(512, LSB_ADJ_MINB) k_adj_collide(Ctx C, BlockShape S, const int *__restrict__ list, int nlist,
                                                      const float *__restrict__ F, const float *__restrict__ lamN,
                                                      float *__restrict__ lamO, const float *__restrict__ LA,
                                                      double *grad) {
  using LT = Lat<Q>;
  constexpr int D = LT::D;
  constexpr int NV = 2 + 2 * 3;  // omega per phase, acceleration per phase
  // per-warp FP64 partial sums in shared memory (no loop-carried registers)
  __shared__ double red[32][NV];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  for (int k = threadIdx.x; k < 32 * NV; k += blockDim.x) red[k / NV][k % NV] = 0.0;
  __syncthreads();
  int cur_case = -1;
  auto flush = [&](int case_id) {
    __syncthreads();
    if (threadIdx.x < NV) {
      double s = 0.0;
      for (int w = 0; w < nw; ++w) {
        s += red[w][threadIdx.x];
        red[w][threadIdx.x] = 0.0;
      }
      if (s != 0.0) atomicAdd(grad + (long long)case_id * NG_ADJ + 5 + threadIdx.x, s);
    }
    __syncthreads();
  };
  for (int w = blockIdx.x; w < nlist; w += gridDim.x) {
    const int gb = __ldg(list + w);
    const int4 bi = __ldg(C.blk_info + gb);
    const LevelDev &L = C.lds[bi.x];
    if (L.case_id != cur_case) {
      if (cur_case >= 0) flush(cur_case);
      cur_case = L.case_id;
    }
    float part[NV];  // this cell's omega and acceleration partials, by phase
#pragma unroll
    for (int k = 0; k < NV; ++k) part[k] = 0.f;
    do {
    const int t = threadIdx.x;
    const int x = (bi.y << S.lg[0]) + (t & (S.bs[0] - 1));
    const int y = (bi.z << S.lg[1]) + ((t >> S.lg[0]) & (S.bs[1] - 1));
    const int z = (bi.w << S.lg[2]) + (t >> (S.lg[0] + S.lg[1]));
    const int n0 = L.n[0], n1 = L.n[1], n2 = L.n[2];
    if (x >= n0 || y >= n1 || z >= n2) break;
    const unsigned p0 = (unsigned)L.p[0], p01 = (unsigned)(L.p[0] * L.p[1]);
    const unsigned c = x + p0 * y + p01 * z;
    const uint8_t tg = C.tag[L.cell_off + c];
    // leaves and the covered cells that leaves stream from collide and push; a
    // push into any other cell is not used, and lambda is zero there
    if (!(tg & (TAG_LEAF | TAG_RLAYER))) break;
    const unsigned N = (unsigned)L.ncell;
    const float *Fl = F + L.cell_off * Q;
    const float *lN = lamN + L.cell_off * Q;
    float *lO = lamO + L.cell_off * Q;
    // ---- transpose of the push
    const bool wxm = x == 0 && !L.per[0], wxp = x == n0 - 1 && !L.per[0];
    const bool wym = y == 0 && !L.per[1], wyp = y == n1 - 1 && !L.per[1];
    const bool wzm = D == 3 && z == 0 && !L.per[2], wzp = D == 3 && z == n2 - 1 && !L.per[2];
    const int dxm = x > 0 ? -1 : n0 - 1, dxp = x < n0 - 1 ? 1 : 1 - n0;
    const int dym = y > 0 ? -(int)p0 : (n1 - 1) * (int)p0, dyp = y < n1 - 1 ? (int)p0 : (1 - n1) * (int)p0;
    const int dzm = z > 0 ? -(int)p01 : (n2 - 1) * (int)p01, dzp = z < n2 - 1 ? (int)p01 : (1 - n2) * (int)p01;
    const bool fine = L.finest != 0;
    uint32_t cm = 0;
    int cb = 0;
    if (fine && (tg & TAG_IFACE)) {
      cm = C.cmask[L.fine_off + c];
      cb = C.cbase[L.fine_off + c];
    }
    const bool ccut = !fine && (tg & TAG_CCUT);
    // lc: adjoint of the post-collision populations.  Held in registers with up to
    // 128 of them per thread (one CTA of 512 per SM): more loads in flight per
    // thread measured faster than two CTAs per SM with lc in shared memory.
    float lc[Q];
#define LC(i) lc[(i)]
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      if (i == LT::REST) {
        LC(i) = lN[LT::REST * N + c];
        continue;
      }
      const int cxi = LT::cx(i), cyi = LT::cy(i), czi = LT::cz(i);
      const int k = LT::opp(i);
      if (cm & (1u << k)) {
        LC(i) = 0.f;
        continue;
      }
      const bool wx = (cxi < 0 && wxm) || (cxi > 0 && wxp);
      const bool wy = (cyi < 0 && wym) || (cyi > 0 && wyp);
      const bool wz = (czi < 0 && wzm) || (czi > 0 && wzp);
      if (!(wx || wy || wz)) {
        const int off = (cxi < 0 ? dxm : (cxi > 0 ? dxp : 0)) + (cyi < 0 ? dym : (cyi > 0 ? dyp : 0)) +
                        (czi < 0 ? dzm : (czi > 0 ? dzp : 0));
        const unsigned ct = (unsigned)((int)c + off);
        LC(i) = lN[i * N + ct];
        if (ccut) {  // coarser level, neighbour of the other phase: the push bounced back
          const uint8_t tt = C.tag[L.cell_off + ct];
          if (!(tt & TAG_GHOST) && ((tt ^ tg) & TAG_GAS)) LC(i) = lN[k * N + c];
        }
      } else if ((wx && !L.slip[0]) || (wy && !L.slip[1]) || (wz && !L.slip[2])) {
        LC(i) = lN[k * N + c];  // no-slip bounce-back
      } else {  // slip walls: the reflected push (into the other phase: bounce-back)
        const int off = (wx ? 0 : (cxi < 0 ? dxm : (cxi > 0 ? dxp : 0))) +
                        (wy ? 0 : (cyi < 0 ? dym : (cyi > 0 ? dyp : 0))) +
                        (wz ? 0 : (czi < 0 ? dzm : (czi > 0 ? dzp : 0)));
        const unsigned ct = (unsigned)((int)c + off);
        const uint8_t tt = C.tag[L.cell_off + ct];
        if (!(tt & TAG_GHOST) && ((tt ^ tg) & TAG_GAS)) LC(i) = lN[k * N + c];
        else LC(i) = lN[mirror_dir<Q>(i, (wx ? 1 : 0) | (wy ? 2 : 0) | (wz ? 4 : 0)) * N + ct];
      }
    }
    if (cm) {
#pragma unroll
      for (int k = 0; k < Q; ++k) {
        if (!(cm & (1u << k))) continue;
        const long long li = cb + __popc(cm & ((1u << k) - 1u));
        if (li >= C.link_cap) continue;
        LC(LT::opp(k)) += LA[2 * li];
        LC(k) += LA[2 * li + 1];
      }
    }
    // ---- transpose of the collision.  f enters only through drho, j and
    // sum lc_i f~_i (omega partial), so it is streamed once and not kept.  The
    // interface cells' moment and strain-rate adjoints are added by k_adj_macro.
    float d = 0.f, jx = 0.f, jy = 0.f, jz = 0.f, slf = 0.f;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      const float fi = Fl[i * N + c];
      d += fi;
      jx += LT::cx(i) * fi;
      jy += LT::cy(i) * fi;
      if (D == 3) jz += LT::cz(i) * fi;
      slf += LC(i) * fi;
    }
    const float drho = d, rho = 1.0f + d, irho = 1.0f / rho;
    const float u[3] = {jx * irho, jy * irho, jz * irho};
    const float usq = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    const int ph = tg & TAG_GAS;
    const float om = L.omega[ph];
    const float ac[3] = {L.acc[ph][0], L.acc[ph][1], L.acc[ph][2]};
    float As = 0.f, Bv[3] = {0.f, 0.f, 0.f}, slfe = 0.f, lac[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      const float cx = LT::cx(i), cy = LT::cy(i), cz = LT::cz(i);
      const float cu = cx * u[0] + cy * u[1] + cz * u[2];
      const float fe = feq_dev<Q>(i, drho, u, usq);
      const float l = LC(i);
      const float wl = LT::w(i) * l;
      // d feq_i / d rho = feq_i / rho (full feq = w + f~eq), d feq_i / d u_a = w rho (3 c_a + 9 cu c_a - 3 u_a)
      As += l * (om * (fe + LT::w(i)) * irho + 3.0f * LT::w(i) * (cx * ac[0] + cy * ac[1] + cz * ac[2]));
      const float g = om * wl * rho;
      Bv[0] += g * (3.0f * cx + 9.0f * cu * cx - 3.0f * u[0]);
      Bv[1] += g * (3.0f * cy + 9.0f * cu * cy - 3.0f * u[1]);
      if (D == 3) Bv[2] += g * (3.0f * cz + 9.0f * cu * cz - 3.0f * u[2]);
      slfe += l * fe;
      lac[0] += 3.0f * wl * rho * cx;
      lac[1] += 3.0f * wl * rho * cy;
      if (D == 3) lac[2] += 3.0f * wl * rho * cz;
    }
    const float lom = slfe - slf;  // sum lc_i (feq_i - f_i)
    float g0[3];
    for (int a = 0; a < 3; ++a) g0[a] = Bv[a] * irho;
    const float base = As - (g0[0] * u[0] + g0[1] * u[1] + g0[2] * u[2]);
#pragma unroll
    for (int j = 0; j < Q; ++j)
      lO[j * N + c] = (1.0f - om) * LC(j) + base + g0[0] * LT::cx(j) + g0[1] * LT::cy(j) + g0[2] * LT::cz(j);
    const float wl = ph ? 0.f : 1.f, wg = ph ? 1.f : 0.f;
    const float r = (float)L.scale;
    const float dnu = -3.0f * om * om / r;  // d omega_l / d nu
    part[0] = wl * lom * dnu;
    part[1] = wg * lom * dnu;
#pragma unroll
    for (int a = 0; a < D; ++a) {
      part[2 + a] = wl * lac[a] * r;
      part[5 + a] = wg * lac[a] * r;
    }
#undef LC
    } while (false);
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      float v = part[k];
      for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
      if (lane == 0) red[warp][k] += (double)v;
    }
  }
  if (cur_case >= 0) flush(cur_case);
}

// ------------------------------------------------------------------ interface-cell moment adjoints
// One thread per interface cell, after k_adj_collide: the adjoints of the cell's
// pre-collision drho, u and strain rate collected by k_adj_links (macro buffer,
// read and cleared for the next step) are carried to the populations and added
// to lambda_n:  lrho + lu . (c_j - u) / rho + k sum_{a<=b} lS_ab (dPi_ab/df_j - Pi_ab / rho),
// with k = -omega / (2 rho c_s^2), Pi_ab = sum c_a c_b (f - feq), and
// dPi_ab/df_j = c_ja c_jb - c_s^2 d_ab + u_a u_b - c_ja u_b - u_a c_jb; the strain
// rate's omega dependence (S / omega) goes to the omega partial.
template <int Q>
__global__ void k_adj_macro(Ctx C, int glevel, const float *__restrict__ F, float *lamO, float *MA, double *grad,
                            int ncase) {
  using LT = Lat<Q>;
  constexpr int D = LT::D;
  constexpr int NS = D * (D + 1) / 2;
  __shared__ double sg[kShCases * 2];
  const bool shared_sum = ncase <= kShCases;
  for (int k = threadIdx.x; k < kShCases * 2; k += blockDim.x) sg[k] = 0.0;
  __syncthreads();
  const int n = min(C.counters[glevel * NCOUNT + 1], (int)C.list_cap);
  const int2 *lst = C.iface_list + (long long)glevel * C.list_cap;
  const long long NF = C.nfine;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
    const int2 it = lst[e];
    const LevelDev &L = C.lds[it.x];
    const long long c = it.y, fc = L.fine_off + c;
    const long long N = L.ncell;
    float m[1 + 3 + 6];
    bool any = false;
    for (int k = 0; k < 1 + D + NS; ++k) {
      m[k] = MA[k * NF + fc];
      MA[k * NF + fc] = 0.f;
      any |= m[k] != 0.f;
    }
    if (!any) continue;
    const float *Fl = F + L.cell_off * Q;
    float *lO = lamO + L.cell_off * Q;
    float d = 0.f, j[3] = {0.f, 0.f, 0.f}, m2[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    for (int i = 0; i < Q; ++i) {
      const float fi = Fl[i * N + c];
      const float c3[3] = {(float)LT::cx(i), (float)LT::cy(i), (float)LT::cz(i)};
      d += fi;
      for (int a = 0; a < D; ++a) {
        j[a] += c3[a] * fi;
        for (int b = a; b < D; ++b) m2[sym<D>(a, b)] += c3[a] * c3[b] * fi;
      }
    }
    const float rho = 1.0f + d, irho = 1.0f / rho;
    const float u[3] = {j[0] * irho, j[1] * irho, j[2] * irho};
    const int ph = C.tag[L.cell_off + c] & TAG_GAS;
    const float om = L.omega[ph];
    const float kk = -1.5f * om * irho;
    const float *mu = m + 1, *mS = m + 1 + D;
    // j-independent parts; Pi_ab = m2_ab - drho c_s^2 d_ab - rho u_a u_b (isotropy of the weights)
    float sP = 0.f, sD = 0.f, sUU = 0.f, muu = 0.f;
    for (int a = 0; a < D; ++a) {
      muu += mu[a] * u[a];
      for (int b = a; b < D; ++b) {
        const float ms = mS[sym<D>(a, b)];
        const float Pab = m2[sym<D>(a, b)] - (a == b ? CS2 * d : 0.f) - rho * u[a] * u[b];
        sP += ms * Pab;
        sUU += ms * u[a] * u[b];
        if (a == b) sD += ms;
      }
    }
    const float base = m[0] - muu * irho + kk * (-CS2 * sD + sUU - sP * irho);
    for (int jj = 0; jj < Q; ++jj) {
      const float cj[3] = {(float)LT::cx(jj), (float)LT::cy(jj), (float)LT::cz(jj)};
      float v = base;
      for (int a = 0; a < D; ++a) {
        v += mu[a] * cj[a] * irho;
        for (int b = a; b < D; ++b)  // for a < b the stored lS holds both orderings
          v += kk * mS[sym<D>(a, b)] * (cj[a] * cj[b] - cj[a] * u[b] - u[a] * cj[b]);
      }
      lO[jj * N + c] += v;
    }
    const double lom = (double)(sP * kk / om) * (double)(-3.0f * om * om / (float)L.scale);  // per nu
    if (lom != 0.0) {
      if (shared_sum) atomicAdd(sg + L.case_id * 2 + ph, lom);
      else atomicAdd(grad + (long long)L.case_id * NG_ADJ + 5 + ph, lom);
    }
  }
  __syncthreads();
  if (shared_sum)
    for (int k = threadIdx.x; k < ncase * 2; k += blockDim.x)
      if (sg[k] != 0.0) atomicAdd(grad + (long long)(k / 2) * NG_ADJ + 5 + (k % 2), sg[k]);
}

// ------------------------------------------------------------------ level-set adjoint
// One thread per interface cell, once after the sweep: the adjoints of the cell's
// normal n = g / |g| and curvature kappa = (|g|^2 tr H - g.H.g) / |g|^3 (summed over
// the window by k_adj_links) go back through the closed-form least-squares
// quadratic of k_geometry (Sec. 2.2): gradient g and Hessian H are linear in the
// stencil sums P = sum v, sx_a = sum o_a v, sxx_a = sum o_a^2 v, sxy = sum o_a o_b v
// over the 3^D points (walls clamp, periodic axes wrap), so each point's phi
// receives l_P + o . l_sx + o^2 . l_sxx + (o_a o_b) . l_sxy.
template <int D>
__global__ void k_adj_geometry(Ctx C, int glevel, GeoAdj G) {
  const int n = min(C.counters[glevel * NCOUNT + 1], (int)C.list_cap);
  const int2 *lst = C.iface_list + (long long)glevel * C.list_cap;
  const long long NF = C.nfine;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
    const int2 it = lst[e];
    const LevelDev &L = C.lds[it.x];
    const long long c = it.y, fc = L.fine_off + c;
    double ln[3] = {0, 0, 0};
    for (int a = 0; a < D; ++a) ln[a] = G.n[a * NF + fc];
    const double lk = G.kappa[fc];
    if (lk == 0.0 && ln[0] == 0.0 && ln[1] == 0.0 && ln[2] == 0.0) continue;
    int x, y, z;
    cell_xyz(L, c, x, y, z);
    double P = 0, sx[3] = {0, 0, 0}, sxx[3] = {0, 0, 0}, sxy[3] = {0, 0, 0};
    for (int oz = (D == 3 ? -1 : 0); oz <= (D == 3 ? 1 : 0); ++oz)
      for (int oy = -1; oy <= 1; ++oy)
        for (int ox = -1; ox <= 1; ++ox) {
          const int xx = clampwrap(L, 0, x + ox), yy = clampwrap(L, 1, y + oy);
          const int zz = D == 3 ? clampwrap(L, 2, z + oz) : 0;
          const double v = (double)C.phi[L.fine_off + cidx(L, xx, yy, zz)];
          const int o[3] = {ox, oy, oz};
          P += v;
          for (int a = 0; a < D; ++a) {
            sx[a] += o[a] * v;
            sxx[a] += o[a] * o[a] * v;
          }
          sxy[0] += ox * oy * v;
          if (D == 3) {
            sxy[1] += ox * oz * v;
            sxy[2] += oy * oz * v;
          }
        }
    // forward fit (as in k_geometry)
    double g[3] = {0, 0, 0}, H[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    double a0, s;
    if (D == 2) {
      const double R = sxx[0] + sxx[1];
      s = (3.0 * R - 4.0 * P) / 6.0;
      a0 = (5.0 * P - 3.0 * R) / 9.0;
      for (int a = 0; a < 2; ++a) {
        g[a] = sx[a] / 6.0;
        H[a][a] = sxx[a] - 6.0 * a0 - 4.0 * s;
      }
      H[0][1] = H[1][0] = sxy[0] / 4.0;
    } else {
      const double R = sxx[0] + sxx[1] + sxx[2];
      s = (R - 2.0 * P) / 6.0;
      a0 = (7.0 * P - 3.0 * R) / 27.0;
      for (int a = 0; a < 3; ++a) {
        g[a] = sx[a] / 18.0;
        H[a][a] = (sxx[a] - 18.0 * a0 - 12.0 * s) / 3.0;
      }
      H[0][1] = H[1][0] = sxy[0] / 12.0;
      H[0][2] = H[2][0] = sxy[1] / 12.0;
      H[1][2] = H[2][1] = sxy[2] / 12.0;
    }
    double g2 = 0, tr = 0, gHg = 0, Hg[3] = {0, 0, 0};
    for (int a = 0; a < D; ++a) {
      g2 += g[a] * g[a];
      tr += H[a][a];
      for (int b = 0; b < D; ++b) Hg[a] += H[a][b] * g[b];
      gHg += g[a] * Hg[a];
    }
    const double mag = sqrt(g2);
    if (!(mag > 1e-12)) continue;  // n = 0, kappa = 0: no dependence
    const double kap = (g2 * tr - gHg) / (mag * mag * mag);
    // l_g, l_H from l_n, l_kappa
    double nd = 0, lg[3] = {0, 0, 0}, lH[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    for (int a = 0; a < D; ++a) nd += g[a] / mag * ln[a];
    for (int a = 0; a < D; ++a) {
      lg[a] = (ln[a] - g[a] / mag * nd) / mag;
      lg[a] += lk * ((2.0 * g[a] * tr - 2.0 * Hg[a]) / (mag * mag * mag) - 3.0 * kap * g[a] / g2);
      for (int b = 0; b < D; ++b) lH[a][b] = lk * ((a == b ? g2 : 0.0) - g[a] * g[b]) / (mag * mag * mag);
    }
    // transpose of the closed-form fit
    double lP = 0, lsx[3] = {0, 0, 0}, lsxx[3] = {0, 0, 0}, lsxy[3] = {0, 0, 0}, la0 = 0, ls = 0, lR = 0;
    if (D == 2) {
      for (int a = 0; a < 2; ++a) {
        lsx[a] = lg[a] / 6.0;
        lsxx[a] += lH[a][a];
        la0 += -6.0 * lH[a][a];
        ls += -4.0 * lH[a][a];
      }
      lsxy[0] = (lH[0][1] + lH[1][0]) / 4.0;
      lP += 5.0 / 9.0 * la0 - 4.0 / 6.0 * ls;
      lR += -3.0 / 9.0 * la0 + 3.0 / 6.0 * ls;
    } else {
      for (int a = 0; a < 3; ++a) {
        lsx[a] = lg[a] / 18.0;
        lsxx[a] += lH[a][a] / 3.0;
        la0 += -6.0 * lH[a][a];
        ls += -4.0 * lH[a][a];
      }
      lsxy[0] = (lH[0][1] + lH[1][0]) / 12.0;
      lsxy[1] = (lH[0][2] + lH[2][0]) / 12.0;
      lsxy[2] = (lH[1][2] + lH[2][1]) / 12.0;
      lP += 7.0 / 27.0 * la0 - 2.0 / 6.0 * ls;
      lR += -3.0 / 27.0 * la0 + 1.0 / 6.0 * ls;
    }
    for (int a = 0; a < D; ++a) lsxx[a] += lR;
    for (int oz = (D == 3 ? -1 : 0); oz <= (D == 3 ? 1 : 0); ++oz)
      for (int oy = -1; oy <= 1; ++oy)
        for (int ox = -1; ox <= 1; ++ox) {
          const int o[3] = {ox, oy, oz};
          double lv = lP + ox * oy * lsxy[0];
          if (D == 3) lv += ox * oz * lsxy[1] + oy * oz * lsxy[2];
          for (int a = 0; a < D; ++a) lv += o[a] * lsx[a] + o[a] * o[a] * lsxx[a];
          const int xx = clampwrap(L, 0, x + ox), yy = clampwrap(L, 1, y + oy);
          const int zz = D == 3 ? clampwrap(L, 2, z + oz) : 0;
          atomicAdd(G.phi + L.fine_off + cidx(L, xx, yy, zz), (float)lv);
        }
  }
}

// ------------------------------------------------------------------ level transfers (multi-level grids)
// Transposes of the Dupuis-Chopard transfers of the forward step (Sec. 2.1, last
// paragraph): the fine ghost ring's values (coarse interpolation at time weight
// theta, f^neq scaled by tau_f / (2 tau_c), fine collision) and the restriction
// (children mean, f^neq scaled by 2 tau_c / tau_f).  The forward values are
// recomputed from the recorded states of the step.

namespace {

// out_j += d/df_j sum_i lam_i f~eq_i(rho(f), u(f)) on deviations f~ = f - w:
// d feq_i / d rho = feq_i / rho, d feq_i / d u_a = w_i rho (3 c_ia + 9 (c_i.u) c_ia - 3 u_a),
// d rho / d f_j = 1, d u_a / d f_j = (c_ja - u_a) / rho.
template <int Q>
__device__ __forceinline__ void feq_T(const float *f, const float *lam, float *out) {
  using LT = Lat<Q>;
  constexpr int D = LT::D;
  float drho, u[3];
  lb_moments<Q>(f, drho, u);
  const float rho = 1.0f + drho, irho = 1.0f / rho;
  const float usq = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
  float As = 0.f, B[3] = {0.f, 0.f, 0.f};
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const float cx = LT::cx(i), cy = LT::cy(i), cz = LT::cz(i);
    const float cu = cx * u[0] + cy * u[1] + cz * u[2];
    As += lam[i] * (feq_dev<Q>(i, drho, u, usq) + LT::w(i)) * irho;
    const float g = lam[i] * LT::w(i) * rho;
    B[0] += g * (3.0f * cx + 9.0f * cu * cx - 3.0f * u[0]);
    B[1] += g * (3.0f * cy + 9.0f * cu * cy - 3.0f * u[1]);
    if (D == 3) B[2] += g * (3.0f * cz + 9.0f * cu * cz - 3.0f * u[2]);
  }
  const float base = As - (B[0] * u[0] + B[1] * u[1] + B[2] * u[2]) * irho;
#pragma unroll
  for (int j = 0; j < Q; ++j)
    out[j] += base + (B[0] * LT::cx(j) + B[1] * LT::cy(j) + B[2] * LT::cz(j)) * irho;
}

// f~ -> f~eq(rho, u) + fac (f~ - f~eq), in place
template <int Q>
__device__ __forceinline__ void rescale_q(float *f, float fac) {
  float drho, u[3];
  lb_moments<Q>(f, drho, u);
  const float usq = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const float fe = feq_dev<Q>(i, drho, u, usq);
    f[i] = fe + fac * (f[i] - fe);
  }
}

// The coarse cells a fine cell interpolates from: the parent and, per axis, the
// upper and lower neighbours where they are leaves (central difference with
// both, one-sided with one), with the weights of the forward interpolation.
// Returns the number of (cell, weight) pairs written (at most 1 + 2 D).
template <int D>
__device__ __forceinline__ int interp_stencil(const Ctx &C, const LevelDev &Lc, int x, int y, int z,
                                              long long *cell, float *wt) {
  const int P[3] = {x >> 1, y >> 1, D == 3 ? (z >> 1) : 0};
  const long long cp = cidx(Lc, P[0], P[1], P[2]);
  int n = 1;
  cell[0] = cp;
  wt[0] = 1.f;
  const int fcrd[3] = {x, y, z};
  for (int a = 0; a < D; ++a) {
    const float delta = ((fcrd[a] & 1) - 0.5f) * 0.5f;
    int up[3] = {P[0], P[1], P[2]}, dn[3] = {P[0], P[1], P[2]};
    up[a] += 1;
    dn[a] -= 1;
    bool upok = wrap(Lc, a, up[a]);
    bool dnok = wrap(Lc, a, dn[a]);
    long long cu = 0, cd = 0;
    if (upok) {
      cu = cidx(Lc, up[0], up[1], up[2]);
      upok = (C.tag[Lc.cell_off + cu] & TAG_LEAF) != 0;
    }
    if (dnok) {
      cd = cidx(Lc, dn[0], dn[1], dn[2]);
      dnok = (C.tag[Lc.cell_off + cd] & TAG_LEAF) != 0;
    }
    if (upok && dnok) {
      cell[n] = cu; wt[n++] = 0.5f * delta;
      cell[n] = cd; wt[n++] = -0.5f * delta;
    } else if (upok) {
      cell[n] = cu; wt[n++] = delta;
      wt[0] -= delta;
    } else if (dnok) {
      cell[n] = cd; wt[n++] = -delta;
      wt[0] += delta;
    }
  }
  return n;
}

// Per-CTA FP64 sums of the transfer partials (nu per phase, acceleration per
// phase), flushed to grad; cases beyond kShCases go straight to global atomics.
struct TransferSums {
  double *sg;
  bool shared_sum;
  __device__ void add(double *grad, int case_id, int k, float v) {
    if (v == 0.f) return;
    if (shared_sum) atomicAdd(sg + case_id * 8 + k, (double)v);
    else atomicAdd(grad + (long long)case_id * NG_ADJ + 5 + k, (double)v);
  }
};

}  // namespace

// One thread per ghost cell g of a fine level: the adjoint of its post-collision
// values is what the fine leaves that pulled them hold in lambda (lamNf, the
// fine level's adjoint after the sub-step): lg_i = lambda(g + c_i, i) where that
// cell is a leaf.  Back through the fine collision, the f^neq rescale and the
// interpolation to the coarse cells, split (1 - theta) to the coarse state at t
// (accumulated in lamX) and theta to the state at t + 1 (lamNc, before the
// coarse sub-step's transpose reads it).
template <int Q>
__global__ void k_adj_ghost(Ctx C, const int2 *cells, int n, float theta, const float *__restrict__ Fold,
                            const float *__restrict__ Fnew, const float *__restrict__ lamNf, float *lamX, float *lamNc,
                            double *grad, int ncase) {
  using LT = Lat<Q>;
  constexpr int D = LT::D;
  __shared__ double sg[kShCases * 8];
  TransferSums T{sg, ncase <= kShCases};
  for (int k = threadIdx.x; k < kShCases * 8; k += blockDim.x) sg[k] = 0.0;
  __syncthreads();
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
    const int2 it = cells[e];
    const LevelDev &F = C.lds[it.x];
    const LevelDev &Lc = C.lds[F.parent_ld];
    const long long c = it.y;
    int x, y, z;
    cell_xyz(F, c, x, y, z);
    float lg[Q];
    bool any = false;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      lg[i] = 0.f;
      if (i == LT::REST) continue;
      int t[3] = {x + LT::cx(i), y + LT::cy(i), z + LT::cz(i)};  // as the forward push: mirrored
      const int o[3] = {x, y, z};                                 // through slip walls
      int mm = 0;
      bool ok = true;
      for (int a = 0; a < D; ++a)
        if (!wrap(F, a, t[a])) {
          if (F.slip[a]) {
            t[a] = o[a];
            mm |= 1 << a;
          } else {
            ok = false;
          }
        }
      if (!ok) continue;
      const long long ct = cidx(F, t[0], t[1], t[2]);
      if (!(C.tag[F.cell_off + ct] & TAG_LEAF)) continue;
      lg[i] = lamNf[F.cell_off * Q + (long long)mirror_dir<Q>(i, mm) * F.ncell + ct];
      any |= lg[i] != 0.f;
    }
    if (!any) continue;
    // forward: interpolation at theta, rescale, fine collision
    long long sc[1 + 2 * 3];
    float sw[1 + 2 * 3];
    const int ns = interp_stencil<D>(C, Lc, x, y, z, sc, sw);
    const long long Nc = Lc.ncell;
    const float *Ao = Fold + Lc.cell_off * Q;
    const float *An = Fnew + Lc.cell_off * Q;
    float fi[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) fi[i] = 0.f;
    for (int s = 0; s < ns; ++s) {
#pragma unroll
      for (int i = 0; i < Q; ++i) {
        float a = Ao[i * Nc + sc[s]];
        if (theta != 0.f) a = (1.0f - theta) * a + theta * An[i * Nc + sc[s]];
        fi[i] += sw[s] * a;
      }
    }
    const long long cpar = sc[0];
    const int ph = C.tag[Lc.cell_off + cpar] & TAG_GAS;
    const float tf = F.tau[ph], tc = Lc.tau[ph];
    const float fac = tf / (2.0f * tc);
    float fr[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) fr[i] = fi[i];
    rescale_q<Q>(fr, fac);
    // transpose of the collision fc = f + om (feq - f) + 3 w rho (c.acc)
    const float om = F.omega[ph];
    const float acc[3] = {F.acc[ph][0], F.acc[ph][1], F.acc[ph][2]};
    float drho, u[3];
    lb_moments<Q>(fr, drho, u);
    const float rho = 1.0f + drho, usq = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    float lr[Q], lom_in[Q];
    float lom = 0.f, lac[3] = {0.f, 0.f, 0.f}, frc = 0.f;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      const float cx = LT::cx(i), cy = LT::cy(i), cz = LT::cz(i);
      lom += lg[i] * (feq_dev<Q>(i, drho, u, usq) - fr[i]);
      const float wl = 3.0f * LT::w(i) * lg[i];
      frc += wl * (cx * acc[0] + cy * acc[1] + cz * acc[2]);
      lac[0] += wl * rho * cx;
      lac[1] += wl * rho * cy;
      lac[2] += wl * rho * cz;
      lr[i] = (1.0f - om) * lg[i];
      lom_in[i] = om * lg[i];
    }
#pragma unroll
    for (int i = 0; i < Q; ++i) lr[i] += frc;  // the forcing's rho
    feq_T<Q>(fr, lom_in, lr);
    // transpose of the rescale f -> feq + fac (f - feq) at fi
    float li[Q], l1[Q];
    float dfe = 0.f;
    {
      float dr2, u2[3];
      lb_moments<Q>(fi, dr2, u2);
      const float us2 = u2[0] * u2[0] + u2[1] * u2[1] + u2[2] * u2[2];
#pragma unroll
      for (int i = 0; i < Q; ++i) {
        dfe += lr[i] * (fi[i] - feq_dev<Q>(i, dr2, u2, us2));
        li[i] = fac * lr[i];
        l1[i] = (1.0f - fac) * lr[i];
      }
    }
    feq_T<Q>(fi, l1, li);
    // transpose of the interpolation, split between the coarse states at t and t + 1
    for (int s = 0; s < ns; ++s) {
#pragma unroll
      for (int i = 0; i < Q; ++i) {
        const float v = sw[s] * li[i];
        const long long o = Lc.cell_off * Q + (long long)i * Nc + sc[s];
        atomicAdd(lamX + o, (1.0f - theta) * v);
        if (theta != 0.f) atomicAdd(lamNc + o, theta * v);
      }
    }
    // partials: omega_f(nu), the rescale factor tau_f / (2 tau_c)(nu), acc_f = r_f acc
    const float rf = (float)F.scale, rc = (float)Lc.scale;
    const float dfac = (3.0f / rf * tc - tf * 3.0f / rc) / (2.0f * tc * tc);
    T.add(grad, F.case_id, ph, lom * (-3.0f * om * om / rf) + dfe * dfac);
    for (int a = 0; a < D; ++a) T.add(grad, F.case_id, 2 + 3 * ph + a, lac[a] * rf);
  }
  __syncthreads();
  if (T.shared_sum)
    for (int k = threadIdx.x; k < ncase * 8; k += blockDim.x)
      if (sg[k] != 0.0) atomicAdd(grad + (long long)(k / 8) * NG_ADJ + 5 + (k % 8), sg[k]);
}

// After the coarse sub-step's transpose: lamX (the ghost rings' share of the
// coarse state at t) joins lamOc and is cleared.  One thread per ghost cell walks
// its interpolation stencil; atomicExch hands each value to one thread.
template <int Q>
__global__ void k_adj_ghost_apply(Ctx C, const int2 *cells, int n, float *lamX, float *lamOc) {
  using LT = Lat<Q>;
  constexpr int D = LT::D;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
    const int2 it = cells[e];
    const LevelDev &F = C.lds[it.x];
    const LevelDev &Lc = C.lds[F.parent_ld];
    const long long c = it.y;
    int x, y, z;
    cell_xyz(F, c, x, y, z);
    long long sc[1 + 2 * 3];
    float sw[1 + 2 * 3];
    const int ns = interp_stencil<D>(C, Lc, x, y, z, sc, sw);
    for (int s = 0; s < ns; ++s)
      for (int i = 0; i < Q; ++i) {
        const long long o = Lc.cell_off * Q + (long long)i * Lc.ncell + sc[s];
        const float v = atomicExch(lamX + o, 0.f);
        if (v != 0.f) lamOc[o] += v;
      }
  }
}

// One thread per restriction-layer cell of a coarse level: its adjoint (written
// by the coarse sub-step's transpose) goes back through the rescale by
// 2 tau_c / tau_f and the mean to the 2^D children's adjoints (lamF, the fine
// level's adjoint at the start of the coarse sub-step), and is cleared.  Ff: the
// fine level's populations the restriction read.
template <int Q>
__global__ void k_adj_restrict(Ctx C, const int2 *cells, int n, const float *__restrict__ Ff, float *lamOc,
                               float *lamF, double *grad, int ncase) {
  using LT = Lat<Q>;
  constexpr int D = LT::D;
  __shared__ double sg[kShCases * 8];
  TransferSums T{sg, ncase <= kShCases};
  for (int k = threadIdx.x; k < kShCases * 8; k += blockDim.x) sg[k] = 0.0;
  __syncthreads();
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
    const int2 it = cells[e];
    const LevelDev &L = C.lds[it.x];
    const LevelDev &F = C.lds[L.child_ld];
    const long long c = it.y;
    int x, y, z;
    cell_xyz(L, c, x, y, z);
    float lr[Q];
    bool any = false;
    float *lo = lamOc + L.cell_off * Q;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      lr[i] = lo[i * L.ncell + c];
      lo[i * L.ncell + c] = 0.f;
      any |= lr[i] != 0.f;
    }
    if (!any) continue;
    const int nz = (D == 3) ? 2 : 1;
    const float inv = 1.0f / (float)(4 * nz);
    const float *Af = Ff + F.cell_off * Q;
    float m[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) m[i] = 0.f;
    for (int sz = 0; sz < nz; ++sz)
      for (int sy = 0; sy < 2; ++sy)
        for (int sx = 0; sx < 2; ++sx) {
          const long long cf = cidx(F, 2 * x + sx, 2 * y + sy, D == 3 ? 2 * z + sz : 0);
#pragma unroll
          for (int i = 0; i < Q; ++i) m[i] += Af[i * F.ncell + cf];
        }
#pragma unroll
    for (int i = 0; i < Q; ++i) m[i] *= inv;
    const int ph = C.tag[L.cell_off + c] & TAG_GAS;
    const float tc = L.tau[ph], tf = F.tau[ph];
    const float fac = 2.0f * tc / tf;
    float lm[Q], l1[Q], dfe = 0.f;
    {
      float dr, u[3];
      lb_moments<Q>(m, dr, u);
      const float usq = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
#pragma unroll
      for (int i = 0; i < Q; ++i) {
        dfe += lr[i] * (m[i] - feq_dev<Q>(i, dr, u, usq));
        lm[i] = fac * lr[i];
        l1[i] = (1.0f - fac) * lr[i];
      }
    }
    feq_T<Q>(m, l1, lm);
    float *lf = lamF + F.cell_off * Q;
    for (int sz = 0; sz < nz; ++sz)
      for (int sy = 0; sy < 2; ++sy)
        for (int sx = 0; sx < 2; ++sx) {
          const long long cf = cidx(F, 2 * x + sx, 2 * y + sy, D == 3 ? 2 * z + sz : 0);
#pragma unroll
          for (int i = 0; i < Q; ++i) lf[i * F.ncell + cf] += lm[i] * inv;
        }
    const float rf = (float)F.scale, rc = (float)L.scale;
    const float dfac = 2.0f * (3.0f / rc * tf - tc * 3.0f / rf) / (tf * tf);
    T.add(grad, L.case_id, ph, dfe * dfac);
  }
  __syncthreads();
  if (T.shared_sum)
    for (int k = threadIdx.x; k < ncase * 8; k += blockDim.x)
      if (sg[k] != 0.0) atomicAdd(grad + (long long)(k / 8) * NG_ADJ + 5 + (k % 8), sg[k]);
}

// ------------------------------------------------------------------ state copies of listed blocks
// All Q populations of the cells of the listed blocks, from one full-size state
// array to another (same offsets).  The adjoint's checkpoints, segment store and
// per-call records hold the cells the step reads (leaves and the covered cells
// leaves stream from); the rest of the dense level boxes is never read.
template <int Q>
__global__ void k_copy_blocks(Ctx C, BlockShape S, const int *list, int n, const float *__restrict__ src,
                              float *__restrict__ dst) {
  for (int w = blockIdx.x; w < n; w += gridDim.x) {
    int x, y, z;
    const LevelDev &L = blk_cell(C, S, list[w], threadIdx.x, x, y, z);
    if (x >= L.n[0] || y >= L.n[1] || z >= L.n[2]) continue;
    const long long c = cidx(L, x, y, z), base = L.cell_off * Q;
#pragma unroll
    for (int i = 0; i < Q; ++i) dst[base + (long long)i * L.ncell + c] = src[base + (long long)i * L.ncell + c];
  }
}

// ------------------------------------------------------------------ launchers
#define LSB_ADJ_Q(Q, fn, L, ...)                                                      \
  do {                                                                                \
    if ((Q) == 9) fn<9><<<(L).grid, (L).block, 0, (L).stream>>>(__VA_ARGS__);         \
    else fn<19><<<(L).grid, (L).block, 0, (L).stream>>>(__VA_ARGS__);                 \
    return cudaGetLastError();                                                        \
  } while (0)

cudaError_t run_adj_seed(int Q, Launch L, Ctx C, BlockShape S, const int *list, int n, const float *F, float *lam,
                         const double *wobs, const double *obs, int stride, float eps, float *lphi) {
  LSB_ADJ_Q(Q, k_adj_seed, L, C, S, list, n, F, lam, wobs, obs, stride, eps, lphi);
}

cudaError_t run_adj_links(int Q, Launch L, Ctx C, int glevel, const float *F, float *lamN, float *LA, float *MA,
                          double *grad, int ncase, GeoAdj G) {
  LSB_ADJ_Q(Q, k_adj_links, L, C, glevel, F, lamN, LA, MA, grad, ncase, G);
}

cudaError_t run_adj_geometry(int D, Launch L, Ctx C, int glevel, GeoAdj G) {
  if (D == 2) k_adj_geometry<2><<<L.grid, L.block, 0, L.stream>>>(C, glevel, G);
  else k_adj_geometry<3><<<L.grid, L.block, 0, L.stream>>>(C, glevel, G);
  return cudaGetLastError();
}

cudaError_t run_adj_collide(int Q, Launch L, Ctx C, BlockShape S, const int *list, int n, const float *F,
                            const float *lamN, float *lamO, const float *LA, double *grad) {
  LSB_ADJ_Q(Q, k_adj_collide, L, C, S, list, n, F, lamN, lamO, LA, grad);
}

cudaError_t run_adj_macro(int Q, Launch L, Ctx C, int glevel, const float *F, float *lamO, float *MA, double *grad,
                          int ncase) {
  LSB_ADJ_Q(Q, k_adj_macro, L, C, glevel, F, lamO, MA, grad, ncase);
}

cudaError_t run_copy_blocks(int Q, Launch L, Ctx C, BlockShape S, const int *list, int n, const float *src,
                            float *dst) {
  LSB_ADJ_Q(Q, k_copy_blocks, L, C, S, list, n, src, dst);
}

cudaError_t run_adj_ghost(int Q, Launch L, Ctx C, const int2 *cells, int n, float theta, const float *Fold,
                          const float *Fnew, const float *lamNf, float *lamX, float *lamNc, double *grad, int ncase) {
  LSB_ADJ_Q(Q, k_adj_ghost, L, C, cells, n, theta, Fold, Fnew, lamNf, lamX, lamNc, grad, ncase);
}

cudaError_t run_adj_ghost_apply(int Q, Launch L, Ctx C, const int2 *cells, int n, float *lamX, float *lamOc) {
  LSB_ADJ_Q(Q, k_adj_ghost_apply, L, C, cells, n, lamX, lamOc);
}

cudaError_t run_adj_restrict(int Q, Launch L, Ctx C, const int2 *cells, int n, const float *Ff, float *lamOc,
                             float *lamF, double *grad, int ncase) {
  LSB_ADJ_Q(Q, k_adj_restrict, L, C, cells, n, Ff, lamOc, lamF, grad, ncase);
}

}  // namespace lsb
