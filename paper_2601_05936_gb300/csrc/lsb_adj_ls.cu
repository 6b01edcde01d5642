// Adjoint of the level-set passes of a step with a MOVING interface (the paper
// has no adjoint; the forward passes are Sec. 2.2 and Eq. hyperbolicExtension).
// Within a window without phase changes, a step maps (f, phi, u~) smoothly:
//   u~ on interface cells = mean u_I of their cut links (moments of f_n, q(phi_n)),
//   n_ext first-order upwind extension sweeps on the other band cells, velocity
//   S(phi) n(phi); TVD-RK3 transport with the fifth-order upwind-biased stencil;
//   one TVD-RK3 pseudo step of the constrained HJ-WENO5 reinitialisation.
// The discrete choices (band, frozen cells, upwind sides, Godunov branch) are
// those of the forward step.  The kernels below apply the transposes of these
// passes as scatter-adds (FP32 atomics): a stencil point that is not updated by
// the pass keeps the pass input's value, so its adjoint goes straight to the
// adjoint of that input.  The lattice Boltzmann part of the step reuses the
// frozen-interface kernels with the geometry of phi_n.
#include "lsb_kernels.h"

namespace lsb {

namespace {

__device__ __forceinline__ bool band_at(const Ctx &C, const LevelDev &L, const BlockShape &S, int x, int y, int z) {
  return (C.bflag[L.block_off + block_of(L, x, y, z, S)] & BF_BAND) != 0;
}

// Level offsets of the seven points at offsets -3..+3 along axis a (walls clamp,
// periodic axes wrap), with their coordinates along a.
__device__ __forceinline__ void line7(const LevelDev &L, int x, int y, int z, int a, long long idx[7], int pc[7][3]) {
  const int crd[3] = {x, y, z};
  for (int m = 0; m < 7; ++m) {
    int p[3] = {x, y, z};
    p[a] = clampwrap(L, a, crd[a] + m - 3);
    idx[m] = cidx(L, p[0], p[1], p[2]);
    pc[m][0] = p[0];
    pc[m][1] = p[1];
    pc[m][2] = p[2];
  }
}

// HJ-WENO5 value and its partial derivatives in the five differences (Jiang & Peng).
__device__ __forceinline__ float weno5_grad(const float v[5], float g[5]) {
  const float eps = 1e-6f;
  const float e[3][5] = {{1.f / 3.f, -7.f / 6.f, 11.f / 6.f, 0.f, 0.f},
                         {0.f, -1.f / 6.f, 5.f / 6.f, 1.f / 3.f, 0.f},
                         {0.f, 0.f, 1.f / 3.f, 5.f / 6.f, -1.f / 6.f}};
  const float b[3][5] = {{1.f, -2.f, 1.f, 0.f, 0.f}, {0.f, 1.f, -2.f, 1.f, 0.f}, {0.f, 0.f, 1.f, -2.f, 1.f}};
  const float c[3][5] = {{1.f, -4.f, 3.f, 0.f, 0.f}, {0.f, 1.f, 0.f, -1.f, 0.f}, {0.f, 0.f, 3.f, -4.f, 1.f}};
  const float gam[3] = {0.1f, 0.6f, 0.3f};
  float d[3], a[3], bv[3], cv[3], sk[3];
  float A = 0.f, num = 0.f;
  for (int k = 0; k < 3; ++k) {
    d[k] = bv[k] = cv[k] = 0.f;
    for (int m = 0; m < 5; ++m) {
      d[k] += e[k][m] * v[m];
      bv[k] += b[k][m] * v[m];
      cv[k] += c[k][m] * v[m];
    }
    sk[k] = 13.f / 12.f * bv[k] * bv[k] + 0.25f * cv[k] * cv[k];
    a[k] = gam[k] / ((sk[k] + eps) * (sk[k] + eps));
    A += a[k];
    num += a[k] * d[k];
  }
  const float val = num / A;
  for (int m = 0; m < 5; ++m) g[m] = 0.f;
  for (int k = 0; k < 3; ++k) {
    const float wk = a[k] / A;
    const float dak = -2.f * gam[k] / ((sk[k] + eps) * (sk[k] + eps) * (sk[k] + eps));
    const float r = (d[k] - val) / A * dak;
    for (int m = 0; m < 5; ++m)
      g[m] += wk * e[k][m] + r * (13.f / 6.f * bv[k] * b[k][m] + 0.5f * cv[k] * c[k][m]);
  }
  return val;
}

}  // namespace

// ------------------------------------------------------------------ forward replay: interface velocity
// u~ on interface cells = mean over cut links of (1 - q) u(x) + q u(y), with the
// pre-collision moments of the stored state F (= f_n) and q from C.phi (= phi_n):
// the values k_ext_init writes from the collide kernel's moments.
template <int Q>
__global__ void k_lsa_init(Ctx C, int glevel, const float *__restrict__ F, float *U0) {
  using LT = Lat<Q>;
  constexpr int D = LT::D;
  const int n = min(C.counters[glevel * NCOUNT + 1], (int)C.list_cap);
  const int2 *lst = C.iface_list + (long long)glevel * C.list_cap;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
    const int2 it = lst[e];
    const LevelDev &L = C.lds[it.x];
    const long long c = it.y;
    int x, y, z;
    cell_xyz(L, c, x, y, z);
    const long long fo = L.fine_off, NF = C.nfine, N = L.ncell;
    const float *Fl = F + L.cell_off * Q;
    const uint32_t m = C.cmask[fo + c];
    float f[Q], rx, ux[3];
#pragma unroll
    for (int j = 0; j < Q; ++j) f[j] = Fl[j * N + c];
    lb_moments<Q>(f, rx, ux);
    const float phx = C.phi[fo + c];
    float acc[3] = {0.f, 0.f, 0.f};
    int cnt = 0;
    for (int k = 0; k < Q; ++k) {
      if (!(m & (1u << k))) continue;
      const int i = LT::opp(k);
      int yx = x + LT::cx(i), yy = y + LT::cy(i), yz = z + LT::cz(i);
      wrap(L, 0, yx); wrap(L, 1, yy); if (D == 3) wrap(L, 2, yz);
      const long long cy_ = cidx(L, yx, yy, yz);
      const float q = phx / (phx - C.phi[fo + cy_]);
      float fy[Q], ry, uy[3];
#pragma unroll
      for (int j = 0; j < Q; ++j) fy[j] = Fl[j * N + cy_];
      lb_moments<Q>(fy, ry, uy);
      for (int a = 0; a < D; ++a) acc[a] += (1.0f - q) * ux[a] + q * uy[a];
      ++cnt;
    }
    for (int a = 0; a < D; ++a) U0[a * NF + fo + c] = acc[a] / (float)cnt;
  }
}

// ------------------------------------------------------------------ transpose of the interface velocity
// For interface cell x with cnt cut links: lu = LS0(x) / cnt per link; the moment
// adjoints go to the macro buffer's u slots of x and y (carried to the populations
// by k_adj_macro), the q adjoint to phi(x), phi(y); LS0(x) is then cleared (the
// pass overwrote u~ there).
template <int Q>
__global__ void k_lsa_init_T(Ctx C, int glevel, const float *__restrict__ F, float *LS0, float *MA, float *LPHI) {
  using LT = Lat<Q>;
  constexpr int D = LT::D;
  const int n = min(C.counters[glevel * NCOUNT + 1], (int)C.list_cap);
  const int2 *lst = C.iface_list + (long long)glevel * C.list_cap;
  const long long NF = C.nfine;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
    const int2 it = lst[e];
    const LevelDev &L = C.lds[it.x];
    const long long c = it.y;
    int x, y, z;
    cell_xyz(L, c, x, y, z);
    const long long fo = L.fine_off, N = L.ncell;
    const float *Fl = F + L.cell_off * Q;
    const uint32_t m = C.cmask[fo + c];
    const int cnt = __popc(m);
    float lu[3] = {0.f, 0.f, 0.f};
    for (int a = 0; a < D; ++a) {
      lu[a] = LS0[a * NF + fo + c] / (float)cnt;
      LS0[a * NF + fo + c] = 0.f;
    }
    float f[Q], rx, ux[3];
#pragma unroll
    for (int j = 0; j < Q; ++j) f[j] = Fl[j * N + c];
    lb_moments<Q>(f, rx, ux);
    const float phx = C.phi[fo + c];
    float mx[3] = {0.f, 0.f, 0.f}, lphx = 0.f;
    for (int k = 0; k < Q; ++k) {
      if (!(m & (1u << k))) continue;
      const int i = LT::opp(k);
      int yx = x + LT::cx(i), yy = y + LT::cy(i), yz = z + LT::cz(i);
      wrap(L, 0, yx); wrap(L, 1, yy); if (D == 3) wrap(L, 2, yz);
      const long long cy_ = cidx(L, yx, yy, yz);
      const float phy = C.phi[fo + cy_];
      const float q = phx / (phx - phy);
      float fy[Q], ry, uy[3];
#pragma unroll
      for (int j = 0; j < Q; ++j) fy[j] = Fl[j * N + cy_];
      lb_moments<Q>(fy, ry, uy);
      float lq = 0.f;
      for (int a = 0; a < D; ++a) {
        mx[a] += (1.0f - q) * lu[a];
        atomicAdd(MA + (1 + a) * NF + fo + cy_, q * lu[a]);
        lq += lu[a] * (uy[a] - ux[a]);
      }
      const float den = (phx - phy) * (phx - phy);
      lphx += -lq * phy / den;
      atomicAdd(LPHI + fo + cy_, lq * phx / den);
    }
    for (int a = 0; a < D; ++a) atomicAdd(MA + (1 + a) * NF + fo + c, mx[a]);
    atomicAdd(LPHI + fo + c, lphx);
  }
}

// ------------------------------------------------------------------ TVD-RK3 bookkeeping of a transposed pass
// Per updated cell c of the pass (band cells; without frozen cells for the
// reinitialisation), for the Shu-Osher stages p1 = p0 + R(p0),
// p2 = 3/4 p0 + 1/4 (p1 + R(p1)), p3 = 1/3 p0 + 2/3 (p2 + R(p2)):
//   mode 0: L0 = L3 / 3, L2 = 2/3 L3      (L0 holds L3 at every other cell)
//   mode 1: L0 += 3/4 L2, L1 = 1/4 L2
//   mode 2: L0 += L1
//   mode 3: L0 += Ls0 / (phi*^2 + 1)^(3/2)  (reinitialisation: S(phi*) in R)
// The stencil transposes (k_lsa_*_rt) add R's Jacobian transposes in between.
template <int D>
__global__ void k_lsa_mix(Ctx C, BlockShape S, int glevel, int mode, int use_frozen, const float *L3, float *L0,
                          float *L1, float *L2, const float *Ls0) {
  const int nl = min(C.counters[glevel * NCOUNT + 3], C.band_cap);
  for (int w = blockIdx.x; w < nl; w += gridDim.x) {
    int x, y, z;
    const LevelDev &L = band_cell(C, S, glevel, w, threadIdx.x, x, y, z);
    if (x >= L.n[0] || y >= L.n[1] || z >= L.n[2]) continue;
    const long long fc = L.fine_off + cidx(L, x, y, z);
    if (use_frozen && C.frozen[fc]) continue;
    if (mode == 0) {
      const float m3 = L3[fc];
      L0[fc] = m3 / 3.0f;
      L2[fc] = 2.0f / 3.0f * m3;
    } else if (mode == 1) {
      const float m2 = L2[fc];
      L0[fc] += 0.75f * m2;
      L1[fc] = 0.25f * m2;
    } else if (mode == 2) {
      L0[fc] += L1[fc];
    } else {
      const float p = C.phi[fc];
      const float d = p * p + 1.0f;
      L0[fc] += Ls0[fc] / (d * sqrtf(d));
    }
  }
}

// Transposed right-hand side of one reinitialisation stage, R(p) = -dtau S0 (|grad p|_G - 1)
// with Godunov's Hamiltonian on HJ-WENO5 one-sided differences.  The stage value p
// is pin at band cells that are not frozen and C.phi (= phi*) elsewhere, as in the
// forward stage; mu = scale * MU(c).  Stencil points updated by the stage receive
// their part in Lt, all others in L0; Ls0(c) accumulates d/dS0.
template <int D>
__global__ void k_lsa_reinit_rt(Ctx C, BlockShape S, int glevel, const float *pin, const float *MU, float scale,
                                float *Lt, float *L0, float *Ls0) {
  const int nl = min(C.counters[glevel * NCOUNT + 3], C.band_cap);
  for (int w = blockIdx.x; w < nl; w += gridDim.x) {
    int x, y, z;
    const LevelDev &L = band_cell(C, S, glevel, w, threadIdx.x, x, y, z);
    if (x >= L.n[0] || y >= L.n[1] || z >= L.n[2]) continue;
    const long long fo = L.fine_off;
    const long long fc = fo + cidx(L, x, y, z);
    if (C.frozen[fc]) continue;
    const float mu = scale * MU[fc];
    if (mu == 0.0f) continue;
    const float s0 = C.s0[fc];
    long long idx[3][7];
    bool upd[3][7];
    float gdm[3][5], gdp[3][5], dga_m[3], dga_p[3];
    float g2 = 0.f;
    for (int a = 0; a < D; ++a) {
      int pc[7][3];
      line7(L, x, y, z, a, idx[a], pc);
      float P[7];
      for (int m = 0; m < 7; ++m) {
        const long long cc = fo + idx[a][m];
        upd[a][m] = pin != C.phi && band_at(C, L, S, pc[m][0], pc[m][1], pc[m][2]) && !C.frozen[cc];
        P[m] = upd[a][m] ? pin[cc] : C.phi[cc];
      }
      const float vm[5] = {P[1] - P[0], P[2] - P[1], P[3] - P[2], P[4] - P[3], P[5] - P[4]};
      const float vp[5] = {P[6] - P[5], P[5] - P[4], P[4] - P[3], P[3] - P[2], P[2] - P[1]};
      const float dm = weno5_grad(vm, gdm[a]);
      const float dp = weno5_grad(vp, gdp[a]);
      float ga;
      bool use_m;
      if (s0 > 0.f) {
        const float a1 = fmaxf(dm, 0.f) * fmaxf(dm, 0.f), a2 = fminf(dp, 0.f) * fminf(dp, 0.f);
        use_m = a1 >= a2;
        ga = use_m ? a1 : a2;
        dga_m[a] = use_m ? 2.f * fmaxf(dm, 0.f) : 0.f;
        dga_p[a] = use_m ? 0.f : 2.f * fminf(dp, 0.f);
      } else {
        const float a1 = fminf(dm, 0.f) * fminf(dm, 0.f), a2 = fmaxf(dp, 0.f) * fmaxf(dp, 0.f);
        use_m = a1 >= a2;
        ga = use_m ? a1 : a2;
        dga_m[a] = use_m ? 2.f * fminf(dm, 0.f) : 0.f;
        dga_p[a] = use_m ? 0.f : 2.f * fmaxf(dp, 0.f);
      }
      g2 += ga;
    }
    const float sq = sqrtf(g2);
    const float dt = L.dtau_reinit;
    Ls0[fc] += mu * (-dt * (sq - 1.0f));
    const float lg2 = sq > 0.f ? mu * (-dt * s0 / (2.0f * sq)) : 0.f;
    if (lg2 == 0.f) continue;
    for (int a = 0; a < D; ++a) {
      float lp[7] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
      const float wm = lg2 * dga_m[a], wp = lg2 * dga_p[a];
      for (int m = 0; m < 5; ++m) {
        lp[m + 1] += wm * gdm[a][m];  // vm[m] = P[m+1] - P[m]
        lp[m] -= wm * gdm[a][m];
        lp[6 - m] += wp * gdp[a][m];  // vp[m] = P[6-m] - P[5-m]
        lp[5 - m] -= wp * gdp[a][m];
      }
      for (int m = 0; m < 7; ++m)
        if (lp[m] != 0.f) atomicAdd((upd[a][m] ? Lt : L0) + fo + idx[a][m], lp[m]);
    }
  }
}

// Transposed right-hand side of one transport stage, L(p) = -sum_a u~_a d_a(p) with the
// fifth-order upwind-biased stencil on the side of sign(u~_a) (C.ut0 = the committed
// u~ of the step).  Stage value: pin at band cells, C.phi (= phi_n) elsewhere.
// mu = scale * MU(c); stencil points in the band get their part in Lt, others in L0;
// LU (adjoint of u~ at c) gets -mu d_a(p).
template <int D>
__global__ void k_lsa_adv_rt(Ctx C, BlockShape S, int glevel, const float *pin, const float *MU, float scale,
                             float *Lt, float *L0, float *LU) {
  const float wm[7] = {-2.f / 60.f, 15.f / 60.f, -60.f / 60.f, 20.f / 60.f, 30.f / 60.f, -3.f / 60.f, 0.f};
  const int nl = min(C.counters[glevel * NCOUNT + 3], C.band_cap);
  const long long NF = C.nfine;
  for (int w = blockIdx.x; w < nl; w += gridDim.x) {
    int x, y, z;
    const LevelDev &L = band_cell(C, S, glevel, w, threadIdx.x, x, y, z);
    if (x >= L.n[0] || y >= L.n[1] || z >= L.n[2]) continue;
    const long long fo = L.fine_off;
    const long long fc = fo + cidx(L, x, y, z);
    const float mu = scale * MU[fc];
    if (mu == 0.0f) continue;
    for (int a = 0; a < D; ++a) {
      long long idx[7];
      int pc[7][3];
      line7(L, x, y, z, a, idx, pc);
      const float ua = C.ut0[a * NF + fc];
      float da = 0.f;
      for (int m = 0; m < 7; ++m) {
        // d5m: weights wm on points 0..5; d5p: -wm mirrored onto points 6..1
        const float cw = ua >= 0.f ? wm[m] : -wm[6 - m];
        if (cw == 0.f) continue;
        const long long cc = fo + idx[m];
        const bool upd = pin != C.phi && band_at(C, L, S, pc[m][0], pc[m][1], pc[m][2]);
        da += cw * (upd ? pin[cc] : C.phi[cc]);
        atomicAdd((upd ? Lt : L0) + cc, -ua * cw * mu);
      }
      LU[a * NF + fc] += -mu * da;
    }
  }
}

// ------------------------------------------------------------------ transpose of an extension sweep
// Forward sweep k on band cells that are not interface cells:
//   u_{k+1}(c) = u_k(c) - dtau sum_a v_a (v_a > 0 ? u_k(c) - u_k(c - e_a) : u_k(c + e_a) - u_k(c)),
// v = S(phi) n(phi) (central n), a neighbour outside the band read from S0 (= the
// committed u~ of the previous step, which the sweeps leave alone).  Lout holds a copy
// of Lin (the identity part); here the rest: Lout(c), Lout(neighbour) or, for a
// neighbour outside the band, LOFF; LV(a, c) accumulates d/dv_a over the sweeps.
template <int D>
__global__ void k_lsa_ext_T(Ctx C, BlockShape S, int glevel, const float *Sk, const float *S0, const float *Lin,
                            float *Lout, float *LOFF, float *LV) {
  const int nl = min(C.counters[glevel * NCOUNT + 3], C.band_cap);
  const long long NF = C.nfine;
  for (int w = blockIdx.x; w < nl; w += gridDim.x) {
    int x, y, z;
    const LevelDev &L = band_cell(C, S, glevel, w, threadIdx.x, x, y, z);
    if (x >= L.n[0] || y >= L.n[1] || z >= L.n[2]) continue;
    const long long fo = L.fine_off;
    const long long c = cidx(L, x, y, z);
    if (C.tag[L.cell_off + c] & TAG_IFACE) continue;
    const int crd[3] = {x, y, z};
    float nv[3], gm = 0.f;
    for (int a = 0; a < D; ++a) {
      int p[3] = {x, y, z}, m[3] = {x, y, z};
      p[a] = clampwrap(L, a, crd[a] + 1);
      m[a] = clampwrap(L, a, crd[a] - 1);
      nv[a] = 0.5f * (C.phi[fo + cidx(L, p[0], p[1], p[2])] - C.phi[fo + cidx(L, m[0], m[1], m[2])]);
      gm += nv[a] * nv[a];
    }
    gm = sqrtf(gm);
    const float ph = C.phi[fo + c];
    const float sg = ph / sqrtf(ph * ph + 1.0f);
    const float dt = L.dtau_ext;
    float lc[3] = {0.f, 0.f, 0.f};
    for (int b = 0; b < D; ++b) lc[b] = Lin[b * NF + fo + c];
    for (int a = 0; a < D; ++a) {
      const float va = gm > 0.f ? sg * nv[a] / gm : 0.f;
      int nb[3] = {x, y, z};
      nb[a] = clampwrap(L, a, crd[a] + (va > 0.f ? -1 : 1));
      const long long cn = cidx(L, nb[0], nb[1], nb[2]);
      const bool inb = band_at(C, L, S, nb[0], nb[1], nb[2]);
      const float *src = inb ? Sk : S0;
      float lva = 0.f;
      for (int b = 0; b < D; ++b) {
        const float u0 = Sk[b * NF + fo + c], un = src[b * NF + fo + cn];
        lva += lc[b] * (-dt * (va > 0.f ? (u0 - un) : (un - u0)));
        if (lc[b] == 0.f || va == 0.f) continue;
        atomicAdd(Lout + b * NF + fo + c, lc[b] * (va > 0.f ? -dt * va : dt * va));
        atomicAdd((inb ? Lout : LOFF) + b * NF + fo + cn, lc[b] * (va > 0.f ? dt * va : -dt * va));
      }
      LV[a * NF + fo + c] += lva;
    }
  }
}

// d/dphi of the extension velocity v = S(phi) n, n = g / |g|, g_a = (phi(c + e_a) - phi(c - e_a)) / 2,
// S(phi) = phi / sqrt(phi^2 + 1), from LV (summed over the sweeps); LV is cleared.
template <int D>
__global__ void k_lsa_ext_v(Ctx C, BlockShape S, int glevel, float *LV, float *LPHI) {
  const int nl = min(C.counters[glevel * NCOUNT + 3], C.band_cap);
  const long long NF = C.nfine;
  for (int w = blockIdx.x; w < nl; w += gridDim.x) {
    int x, y, z;
    const LevelDev &L = band_cell(C, S, glevel, w, threadIdx.x, x, y, z);
    if (x >= L.n[0] || y >= L.n[1] || z >= L.n[2]) continue;
    const long long fo = L.fine_off;
    const long long c = cidx(L, x, y, z);
    if (C.tag[L.cell_off + c] & TAG_IFACE) continue;
    float lv[3] = {0.f, 0.f, 0.f};
    bool any = false;
    for (int a = 0; a < D; ++a) {
      lv[a] = LV[a * NF + fo + c];
      LV[a * NF + fo + c] = 0.f;
      any |= lv[a] != 0.f;
    }
    if (!any) continue;
    const int crd[3] = {x, y, z};
    long long ip[3], im[3];
    float nv[3], gm = 0.f;
    for (int a = 0; a < D; ++a) {
      int p[3] = {x, y, z}, m[3] = {x, y, z};
      p[a] = clampwrap(L, a, crd[a] + 1);
      m[a] = clampwrap(L, a, crd[a] - 1);
      ip[a] = fo + cidx(L, p[0], p[1], p[2]);
      im[a] = fo + cidx(L, m[0], m[1], m[2]);
      nv[a] = 0.5f * (C.phi[ip[a]] - C.phi[im[a]]);
      gm += nv[a] * nv[a];
    }
    gm = sqrtf(gm);
    if (!(gm > 0.f)) continue;
    const float ph = C.phi[fo + c];
    const float d = ph * ph + 1.0f;
    const float sg = ph / sqrtf(d);
    float ls = 0.f, dot = 0.f;
    for (int a = 0; a < D; ++a) {
      ls += lv[a] * nv[a] / gm;
      dot += nv[a] / gm * sg * lv[a];
    }
    atomicAdd(LPHI + fo + c, ls / (d * sqrtf(d)));
    for (int a = 0; a < D; ++a) {
      const float lg = (sg * lv[a] - nv[a] / gm * dot) / gm;
      atomicAdd(LPHI + ip[a], 0.5f * lg);
      atomicAdd(LPHI + im[a], -0.5f * lg);
    }
  }
}

__global__ void k_lsa_axpy(long long n, const float *x, float *y) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] += x[i];
}

// ------------------------------------------------------------------ launchers
#define LSA_Q(kern, ...)                                                          \
  do {                                                                            \
    if (Q == 9) kern<9><<<L.grid, L.block, 0, L.stream>>>(__VA_ARGS__);           \
    else kern<19><<<L.grid, L.block, 0, L.stream>>>(__VA_ARGS__);                 \
    return cudaGetLastError();                                                    \
  } while (0)
#define LSA_D(kern, ...)                                                          \
  do {                                                                            \
    if (D == 2) kern<2><<<L.grid, L.block, 0, L.stream>>>(__VA_ARGS__);           \
    else kern<3><<<L.grid, L.block, 0, L.stream>>>(__VA_ARGS__);                  \
    return cudaGetLastError();                                                    \
  } while (0)

cudaError_t run_lsa_init(int Q, Launch L, Ctx C, int glevel, const float *F, float *U0) {
  LSA_Q(k_lsa_init, C, glevel, F, U0);
}
cudaError_t run_lsa_init_T(int Q, Launch L, Ctx C, int glevel, const float *F, float *LS0, float *MA, float *LPHI) {
  LSA_Q(k_lsa_init_T, C, glevel, F, LS0, MA, LPHI);
}
cudaError_t run_lsa_mix(int D, Launch L, Ctx C, BlockShape S, int glevel, int mode, int use_frozen, const float *L3,
                        float *L0, float *L1, float *L2, const float *Ls0) {
  LSA_D(k_lsa_mix, C, S, glevel, mode, use_frozen, L3, L0, L1, L2, Ls0);
}
cudaError_t run_lsa_reinit_rt(int D, Launch L, Ctx C, BlockShape S, int glevel, const float *pin, const float *MU,
                              float scale, float *Lt, float *L0, float *Ls0) {
  LSA_D(k_lsa_reinit_rt, C, S, glevel, pin, MU, scale, Lt, L0, Ls0);
}
cudaError_t run_lsa_adv_rt(int D, Launch L, Ctx C, BlockShape S, int glevel, const float *pin, const float *MU,
                           float scale, float *Lt, float *L0, float *LU) {
  LSA_D(k_lsa_adv_rt, C, S, glevel, pin, MU, scale, Lt, L0, LU);
}
cudaError_t run_lsa_ext_T(int D, Launch L, Ctx C, BlockShape S, int glevel, const float *Sk, const float *S0,
                          const float *Lin, float *Lout, float *LOFF, float *LV) {
  LSA_D(k_lsa_ext_T, C, S, glevel, Sk, S0, Lin, Lout, LOFF, LV);
}
cudaError_t run_lsa_ext_v(int D, Launch L, Ctx C, BlockShape S, int glevel, float *LV, float *LPHI) {
  LSA_D(k_lsa_ext_v, C, S, glevel, LV, LPHI);
}
cudaError_t run_lsa_axpy(Launch L, long long n, const float *x, float *y) {
  k_lsa_axpy<<<L.grid, L.block, 0, L.stream>>>(n, x, y);
  return cudaGetLastError();
}

}  // namespace lsb

namespace lsb {

// Latch whether the last classification of level glevel listed flipped cells.
__global__ void k_lsa_flipflag(const int *counters, int glevel, int *flag) {
  if (threadIdx.x == 0 && blockIdx.x == 0 && counters[glevel * NCOUNT + 2] > 0) *flag = 1;
}

cudaError_t run_lsa_flipflag(Launch L, const int *counters, int glevel, int *flag) {
  k_lsa_flipflag<<<1, 32, 0, L.stream>>>(counters, glevel, flag);
  return cudaGetLastError();
}

}  // namespace lsb
