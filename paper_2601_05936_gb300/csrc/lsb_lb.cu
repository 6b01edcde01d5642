// Lattice Boltzmann kernels: fused BGK collide + push streaming with wall
// bounce-back (Sec. 2.1, Eq. 1, feq, omega, forcing, bb at q = 1/2), the
// interface bounce-back post-pass (Sec. 2.3, Eq. bb, bb_cc, Sdecomp), the
// Dupuis-Chopard level transfers (Sec. 2.1 last paragraph), initialisation and
// the float64 observables (Sec. 3.2).
//
// Populations are stored as deviations f~ = f - w (per-phase rest density 1),
// structure of arrays per level: f[q * ncell + cell], x fastest, so a warp of a
// block row touches consecutive words for every q.  The state between steps is
// the PRE-collision (post-stream) population; a step reads it once, collides in
// registers and pushes every population to its destination once: 2*Q*sizeof(T)
// bytes of HBM traffic per cell update.
#include <cuda.h>

#include <algorithm>
#include <mutex>
#include <type_traits>

#include "lsb_kernels.h"
#include "lsb_tma.cuh"

// CTAs of 128 threads per SM the ghost-ring and cut-link kernels are compiled for
// (registers capped to fit; 0 leaves the compiler's choice)
#ifndef LSB_GHOST_MINB
#define LSB_GHOST_MINB 0
#endif
#ifndef LSB_LINK_MINB
#define LSB_LINK_MINB 0
#endif
#if LSB_GHOST_MINB > 0
#define LSB_GHOST_LB __launch_bounds__(128, LSB_GHOST_MINB)
#else
#define LSB_GHOST_LB
#endif
#if LSB_LINK_MINB > 0
#define LSB_LINK_LB __launch_bounds__(128, LSB_LINK_MINB)
#else
#define LSB_LINK_LB
#endif

namespace lsb {

// BGK collision with forcing (Eq. 1), in place on deviations f~ = f - w, written per pair
// (i, opp(i)):
//   f_i' = (1 - om) f_i + w_i [om drho + rho (H cu^2 - K) + 3 rho c_i.v],
//   H = 9 om / 2, K = 3 om usq / 2, v = om u + acc, cu = c_i.u,
// where the first two terms are even and the last odd under c_i -> -c_i, so one evaluation
// serves both populations of a pair.  drho and u are the pre-collision moments.
template <int Q>
__device__ __forceinline__ void lb_collide(float *f, float om, const float acc[3], float &drho, float u[3]) {
  using LT = Lat<Q>;
  lb_moments<Q>(f, drho, u);
  const float rho = 1.0f + drho;
  const float usq = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
  const float keep = 1.0f - om, A = om * drho, K = 1.5f * om * usq, H = 4.5f * om, r3 = 3.0f * rho;
  const float v0 = om * u[0] + acc[0], v1 = om * u[1] + acc[1], v2 = om * u[2] + acc[2];
  f[LT::REST] = keep * f[LT::REST] + LT::w(LT::REST) * (A - rho * K);
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    if (i == LT::REST || LT::opp(i) < i) continue;
    const int k = LT::opp(i);
    const float cx = LT::cx(i), cy = LT::cy(i), cz = LT::cz(i);
    const float cu = cx * u[0] + cy * u[1] + cz * u[2];
    const float cv = cx * v0 + cy * v1 + cz * v2;
    const float P = LT::w(i) * (A + rho * (H * cu * cu - K));
    const float R = LT::w(i) * r3 * cv;
    f[i] = keep * f[i] + (P + R);
    f[k] = keep * f[k] + (P - R);
  }
}

// Cumulant collision on D3Q27 (the paper's gas operator in 3D, Sec. 3.2), in place on
// deviations f~ = f - w, with forcing as for BGK.  The central moments follow from three
// passes of 3-point transforms (z, y, x: populations at -1, 0, +1 -> orders 0, 1, 2 about
// u_a).  The second cumulants (= central moments / rho) relax: off-diagonal ones and the
// differences of the diagonal ones with om, the trace with rate 1 to 3 c_s^2 = 1.  Every
// higher cumulant relaxes with rate 1 to zero, so the post-collision central moments of
// orders 3 to 6 are those of a Gaussian with the relaxed second moments (odd ones vanish;
// even ones by Isserlis' theorem); the inverse passes give the populations.
__device__ __forceinline__ void cumulant_collide27(float *f, float om, const float acc[3], float &drho, float u[3]) {
  using LT = Lat<27>;
  lb_moments<27>(f, drho, u);
  const float rho = 1.0f + drho, ir = 1.0f / rho;
  float m[27];  // slot (cx + 1) 9 + (cy + 1) 3 + (cz + 1); after the passes (px 9 + py 3 + pz): central moments
#pragma unroll
  for (int i = 0; i < 27; ++i) m[(LT::cx(i) + 1) * 9 + (LT::cy(i) + 1) * 3 + (LT::cz(i) + 1)] = f[i] + LT::w(i);
  auto fwd = [](float &a, float &b, float &c, float v) {
    const float M0 = a + b + c, M1 = c - a, M2 = a + c;
    a = M0;
    b = M1 - v * M0;
    c = M2 - 2.0f * v * M1 + v * v * M0;
  };
#pragma unroll
  for (int p = 0; p < 9; ++p) fwd(m[p * 3], m[p * 3 + 1], m[p * 3 + 2], u[2]);
#pragma unroll
  for (int p = 0; p < 9; ++p) fwd(m[(p / 3) * 9 + (p % 3)], m[(p / 3) * 9 + 3 + (p % 3)], m[(p / 3) * 9 + 6 + (p % 3)], u[1]);
#pragma unroll
  for (int p = 0; p < 9; ++p) fwd(m[p], m[9 + p], m[18 + p], u[0]);
  const float kxx = m[18] * ir, kyy = m[6] * ir, kzz = m[2] * ir;
  const float kxy = m[12] * ir, kxz = m[10] * ir, kyz = m[4] * ir;
  const float r1 = 1.0f - om;
  const float dxy = r1 * (kxx - kyy), dxz = r1 * (kxx - kzz);
  const float sxx = (1.0f + dxy + dxz) * (1.0f / 3.0f), syy = sxx - dxy, szz = sxx - dxz;
  const float sxy = r1 * kxy, sxz = r1 * kxz, syz = r1 * kyz;
#pragma unroll
  for (int p = 0; p < 27; ++p) m[p] = 0.f;
  m[0] = rho;
  m[18] = rho * sxx; m[6] = rho * syy; m[2] = rho * szz;
  m[12] = rho * sxy; m[10] = rho * sxz; m[4] = rho * syz;
  m[24] = rho * (sxx * syy + 2.0f * sxy * sxy);  // (2, 2, 0)
  m[20] = rho * (sxx * szz + 2.0f * sxz * sxz);  // (2, 0, 2)
  m[8] = rho * (syy * szz + 2.0f * syz * syz);   // (0, 2, 2)
  m[22] = rho * (sxx * syz + 2.0f * sxy * sxz);  // (2, 1, 1)
  m[16] = rho * (syy * sxz + 2.0f * sxy * syz);  // (1, 2, 1)
  m[14] = rho * (szz * sxy + 2.0f * sxz * syz);  // (1, 1, 2)
  m[26] = rho * (sxx * syy * szz + 2.0f * (sxx * syz * syz + syy * sxz * sxz + szz * sxy * sxy) +
                 8.0f * sxy * sxz * syz);       // (2, 2, 2)
  auto bwd = [](float &a, float &b, float &c, float v) {
    const float M0 = a, M1 = b + v * M0, M2 = c + 2.0f * v * M1 - v * v * M0;
    a = 0.5f * (M2 - M1);
    b = M0 - M2;
    c = 0.5f * (M2 + M1);
  };
#pragma unroll
  for (int p = 0; p < 9; ++p) bwd(m[p], m[9 + p], m[18 + p], u[0]);
#pragma unroll
  for (int p = 0; p < 9; ++p) bwd(m[(p / 3) * 9 + (p % 3)], m[(p / 3) * 9 + 3 + (p % 3)], m[(p / 3) * 9 + 6 + (p % 3)], u[1]);
#pragma unroll
  for (int p = 0; p < 9; ++p) bwd(m[p * 3], m[p * 3 + 1], m[p * 3 + 2], u[2]);
#pragma unroll
  for (int i = 0; i < 27; ++i) {
    const float F = 3.0f * LT::w(i) * rho * (LT::cx(i) * acc[0] + LT::cy(i) * acc[1] + LT::cz(i) * acc[2]);
    f[i] = m[(LT::cx(i) + 1) * 9 + (LT::cy(i) + 1) * 3 + (LT::cz(i) + 1)] - LT::w(i) + F;
  }
}

// drho, u and the strain rate of an interface cell's pre-collision populations, kept for the
// interface condition (Eq. bb_cc, Sdecomp) in the finest-level macro planes (drho, u[D], S):
// S = -(om / (2 rho c_s^2)) sum_i c_i c_i (f_i - feq_i).  In deviation form the equilibrium's
// second moments are sum_i c_a c_b f~eq_i = drho c_s^2 delta_ab + rho u_a u_b, for the BGK
// equilibrium and for the cumulant model's Gaussian alike, so no per-population feq is needed.
// fi(i) returns pre-collision population i (from the stage or buffer A).
template <int Q, typename Ld>
__device__ __forceinline__ void store_iface_macro(const Ctx &C, long long fc, Ld fi, float om) {
  using LT = Lat<Q>;
  constexpr int D = LT::D;
  float d = 0, jx = 0, jy = 0, jz = 0, pxx = 0, pxy = 0, pxz = 0, pyy = 0, pyz = 0, pzz = 0;
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const float cx = LT::cx(i), cy = LT::cy(i), cz = LT::cz(i), v = fi(i);
    d += v;
    jx += cx * v;
    jy += cy * v;
    pxx += cx * cx * v;
    pxy += cx * cy * v;
    pyy += cy * cy * v;
    if (D == 3) {
      jz += cz * v;
      pxz += cx * cz * v;
      pyz += cy * cz * v;
      pzz += cz * cz * v;
    }
  }
  const float drho = d, inv = 1.0f / (1.0f + d);
  const float u[3] = {jx * inv, jy * inv, jz * inv};
  const float rho = 1.0f + drho, s = -1.5f * om / rho, iso = CS2 * drho;
  const long long NF = C.nfine;
  float *M = C.macro;
  M[fc] = drho;
  for (int a = 0; a < D; ++a) M[(1 + a) * NF + fc] = u[a];
  const float sxx = s * (pxx - iso - rho * u[0] * u[0]), sxy = s * (pxy - rho * u[0] * u[1]);
  const float syy = s * (pyy - iso - rho * u[1] * u[1]);
  if (D == 2) {
    M[3 * NF + fc] = sxx; M[4 * NF + fc] = sxy; M[5 * NF + fc] = syy;
  } else {
    M[4 * NF + fc] = sxx; M[5 * NF + fc] = sxy; M[6 * NF + fc] = s * (pxz - rho * u[0] * u[2]);
    M[7 * NF + fc] = syy; M[8 * NF + fc] = s * (pyz - rho * u[1] * u[2]);
    M[9 * NF + fc] = s * (pzz - iso - rho * u[2] * u[2]);
  }
}

// The cell's phase operator: BGK, or on D3Q27 the cumulant model where the level asks for it.
template <int Q>
__device__ __forceinline__ void collide_phase(float *f, float om, const float acc[3], float &drho, float u[3],
                                              bool cumulant) {
  if constexpr (Q == 27) {
    if (cumulant) {
      cumulant_collide27(f, om, acc, drho, u);
      return;
    }
  }
  lb_collide<Q>(f, om, acc, drho, u);
}

// ------------------------------------------------------------------ init
// Rest equilibrium with the hydrostatic density rho_hat = 1 - g.(x - x_ref)/c_s^2.
template <int Q, typename T>
__global__ void k_init(Ctx C, BlockShape S, const int *list, int nlist) {
  LSB_GRID_WAIT();
  using LT = Lat<Q>;
  for (int w = blockIdx.x; w < nlist; w += gridDim.x) {
    int gb = list[w];
    int x, y, z;
    const LevelDev &L = blk_cell(C, S, gb, threadIdx.x, x, y, z);
    if (x >= L.n[0] || y >= L.n[1] || z >= L.n[2]) continue;
    long long c = cidx(L, x, y, z);
    float xc[3] = {(x + 0.5f) * L.scale, (y + 0.5f) * L.scale, (z + 0.5f) * L.scale};
    float drho = 0.f;
    for (int a = 0; a < LT::D; ++a) drho -= L.grav[a] * (xc[a] - L.x_ref[a]) / CS2;
    if (C.tag[L.cell_off + c] & TAG_GAS) drho += L.p_gas0 / (L.rho_phys[1] * CS2);
    T *A = fA<T, Q>(C, L);
    float u0[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int i = 0; i < Q; ++i) Store<T>::st(A + i * L.ncell + c, feq_dev<Q>(i, drho, u0, 0.f), C.fp16_scale);
  }
}

// ------------------------------------------------------------------ collide + stream
#ifndef LSB_CS_MINB
#define LSB_CS_MINB 2  // CTAs of 512 threads per SM the register budget is sized for
#endif

// One CTA per block of the work list, one thread per cell.  Leaf cells and
// the covered cells a leaf streams from (TAG_RLAYER) collide and push.  On the
// finest level, band blocks also write the pre-collision moments and strain
// rate (input of the interface condition and the level-set velocity), and a
// push across the interface is parked in the link buffer for the post-pass.
// The neighbour offsets along each axis (-1, +1: plain, wrapped on periodic
// axes, or a wall) are formed once per cell, so every population's
// destination is one add and boundary cells take no divergent slow path.
template <int Q, typename T>
__global__ void __launch_bounds__(512, (Q == 27 ? 1 : LSB_CS_MINB)) k_collide_stream(Ctx C, BlockShape S,
                                                                     const int *__restrict__ list, int nlist) {
  LSB_GRID_WAIT();
  using LT = Lat<Q>;
  constexpr int D = LT::D;
  for (int w = blockIdx.x; w < nlist; w += gridDim.x) {
    const int gb = __ldg(list + w);
    const int4 bi = __ldg(C.blk_info + gb);
    const LevelDev &L = C.lds[bi.x];
    const int t = threadIdx.x;
    const int x = (bi.y << S.lg[0]) + (t & (S.bs[0] - 1));
    const int y = (bi.z << S.lg[1]) + ((t >> S.lg[0]) & (S.bs[1] - 1));
    const int z = (bi.w << S.lg[2]) + (t >> (S.lg[0] + S.lg[1]));
    const int n0 = L.n[0], n1 = L.n[1], n2 = L.n[2];
    if (x >= n0 || y >= n1 || z >= n2) continue;
    const unsigned p0 = (unsigned)L.p[0], p01 = (unsigned)(L.p[0] * L.p[1]);
    const unsigned c = x + p0 * y + p01 * z;
    const uint8_t tg = C.tag[L.cell_off + c];
    if (!(tg & (TAG_LEAF | TAG_RLAYER))) continue;
    const unsigned N = (unsigned)L.ncell;
    const T *__restrict__ A = fA<T, Q>(C, L);
    T *__restrict__ B = fB<T, Q>(C, L);
    const int ph = tg & TAG_GAS;
    const bool fine = L.finest != 0;
    if (fine && (tg & TAG_IFACE)) {  // before the populations are held in registers
      const T *A2;  // an opaque copy: these loads are not reused for f below
      asm("mov.b64 %0, %1;" : "=l"(A2) : "l"(A));
      store_iface_macro<Q>(C, L.fine_off + c, [&](int i) { return Store<T>::ld(A2 + (i * N + c), C.fp16_inv); },
                           L.omega[ph]);
    }
    float f[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) f[i] = Store<T>::ld(A + (i * N + c), C.fp16_inv);
    const float acc[3] = {L.acc[ph][0], L.acc[ph][1], L.acc[ph][2]};
    float drho, u[3];
    collide_phase<Q>(f, L.omega[ph], acc, drho, u, L.cumulant[ph]);
    // per-axis neighbour offsets and wall flags
    const bool wxm = x == 0 && !L.per[0], wxp = x == n0 - 1 && !L.per[0];
    const bool wym = y == 0 && !L.per[1], wyp = y == n1 - 1 && !L.per[1];
    const bool wzm = D == 3 && z == 0 && !L.per[2], wzp = D == 3 && z == n2 - 1 && !L.per[2];
    const int dxm = x > 0 ? -1 : n0 - 1, dxp = x < n0 - 1 ? 1 : 1 - n0;
    const int dym = y > 0 ? -(int)p0 : (n1 - 1) * (int)p0, dyp = y < n1 - 1 ? (int)p0 : (1 - n1) * (int)p0;
    const int dzm = z > 0 ? -(int)p01 : (n2 - 1) * (int)p01, dzp = z < n2 - 1 ? (int)p01 : (1 - n2) * (int)p01;
    uint32_t cm = 0;
    int cb = 0;
    if (fine && (tg & TAG_IFACE)) {
      cm = C.cmask[L.fine_off + c];
      cb = C.cbase[L.fine_off + c];
    }
    const bool ccut = !fine && (tg & TAG_CCUT);
    Store<T>::st(B + (LT::REST * N + c), f[LT::REST], C.fp16_scale);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      if (i == LT::REST) continue;
      const int cxi = LT::cx(i), cyi = LT::cy(i), czi = LT::cz(i);
      const int k = LT::opp(i);
      if (cm & (1u << k)) {  // x + c_i lies across the interface: park for the post-pass
        const long long li = cb + __popc(cm & ((1u << k) - 1u));
        if (li < C.link_cap) {
          C.linkbuf[2 * li] = f[i];
          C.linkbuf[2 * li + 1] = f[k];
        }
        continue;
      }
      const bool wx = (cxi < 0 && wxm) || (cxi > 0 && wxp);
      const bool wy = (cyi < 0 && wym) || (cyi > 0 && wyp);
      const bool wz = (czi < 0 && wzm) || (czi > 0 && wzp);
      if (!(wx || wy || wz)) {
        const int off = (cxi < 0 ? dxm : (cxi > 0 ? dxp : 0)) + (cyi < 0 ? dym : (cyi > 0 ? dyp : 0)) +
                        (czi < 0 ? dzm : (czi > 0 ? dzp : 0));
        const unsigned ct = (unsigned)((int)c + off);
        if (ccut) {  // coarser level, neighbour of the other phase: plain bounce-back
          const uint8_t tt = C.tag[L.cell_off + ct];
          if (!(tt & TAG_GHOST) && ((tt ^ tg) & TAG_GAS)) {
            Store<T>::st(B + (k * N + c), f[i], C.fp16_scale);
            continue;
          }
        }
        Store<T>::st(B + (i * N + ct), f[i], C.fp16_scale);
      } else {
        const bool nx = wx && !L.slip[0], ny = wy && !L.slip[1], nz = wz && !L.slip[2];
        if (__builtin_expect(nx || ny || nz, 1)) {
          // half-way bounce-back with the moving-wall term, i pointing at the (no-slip) wall
          const int face = nx ? (cxi < 0 ? 0 : 1) : (ny ? (cyi < 0 ? 2 : 3) : (czi < 0 ? 4 : 5));
          const float *uw = L.wall_u[face];
          const float du = cxi * uw[0] + cyi * uw[1] + czi * uw[2];
          Store<T>::st(B + (k * N + c), f[i] - 6.0f * LT::w(i) * du, C.fp16_scale);
        } else {
          // slip walls only: specular reflection, moved on along the other axes; into the
          // other phase (not a ghost cell) plain bounce-back
          const int off = (wx ? 0 : (cxi < 0 ? dxm : (cxi > 0 ? dxp : 0))) +
                          (wy ? 0 : (cyi < 0 ? dym : (cyi > 0 ? dyp : 0))) +
                          (wz ? 0 : (czi < 0 ? dzm : (czi > 0 ? dzp : 0)));
          const unsigned ct = (unsigned)((int)c + off);
          const uint8_t tt = C.tag[L.cell_off + ct];
          if (!(tt & TAG_GHOST) && ((tt ^ tg) & TAG_GAS))
            Store<T>::st(B + (k * N + c), f[i], C.fp16_scale);
          else
            Store<T>::st(B + (mirror_dir<Q>(i, (wx ? 1 : 0) | (wy ? 2 : 0) | (wz ? 4 : 0)) * N + ct), f[i],
                         C.fp16_scale);
        }
      }
    }
  }
}

// ------------------------------------------------------------------ collide + stream, TMA-staged
// Same update as k_collide_stream, with the A populations of each block
// brought into shared memory by one TMA tensor load (a box of
// bs0 x bs1 x bs2 cells x Q populations) into one of two stages.  When the
// level's cell tags have a tensor map too (block rows of whole 16-byte units),
// the block's tags come with the same stage, so no thread waits on a global
// load before its collision.  Persistent CTAs take blocks from the work list (in
// turn, or from a counter: see the kernel); one thread issues the loads.  A stage is released as soon as every thread has copied its
// populations into registers, and is refilled at once with the block after
// next, so two loads per CTA are in flight while it collides and pushes.  Every
// thread waits on the stage's mbarrier with an iteration limit; on expiry the
// error word gets ERR_TIMEOUT and the whole CTA stops after a bounded wait for
// its other load in flight.

template <typename T>
__device__ __forceinline__ float stage_ld(const T *p, float inv);
template <>
__device__ __forceinline__ float stage_ld<float>(const float *p, float) {
  return *p;
}
template <>
__device__ __forceinline__ float stage_ld<__half>(const __half *p, float inv) {
  return __half2float(*p) * inv;
}

// Per-block values the TMA-issuing thread publishes with each stage it fills, in the
// ring slot of the iteration that consumes the stage; the stage's mbarrier
// (arrive = release, wait = acquire) makes them visible.
struct BlockMeta {
  long long cell_off, fine_off;
  unsigned ncell, p0, p01;
  int gb, ld, level, x0, y0, z0, n0, n1, n2, finest, per[3], cum[2];
  float omega[2], acc[2][3];
};

template <int Q, typename T>
// work (optional): two counters, zero at launch.  Then thread 0 takes each next list
// index from work[0] instead of walking blockIdx.x + k gridDim.x, so that CTAs that become
// resident late (beside another kernel) take fewer blocks; the last CTA to finish
// (work[1]) sets both back to zero for the next launch.
__global__ void __launch_bounds__(512, 2) k_collide_stream_tma(Ctx C, BlockShape S, const int *__restrict__ list,
                                                               int nlist, const CUtensorMap *__restrict__ tmaps,
                                                               const CUtensorMap *__restrict__ tmaps_tag,
                                                               int *work) {
  LSB_GRID_WAIT();
  using LT = Lat<Q>;
  constexpr int D = LT::D;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bar[2];
  __shared__ BlockMeta meta[4];  // iteration it uses meta[it & 3]; two blocks are staged ahead
  const int nt = blockDim.x;
  const bool stag = tmaps_tag != nullptr;
  const unsigned stage_bytes = (unsigned)(Q * nt * sizeof(T));
  const unsigned tag_off = (stage_bytes + 127u) & ~127u;  // TMA destinations 128-byte aligned
  const unsigned stage_stride = (tag_off + nt + 127u) & ~127u;
  if (threadIdx.x == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  // thread 0: publish block w's metadata into meta[ms] and start its TMA load into stage st
  auto issue = [&](int w, int st, int ms) {
    const int gb = __ldg(list + w);
    const int4 bi = __ldg(C.blk_info + gb);
    const LevelDev &L = C.lds[bi.x];
    BlockMeta &m = meta[ms];
    m.gb = gb;
    m.ld = bi.x;
    m.level = L.level;
    m.x0 = bi.y << S.lg[0];
    m.y0 = bi.z << S.lg[1];
    m.z0 = bi.w << S.lg[2];
    m.n0 = L.n[0]; m.n1 = L.n[1]; m.n2 = L.n[2];
    m.p0 = (unsigned)L.p[0];
    m.p01 = (unsigned)(L.p[0] * L.p[1]);
    m.ncell = (unsigned)L.ncell;
    m.cell_off = L.cell_off;
    m.fine_off = L.fine_off;
    m.finest = L.finest;
    for (int a = 0; a < 3; ++a) m.per[a] = L.per[a];
    for (int k = 0; k < 2; ++k) {
      m.cum[k] = L.cumulant[k];
      m.omega[k] = L.omega[k];
      for (int a = 0; a < 3; ++a) m.acc[k][a] = L.acc[k][a];
    }
    const CUtensorMap *tm = tmaps + 2 * bi.x + C.par[L.level];
    T *dst = reinterpret_cast<T *>(smem_raw + st * stage_stride);
    mbar_expect_tx(&bar[st], stage_bytes + (stag ? (unsigned)nt : 0u));
    if (D == 3) tma_load_4d(dst, tm, m.x0, m.y0, m.z0, 0, &bar[st]);
    else tma_load_3d(dst, tm, m.x0, m.y0, 0, &bar[st]);
    if (stag) {
      unsigned char *tdst = smem_raw + st * stage_stride + tag_off;
      if (D == 3) tma_load_3d(tdst, tmaps_tag + bi.x, m.x0, m.y0, m.z0, &bar[st]);
      else tma_load_2d(tdst, tmaps_tag + bi.x, m.x0, m.y0, &bar[st]);
    }
  };
  const int G = gridDim.x;
  // the list index of this CTA's k-th block; meta[slot].gb = -1 marks an iteration with none
  auto take = [&](int k) { return work ? atomicAdd(work, 1) : (int)blockIdx.x + k * G; };
  // thread 0 takes each index one load ahead of its use (nextw), so that the counter's
  // round trip overlaps its block's collision instead of delaying the next load
  int nextw = nlist;
  auto issue_next = [&](int k, int st, int ms) {
    const int w = nextw;
    if (w < nlist) {
      issue(w, st, ms);
      nextw = take(k + 1);
    } else {
      meta[ms].gb = -1;
    }
  };
  if (threadIdx.x == 0) {
    nextw = take(0);
    issue_next(0, 0, 0);
    issue_next(1, 1, 1);
  }
  __syncthreads();
  // bounded wait for the load of iteration j (stage j & 1, its (j >> 1)-th use)
  auto wait_stage = [&](int j) {
    for (unsigned spins = 0; !mbar_try_wait(&bar[j & 1], (j >> 1) & 1);)
      if (++spins > kWaitLimit) return false;
    return true;
  };
  // the last CTA out resets the work counters (every CTA passes here once)
  auto finish = [&]() {
    if (work && threadIdx.x == 0 && atomicAdd(work + 1, 1) == (int)gridDim.x - 1) {
      work[0] = 0;
      work[1] = 0;
    }
  };
  for (int it = 0;; ++it) {
    // set by thread 0 two iterations ago, before a barrier every thread has passed since
    if (meta[it & 3].gb < 0) break;
    const int st = it & 1;
    const bool ok = wait_stage(it);
    const BlockMeta &m = meta[it & 3];
    const int t = threadIdx.x;
    const int x = m.x0 + (t & (S.bs[0] - 1));
    const int y = m.y0 + ((t >> S.lg[0]) & (S.bs[1] - 1));
    const int z = m.z0 + (t >> (S.lg[0] + S.lg[1]));
    const int n0 = m.n0, n1 = m.n1, n2 = m.n2;
    const unsigned p0 = m.p0, p01 = m.p01;
    const unsigned c = x + p0 * y + p01 * z;
    bool act = ok && x < n0 && y < n1 && z < n2;
    uint8_t tg = 0;
    if (act) {
      tg = stag ? smem_raw[st * stage_stride + tag_off + t] : C.tag[m.cell_off + c];
      act = (tg & (TAG_LEAF | TAG_RLAYER)) != 0;
    }
    const int ph = tg & TAG_GAS;
    const bool cut = act && m.finest && (tg & TAG_IFACE);
    float f[Q];
    if (act) {
      const T *sp = reinterpret_cast<const T *>(smem_raw + st * stage_stride);
      if (cut)  // before the populations are held in registers
        store_iface_macro<Q>(C, m.fine_off + c, [&](int i) { return stage_ld<T>(sp + i * nt + t, C.fp16_inv); },
                             m.omega[ph]);
#pragma unroll
      for (int i = 0; i < Q; ++i) f[i] = stage_ld<T>(sp + i * nt + t, C.fp16_inv);
    }
    // every thread holds its populations: stage st takes the block after next
    if (__syncthreads_or(!ok)) {  // a load never arrived: drain the other one in flight, stop
      if (t == 0) {
        atomicOr(C.err, ERR_TIMEOUT);
        if (meta[(it + 1) & 3].gb >= 0) wait_stage(it + 1);
      }
      finish();
      return;
    }
    if (t == 0) issue_next(it + 2, st, (it + 2) & 3);
    do {
      if (!act) break;

      const unsigned N = m.ncell;
      T *__restrict__ B = reinterpret_cast<T *>(C.buf[1 - C.par[m.level]]) + m.cell_off * Q;
      const float acc[3] = {m.acc[ph][0], m.acc[ph][1], m.acc[ph][2]};
      float drho, u[3];
      collide_phase<Q>(f, m.omega[ph], acc, drho, u, m.cum[ph]);
      const bool wxm = x == 0 && !m.per[0], wxp = x == n0 - 1 && !m.per[0];
      const bool wym = y == 0 && !m.per[1], wyp = y == n1 - 1 && !m.per[1];
      const bool wzm = D == 3 && z == 0 && !m.per[2], wzp = D == 3 && z == n2 - 1 && !m.per[2];
      const int dxm = x > 0 ? -1 : n0 - 1, dxp = x < n0 - 1 ? 1 : 1 - n0;
      const int dym = y > 0 ? -(int)p0 : (n1 - 1) * (int)p0, dyp = y < n1 - 1 ? (int)p0 : (1 - n1) * (int)p0;
      const int dzm = z > 0 ? -(int)p01 : (n2 - 1) * (int)p01, dzp = z < n2 - 1 ? (int)p01 : (1 - n2) * (int)p01;
      uint32_t cm = 0;
      int cb = 0;
      if (cut) {
        cm = C.cmask[m.fine_off + c];
        cb = C.cbase[m.fine_off + c];
      }
      Store<T>::st(B + (LT::REST * N + c), f[LT::REST], C.fp16_scale);
      // cells next to the other phase on a coarser level take a checking copy of the loop
      auto push = [&](auto check) {
        constexpr bool CHECK = decltype(check)::value;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
          if (i == LT::REST) continue;
          const int cxi = LT::cx(i), cyi = LT::cy(i), czi = LT::cz(i);
          const int k = LT::opp(i);
          if (cm & (1u << k)) {
            const long long li = cb + __popc(cm & ((1u << k) - 1u));
            if (li < C.link_cap) {
              C.linkbuf[2 * li] = f[i];
              C.linkbuf[2 * li + 1] = f[k];
            }
            continue;
          }
          const bool wx = (cxi < 0 && wxm) || (cxi > 0 && wxp);
          const bool wy = (cyi < 0 && wym) || (cyi > 0 && wyp);
          const bool wz = (czi < 0 && wzm) || (czi > 0 && wzp);
          if (!(wx || wy || wz)) {
            const int off = (cxi < 0 ? dxm : (cxi > 0 ? dxp : 0)) + (cyi < 0 ? dym : (cyi > 0 ? dyp : 0)) +
                            (czi < 0 ? dzm : (czi > 0 ? dzp : 0));
            const unsigned ct = (unsigned)((int)c + off);
            if constexpr (CHECK) {  // coarser level, neighbour of the other phase: plain bounce-back
              const uint8_t tt = C.tag[m.cell_off + ct];
              if (!(tt & TAG_GHOST) && ((tt ^ tg) & TAG_GAS)) {
                Store<T>::st(B + (k * N + c), f[i], C.fp16_scale);
                continue;
              }
            }
            Store<T>::st(B + (i * N + ct), f[i], C.fp16_scale);
          } else {
            const LevelDev &Ld = C.lds[m.ld];
            const bool nx = wx && !Ld.slip[0], ny = wy && !Ld.slip[1], nz = wz && !Ld.slip[2];
            if (nx || ny || nz) {  // no-slip: half-way bounce-back with the moving-wall term
              const int face = nx ? (cxi < 0 ? 0 : 1) : (ny ? (cyi < 0 ? 2 : 3) : (czi < 0 ? 4 : 5));
              const float *uw = Ld.wall_u[face];
              const float du = cxi * uw[0] + cyi * uw[1] + czi * uw[2];
              Store<T>::st(B + (k * N + c), f[i] - 6.0f * LT::w(i) * du, C.fp16_scale);
            } else {  // slip: specular reflection (into the other phase: plain bounce-back)
              const int off = (wx ? 0 : (cxi < 0 ? dxm : (cxi > 0 ? dxp : 0))) +
                              (wy ? 0 : (cyi < 0 ? dym : (cyi > 0 ? dyp : 0))) +
                              (wz ? 0 : (czi < 0 ? dzm : (czi > 0 ? dzp : 0)));
              const unsigned ct = (unsigned)((int)c + off);
              const uint8_t tt = C.tag[m.cell_off + ct];
              if (!(tt & TAG_GHOST) && ((tt ^ tg) & TAG_GAS))
                Store<T>::st(B + (k * N + c), f[i], C.fp16_scale);
              else
                Store<T>::st(B + (mirror_dir<Q>(i, (wx ? 1 : 0) | (wy ? 2 : 0) | (wz ? 4 : 0)) * N + ct), f[i],
                             C.fp16_scale);
            }
          }
        }
      };
      if (!m.finest && (tg & TAG_CCUT)) push(std::true_type{});
      else push(std::false_type{});
    } while (false);
  }
  finish();
}

// ------------------------------------------------------------------ interface post-pass
// For every cut link (x, k): Eq. bb with the momentum term of Eq. bb_cc;
// i = opp(k) points from x (phase A) to x + c_i (phase B).  One thread per link
// (the link list of the classification, in link-buffer order).
// On the CTAs [b0, b0 + nb) of the launch.
template <int Q, typename T>
__device__ __forceinline__ void d_interface_bc(const Ctx &C, int glevel, int b0, int nb) {
  using LT = Lat<Q>;
  constexpr int D = LT::D;
  const long long n = min((long long)C.counters[glevel * NCOUNT + 0], C.link_cap);
  for (long long e = ((long long)blockIdx.x - b0) * blockDim.x + threadIdx.x; e < n;
       e += (long long)nb * blockDim.x) {
    const int2 it = C.link_cell[C.link_list_off[glevel] + e];
    const int k = C.link_dir[C.link_list_off[glevel] + e];
    const LevelDev &L = C.lds[it.x];
    const long long c = it.y;
    int x, y, z;
    cell_xyz(L, c, x, y, z);
    const long long fo = L.fine_off;
    const long long NF = C.nfine;
    const uint8_t tg = C.tag[L.cell_off + c];
    const int A = tg & TAG_GAS;
    const int Bp = 1 - A;
    const long long N = L.ncell;
    T *Bf = fB<T, Q>(C, L);
    const float *M = C.macro;
    const float phx = C.phi[fo + c];
    const float rA = M[fo + c];
    float uA[3] = {0.f, 0.f, 0.f}, SA[6] = {0, 0, 0, 0, 0, 0}, nx[3] = {0.f, 0.f, 0.f};
    for (int a = 0; a < D; ++a) {
      uA[a] = M[(1 + a) * NF + fo + c];
      nx[a] = C.nvec[a * NF + fo + c];
    }
    const int MS = 1 + D;
    for (int s = 0; s < D * (D + 1) / 2; ++s) SA[s] = M[(MS + s) * NF + fo + c];
    const float kx = C.kappa[fo + c];
    const float etaA = L.eta[A], etaB = L.eta[Bp];
    const float eta_bar = 0.5f * (etaA + etaB);
    const float jeta = etaB - etaA;
    const float sgn = (A == 0) ? 1.0f : -1.0f;
    {
      const int i = LT::opp(k);
      const long long li = e;
      const float fi = C.linkbuf[2 * li], fk = C.linkbuf[2 * li + 1];
      int yx = x + LT::cx(i), yy = y + LT::cy(i), yz = z + LT::cz(i);
      wrap(L, 0, yx); wrap(L, 1, yy); if (D == 3) wrap(L, 2, yz);
      const long long cy_ = cidx(L, yx, yy, yz);
      const float phy = C.phi[fo + cy_];
      const float q = phx / (phx - phy);
      // u_I, n, kappa along the link; Sbar, [p], eta from the two nodes
      float uI[3], nv[3], Sb[6];
      float nn = 0.f;
      for (int a = 0; a < 3; ++a) { uI[a] = 0.f; nv[a] = 0.f; }
      for (int a = 0; a < D; ++a) {
        uI[a] = (1.0f - q) * uA[a] + q * M[(1 + a) * NF + fo + cy_];
        nv[a] = (1.0f - q) * nx[a] + q * C.nvec[a * NF + fo + cy_];
        nn += nv[a] * nv[a];
      }
      nn = sqrtf(nn);
      for (int a = 0; a < D; ++a) nv[a] = nn > 0.f ? sgn * nv[a] / nn : 0.f;
      const float kap = sgn * ((1.0f - q) * kx + q * C.kappa[fo + cy_]);
      for (int s = 0; s < D * (D + 1) / 2; ++s) Sb[s] = 0.5f * (SA[s] + M[(MS + s) * NF + fo + cy_]);
      const float rB = M[fo + cy_];
      const float jp = CS2 * (L.rho_phys[Bp] * rB - L.rho_phys[A] * rA);
      // symmetric tensor access
      auto Sget = [&](int a, int b) -> float {
        if (D == 2) return (a == 0 && b == 0) ? Sb[0] : ((a == 1 && b == 1) ? Sb[2] : Sb[1]);
        int lo = a < b ? a : b, hi = a < b ? b : a;
        if (lo == 0) return Sb[hi];            // xx, xy, xz
        if (lo == 1) return Sb[2 + hi];        // yy, yz
        return Sb[5];                          // zz
      };
      float v[3] = {0.f, 0.f, 0.f};
      float Snn = 0.f;
      for (int a = 0; a < D; ++a) {
        for (int b = 0; b < D; ++b) v[a] += Sget(a, b) * nv[b];
        Snn += nv[a] * v[a];
      }
      float vt[3], cn = 0.f, cvt = 0.f, cuI = 0.f;
      const float ci[3] = {(float)LT::cx(i), (float)LT::cy(i), (float)LT::cz(i)};
      for (int a = 0; a < D; ++a) {
        vt[a] = v[a] - Snn * nv[a];
        cn += ci[a] * nv[a];
        cvt += ci[a] * vt[a];
        cuI += ci[a] * uI[a];
      }
      const float alpha = (jp + L.sigma * kap) / (2.0f * eta_bar) - (jeta / eta_bar) * Snn;
      const float ccS = alpha * cn * cn - 2.0f * (jeta / eta_bar) * cn * cvt;
      const float df = -6.0f * LT::w(i) * (cuI - q * (1.0f - q) * ccS);
      // Bouzidi branches (linear); the q < 1/2 branch needs x - c_i in phase A
      float val;
      if (q >= 0.5f) {
        val = fi / (2.0f * q) + (2.0f * q - 1.0f) / (2.0f * q) * fk + df / (2.0f * q);
      } else {
        int bx = x - LT::cx(i), by = y - LT::cy(i), bz = z - LT::cz(i);
        bool ok = wrap(L, 0, bx) && wrap(L, 1, by) && (D == 2 || wrap(L, 2, bz));
        if (ok) {
          const long long cbk = cidx(L, bx, by, bz);
          const uint8_t tb = C.tag[L.cell_off + cbk];
          ok = (tb & TAG_LEAF) && ((tb & TAG_GAS) == A);
          if (ok) {
            const float fb = Store<T>::ld(Bf + i * N + c, C.fp16_inv);
            val = 2.0f * q * fi + (1.0f - 2.0f * q) * fb + df;
          }
        }
        if (!ok) val = fi + df;
      }
      Store<T>::st(Bf + k * N + c, val, C.fp16_scale);
    }
  }
}
template <int Q, typename T>
__global__ void LSB_LINK_LB k_interface_bc(Ctx C, int glevel) {
  LSB_GRID_WAIT();
  d_interface_bc<Q, T>(C, glevel, 0, gridDim.x);
}
// The interface pass and the interface cells' u~ (the level set's first pass) in one
// launch: neither reads what the other writes (the pass writes populations, u~ comes
// from the moments the collide stored), so CTAs [0, gi) take the interface cells (the
// longer chain per thread, so its CTAs are scheduled first) and the rest the cut links.
template <int Q, typename T>
__global__ void LSB_LINK_LB k_iface_init(Ctx C, int glevel, int gi) {
  LSB_GRID_WAIT();
  if ((int)blockIdx.x < gi) d_ext_init<Q>(C, glevel, 0, gi);
  else d_interface_bc<Q, T>(C, glevel, gi, (int)gridDim.x - gi);
}

// ------------------------------------------------------------------ level transfers
// f~ -> f~eq(rho, u) + fac * (f~ - f~eq)
template <int Q>
__device__ __forceinline__ void rescale_neq(float *f, float fac) {
  float drho, u[3];
  lb_moments<Q>(f, drho, u);
  float usq = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    float fe = feq_dev<Q>(i, drho, u, usq);
    f[i] = fe + fac * (f[i] - fe);
  }
}

// Covered coarse cells (TAG_RLAYER): mean of the 2^D children's pre-collision
// populations, f^neq scaled by 2 tau_c / tau_f.  mode 1 (regrid coarsening):
// every cell of the listed blocks.
template <int Q, typename T>
__global__ void k_restrict(Ctx C, BlockShape S, const int *list, int nlist, int all_cells) {
  LSB_GRID_WAIT();
  using LT = Lat<Q>;
  constexpr int D = LT::D;
  for (int w = blockIdx.x; w < nlist; w += gridDim.x) {
    int gb = list[w];
    int x, y, z;
    const LevelDev &L = blk_cell(C, S, gb, threadIdx.x, x, y, z);
    if (x >= L.n[0] || y >= L.n[1] || z >= L.n[2]) continue;
    long long c = cidx(L, x, y, z);
    uint8_t tg = C.tag[L.cell_off + c];
    if (!all_cells && !(tg & TAG_RLAYER)) continue;
    const LevelDev &F = C.lds[L.child_ld];
    const T *Af = fA<T, Q>(C, F);
    float f[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) f[i] = 0.f;
    const int nz = (D == 3) ? 2 : 1;
    for (int sz = 0; sz < nz; ++sz)
      for (int sy = 0; sy < 2; ++sy)
        for (int sx = 0; sx < 2; ++sx) {
          long long cf = cidx(F, 2 * x + sx, 2 * y + sy, D == 3 ? 2 * z + sz : 0);
#pragma unroll
          for (int i = 0; i < Q; ++i) f[i] += Store<T>::ld(Af + i * F.ncell + cf, C.fp16_inv);
        }
    const float inv = 1.0f / (float)(4 * nz);
#pragma unroll
    for (int i = 0; i < Q; ++i) f[i] *= inv;
    int ph = tg & TAG_GAS;
    rescale_neq<Q>(f, 2.0f * L.tau[ph] / F.tau[ph]);
    T *Ac = fA<T, Q>(C, L);
#pragma unroll
    for (int i = 0; i < Q; ++i) Store<T>::st(Ac + i * L.ncell + c, f[i], C.fp16_scale);
  }
}

// Linear interpolation of coarse populations at the centre of fine cell (x,y,z):
// central gradients where both coarse neighbours are leaves (TAG_LEAF), one-sided
// where only one is, none otherwise; theta blends the coarse state at t (A) and
// t+1 (B) for the second fine substep.
template <int Q, typename T>
__device__ __forceinline__ void interp_coarse(const Ctx &C, const LevelDev &Lc, int x, int y, int z,
                                              float theta, float *out) {
  using LT = Lat<Q>;
  constexpr int D = LT::D;
  const T *Ac = fA<T, Q>(C, Lc);
  const T *Bc = fB<T, Q>(C, Lc);
  const int P[3] = {x >> 1, y >> 1, D == 3 ? (z >> 1) : 0};
  // Q x cells of a level stay below 2^32 (checked at creation): 32-bit offsets
  const unsigned Nc = (unsigned)Lc.ncell;
  auto load = [&](unsigned cc, float *dst) {
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      float a = Store<T>::ld(Ac + (i * Nc + cc), C.fp16_inv);
      if (theta != 0.f) a = (1.0f - theta) * a + theta * Store<T>::ld(Bc + (i * Nc + cc), C.fp16_inv);
      dst[i] = a;
    }
  };
  const unsigned cp = (unsigned)cidx(Lc, P[0], P[1], P[2]);
  float fp[Q];
  load(cp, fp);
#pragma unroll
  for (int i = 0; i < Q; ++i) out[i] = fp[i];
  const int fcrd[3] = {x, y, z};
  for (int a = 0; a < D; ++a) {
    const float delta = ((fcrd[a] & 1) - 0.5f) * 0.5f;
    int up[3] = {P[0], P[1], P[2]}, dn[3] = {P[0], P[1], P[2]};
    up[a] += 1;
    dn[a] -= 1;
    bool upok = wrap(Lc, a, up[a]);
    bool dnok = wrap(Lc, a, dn[a]);
    unsigned cu = 0, cd = 0;
    if (upok) {
      cu = (unsigned)cidx(Lc, up[0], up[1], up[2]);
      upok = (C.tag[Lc.cell_off + cu] & TAG_LEAF) != 0;
    }
    if (dnok) {
      cd = (unsigned)cidx(Lc, dn[0], dn[1], dn[2]);
      dnok = (C.tag[Lc.cell_off + cd] & TAG_LEAF) != 0;
    }
    if (!upok && !dnok) continue;
    float fu[Q], fd[Q];
    if (upok) load(cu, fu);
    if (dnok) load(cd, fd);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      float g = (upok && dnok) ? 0.5f * (fu[i] - fd[i]) : (upok ? fu[i] - fp[i] : fp[i] - fd[i]);
      out[i] += delta * g;
    }
  }
}

// Regrid: fill every cell of the listed (newly active) fine blocks from the
// coarse level (interpolation + f^neq scaling, no collision).  The coarse
// TAG_LEAF must mark the cells that hold valid data (old or new leaves).
template <int Q, typename T>
__global__ void k_prolong(Ctx C, BlockShape S, const int *list, int nlist) {
  LSB_GRID_WAIT();
  using LT = Lat<Q>;
  constexpr int D = LT::D;
  for (int w = blockIdx.x; w < nlist; w += gridDim.x) {
    const int gb = list[w];
    int x, y, z;
    const LevelDev &F = blk_cell(C, S, gb, threadIdx.x, x, y, z);
    if (x >= F.n[0] || y >= F.n[1] || z >= F.n[2]) continue;
    const long long c = cidx(F, x, y, z);
    const LevelDev &Lc = C.lds[F.parent_ld];
    float f[Q];
    interp_coarse<Q, T>(C, Lc, x, y, z, 0.f, f);
    const long long cpar = cidx(Lc, x >> 1, y >> 1, D == 3 ? (z >> 1) : 0);
    const int ph = C.tag[Lc.cell_off + cpar] & TAG_GAS;
    rescale_neq<Q>(f, F.tau[ph] / (2.0f * Lc.tau[ph]));
    T *Af = fA<T, Q>(C, F);
#pragma unroll
    for (int i = 0; i < Q; ++i) Store<T>::st(Af + i * F.ncell + c, f[i], C.fp16_scale);
  }
}

// ------------------------------------------------------------------ tags from block status
// Per cell: phase from phi at the finest cell under the cell's lowest corner,
// TAG_LEAF / TAG_RLAYER / TAG_GHOST from the block statuses of the cell and of
// its lattice neighbours.  Finest-level interface bits are rebuilt by the
// classification that follows every regrid.
template <int Q>
__global__ void k_level_tags(Ctx C, BlockShape S, const int *list, int nlist) {
  LSB_GRID_WAIT();
  using LT = Lat<Q>;
  constexpr int D = LT::D;
  for (int w = blockIdx.x; w < nlist; w += gridDim.x) {
    const int gb = list[w];
    int x, y, z;
    const LevelDev &L = blk_cell(C, S, gb, threadIdx.x, x, y, z);
    if (x >= L.n[0] || y >= L.n[1] || z >= L.n[2]) continue;
    const long long c = cidx(L, x, y, z);
    const LevelDev &Fn = C.lds[L.fine_ld];
    const long long cf = cidx(Fn, x * L.scale, y * L.scale, z * L.scale);
    uint8_t tg = (C.phi[Fn.fine_off + cf] >= 0.0f) ? TAG_GAS : 0;
    const int8_t st = C.bstat[gb];
    bool near_leaf = false, ccut = false;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      if (i == LT::REST) continue;
      int tx = x + LT::cx(i), ty = y + LT::cy(i), tz = z + LT::cz(i);
      if (!(wrap(L, 0, tx) && wrap(L, 1, ty) && (D == 2 || wrap(L, 2, tz)))) continue;
      const int8_t sb = C.bstat[L.block_off + block_of(L, tx, ty, tz, S)];
      if (sb == BLK_LEAF) near_leaf = true;
      // coarser levels: a neighbour of the other phase that is not a ghost cell (the
      // inactive neighbours of leaves are their ghost ring; a covered cell's are active)
      if (!L.finest && sb != BLK_INACTIVE) {
        const long long ct = cidx(Fn, tx * L.scale, ty * L.scale, tz * L.scale);
        if ((C.phi[Fn.fine_off + ct] >= 0.0f) != ((tg & TAG_GAS) != 0)) ccut = true;
      }
    }
    if (st == BLK_LEAF) tg |= TAG_LEAF;
    if (st == BLK_REFINED && near_leaf) tg |= TAG_RLAYER;
    if (ccut && (tg & (TAG_LEAF | TAG_RLAYER))) tg |= TAG_CCUT;
    if (st == BLK_INACTIVE && near_leaf) tg |= TAG_GHOST;
    if (tg & TAG_GAS) tg |= TAG_PREVGAS;
    C.tag[L.cell_off + c] = tg;
  }
}

// ------------------------------------------------------------------ observables
// Per case, float64: mass of each phase, gas volume, leaf count, centroid and
// velocity of the gas (sharp Heaviside, Sec. 3.2), lengths in finest cells.
// Persistent CTAs accumulate in registers while the case stays the same, then
// reduce through warp shuffles and shared memory: one set of atomics per CTA
// and case run instead of one per warp and block.  eps > 0: gas volume, centroid
// and velocity weighted by the smoothed indicator H_eps of phi at the leaf's first
// finest child instead of the leaf's phase (masses stay phase sums).
//
// Per-thread partials are FP32 over the thread's few cells, FP64 from the warp sum on:
// cell volumes, counts and centroid terms are integer-valued (exact in FP32 while a
// thread's sums stay below 2^24); mass is kept as volume + vol * drho with the small
// second part summed apart.
template <int D>
struct ObsAcc {
  static constexpr int NV = 4 + 2 * D;
  float vol_l = 0.f, vol_g = 0.f, dm_l = 0.f, dm_g = 0.f, v[NV];
  int cur_case = -1;
  __device__ ObsAcc() {
    for (int k = 0; k < NV; ++k) v[k] = 0.f;
  }
  // one leaf cell with populations f
  template <int Q>
  __device__ __forceinline__ void cell(const Ctx &C, const LevelDev &L, int x, int y, int z, uint8_t tg,
                                       const float *f, float eps) {
    float drho, u[3];
    lb_moments<Q>(f, drho, u);
    float vol = 1.f;
    for (int a = 0; a < D; ++a) vol *= (float)L.scale;
    const int gas = tg & TAG_GAS;
    if (gas) {
      vol_g += vol;
      dm_g += vol * drho;
    } else {
      vol_l += vol;
      dm_l += vol * drho;
    }
    v[3] += 1.f;
    const bool finite = isfinite(drho) && isfinite(u[0]) && isfinite(u[1]) && isfinite(u[2]);
    if (!finite) atomicOr(C.err, ERR_NONFINITE);
    const float h = eps > 0.f ? smooth_h(C.phi[corner_phi_index(C, L, x, y, z)], eps) : (gas ? 1.f : 0.f);
    if (h != 0.f) {
      const float vh = vol * h;
      v[2] += vh;
      const int crd[3] = {x, y, z};
      for (int a = 0; a < D; ++a) {
        v[4 + a] += vh * ((float)crd[a] + 0.5f) * (float)L.scale;
        v[4 + D + a] += vh * u[a];
      }
    }
  }
  // the CTA's partials of case_id into out (every thread of the CTA calls this)
  __device__ void flush(double *out, int stride, int case_id, double (*red)[NV]) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    for (int k = 0; k < NV; ++k) {
      double s = k == 0 ? (double)vol_l + (double)dm_l : (k == 1 ? (double)vol_g + (double)dm_g : (double)v[k]);
      for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
      if (lane == 0) red[warp][k] = s;
      v[k] = 0.f;
    }
    vol_l = vol_g = dm_l = dm_g = 0.f;
    __syncthreads();
    if (threadIdx.x < NV) {
      double s = 0.0;
      for (int w = 0; w < nw; ++w) s += red[w][threadIdx.x];
      if (s != 0.0) atomicAdd(out + (long long)case_id * stride + threadIdx.x, s);
    }
    __syncthreads();
  }
  // called with each block's case before its cells (uniform over the CTA)
  __device__ __forceinline__ void enter(double *out, int stride, int case_id, double (*red)[NV]) {
    if (case_id != cur_case) {
      if (cur_case >= 0) flush(out, stride, cur_case, red);
      cur_case = case_id;
    }
  }
  __device__ __forceinline__ void finish(double *out, int stride, double (*red)[NV]) {
    if (cur_case >= 0) flush(out, stride, cur_case, red);
  }
};

template <int Q, typename T>
__global__ void __launch_bounds__(512, LSB_OBS_MINB) k_observables(Ctx C, BlockShape S, const int *list, int nlist,
                                                                   double *out, int stride, float eps) {
  LSB_GRID_WAIT();
  constexpr int D = Lat<Q>::D;
  __shared__ double red[32][ObsAcc<D>::NV];
  ObsAcc<D> acc;
  // the next block's list entry and coordinates are loaded while this one is summed
  int4 next = blockIdx.x < nlist ? __ldg(C.blk_info + __ldg(list + blockIdx.x)) : make_int4(0, 0, 0, 0);
  for (int w = blockIdx.x; w < nlist; w += gridDim.x) {
    const int4 bi = next;
    if (w + gridDim.x < nlist) next = __ldg(C.blk_info + __ldg(list + w + gridDim.x));
    const LevelDev &L = C.lds[bi.x];
    acc.enter(out, stride, L.case_id, red);
    const int x = (bi.y << S.lg[0]) + (threadIdx.x & (S.bs[0] - 1));
    const int y = (bi.z << S.lg[1]) + ((threadIdx.x >> S.lg[0]) & (S.bs[1] - 1));
    const int z = (bi.w << S.lg[2]) + (threadIdx.x >> (S.lg[0] + S.lg[1]));
    if (x < L.n[0] && y < L.n[1] && z < L.n[2]) {
      const unsigned c = (unsigned)cidx(L, x, y, z);
      // the populations are loaded beside the cell's tag (every cell of a listed block
      // holds them), so the two loads do not wait on each other
      const uint8_t tg = C.tag[L.cell_off + c];
      const T *A = fA<T, Q>(C, L);
      const unsigned N = (unsigned)L.ncell;
      float f[Q];
#pragma unroll
      for (int i = 0; i < Q; ++i) f[i] = Store<T>::ld(A + (i * N + c), C.fp16_inv);
      if (tg & TAG_LEAF) acc.template cell<Q>(C, L, x, y, z, tg, f, eps);
    }
  }
  acc.finish(out, stride, red);
}

// The same sums with each block's populations (and tags) brought into shared memory
// by one TMA load, two stages per CTA as in the TMA-staged collide-and-stream: a
// block's Q population planes arrive in one bulk copy instead of Q loads per thread,
// so the pass streams at the copy rate instead of waiting on the loads each thread
// keeps in flight.  The stage is refilled once every thread holds its populations;
// waits are bounded (ERR_TIMEOUT, then a bounded wait for the other load in flight).
struct ObsMeta {
  int ld, x0, y0, z0;
};
template <int Q, typename T>
__global__ void __launch_bounds__(512, 2) k_observables_tma(Ctx C, BlockShape S, const int *__restrict__ list,
                                                            int nlist, double *out, int stride, float eps,
                                                            const CUtensorMap *__restrict__ tmaps,
                                                            const CUtensorMap *__restrict__ tmaps_tag) {
  LSB_GRID_WAIT();
  constexpr int D = Lat<Q>::D;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bar[2];
  __shared__ ObsMeta meta[4];  // iteration it uses meta[it & 3]; two blocks are staged ahead
  __shared__ double red[32][ObsAcc<D>::NV];
  const int nt = blockDim.x;
  const bool stag = tmaps_tag != nullptr;
  const unsigned stage_bytes = (unsigned)(Q * nt * sizeof(T));
  const unsigned tag_off = (stage_bytes + 127u) & ~127u;
  const unsigned stage_stride = (tag_off + nt + 127u) & ~127u;
  if (threadIdx.x == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  // the issuing thread holds the coordinates of the next block it will load, fetched one
  // load ahead, so an issue waits on no list lookup
  int4 pre = make_int4(0, 0, 0, 0);
  auto fetch = [&](int w) {
    if (w < nlist) pre = __ldg(C.blk_info + __ldg(list + w));
  };
  auto issue = [&](int st, int ms) {
    const int4 bi = pre;
    const LevelDev &L = C.lds[bi.x];
    ObsMeta &m = meta[ms];
    m.ld = bi.x;
    m.x0 = bi.y << S.lg[0];
    m.y0 = bi.z << S.lg[1];
    m.z0 = bi.w << S.lg[2];
    const CUtensorMap *tm = tmaps + 2 * bi.x + C.par[L.level];
    mbar_expect_tx(&bar[st], stage_bytes + (stag ? (unsigned)nt : 0u));
    T *dst = reinterpret_cast<T *>(smem_raw + st * stage_stride);
    if (D == 3) tma_load_4d(dst, tm, m.x0, m.y0, m.z0, 0, &bar[st]);
    else tma_load_3d(dst, tm, m.x0, m.y0, 0, &bar[st]);
    if (stag) {
      unsigned char *tdst = smem_raw + st * stage_stride + tag_off;
      if (D == 3) tma_load_3d(tdst, tmaps_tag + bi.x, m.x0, m.y0, m.z0, &bar[st]);
      else tma_load_2d(tdst, tmaps_tag + bi.x, m.x0, m.y0, &bar[st]);
    }
  };
  const int G = gridDim.x;
  if (threadIdx.x == 0) {
    fetch(blockIdx.x);
    if ((int)blockIdx.x < nlist) issue(0, 0);
    fetch(blockIdx.x + G);
    if ((int)blockIdx.x + G < nlist) issue(1, 1);
    fetch(blockIdx.x + 2 * G);
  }
  auto wait_stage = [&](int j) {
    for (unsigned spins = 0; !mbar_try_wait(&bar[j & 1], (j >> 1) & 1);)
      if (++spins > kWaitLimit) return false;
    return true;
  };
  ObsAcc<D> acc;
  int it = 0;
  for (int w = blockIdx.x; w < nlist; w += G, ++it) {
    const int st = it & 1;
    const bool ok = wait_stage(it);
    const ObsMeta m = meta[it & 3];
    const LevelDev &L = C.lds[m.ld];
    const int t = threadIdx.x;
    const int x = m.x0 + (t & (S.bs[0] - 1));
    const int y = m.y0 + ((t >> S.lg[0]) & (S.bs[1] - 1));
    const int z = m.z0 + (t >> (S.lg[0] + S.lg[1]));
    bool act = ok && x < L.n[0] && y < L.n[1] && z < L.n[2];
    uint8_t tg = 0;
    if (act) {
      tg = stag ? smem_raw[st * stage_stride + tag_off + t] : C.tag[L.cell_off + cidx(L, x, y, z)];
      act = (tg & TAG_LEAF) != 0;
    }
    float f[Q];
    if (act) {
      const T *sp = reinterpret_cast<const T *>(smem_raw + st * stage_stride);
#pragma unroll
      for (int i = 0; i < Q; ++i) f[i] = stage_ld<T>(sp + i * nt + t, C.fp16_inv);
    }
    if (__syncthreads_or(!ok)) {  // a load never arrived: drain the other one in flight, stop
      if (t == 0) {
        atomicOr(C.err, ERR_TIMEOUT);
        if (w + G < nlist) wait_stage(it + 1);
      }
      return;
    }
    if (t == 0 && w + 2 * G < nlist) {
      issue(st, (it + 2) & 3);
      fetch(w + 3 * G);
    }
    acc.enter(out, stride, L.case_id, red);
    if (act) acc.template cell<Q>(C, L, x, y, z, tg, f, eps);
  }
  acc.finish(out, stride, red);
}

// ------------------------------------------------------------------ field export
// Dense copy of one level: populations (full f = f~ + w), rho_hat, u.
template <int Q, typename T>
__global__ void k_export(Ctx C, int ld, int field, float *dst) {
  LSB_GRID_WAIT();
  using LT = Lat<Q>;
  const LevelDev &L = C.lds[ld];
  const long long ntrue = (long long)L.n[0] * L.n[1] * L.n[2];
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < ntrue;
       e += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(e % L.n[0]);
    const int y = (int)((e / L.n[0]) % L.n[1]);
    const int z = (int)(e / ((long long)L.n[0] * L.n[1]));
    const long long c = cidx(L, x, y, z);
    const T *A = fA<T, Q>(C, L);
    float f[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) f[i] = Store<T>::ld(A + i * L.ncell + c, C.fp16_inv);
    if (field == 4) {
#pragma unroll
      for (int i = 0; i < Q; ++i) dst[i * ntrue + e] = f[i] + LT::w(i);
    } else {
      float drho, u[3];
      lb_moments<Q>(f, drho, u);
      if (field == 0) dst[e] = 1.0f + drho;
      else
        for (int a = 0; a < LT::D; ++a) dst[a * ntrue + e] = u[a];
    }
  }
}

// ------------------------------------------------------------------ compact cell lists
// Append (ld, cell) of every cell of the listed blocks whose tag has any bit of
// `bits` (ghost ring or restriction layer), so that the level transfers run
// one thread per cell instead of one CTA per mostly idle block.
__global__ void k_collect(Ctx C, BlockShape S, const int *list, int nlist, int bits, int2 *out, int *count,
                          int cap) {
  LSB_GRID_WAIT();
  for (int w = blockIdx.x; w < nlist; w += gridDim.x) {
    const int gb = list[w];
    int x, y, z;
    const LevelDev &L = blk_cell(C, S, gb, threadIdx.x, x, y, z);
    if (x >= L.n[0] || y >= L.n[1] || z >= L.n[2]) continue;
    const long long c = cidx(L, x, y, z);
    if (!(C.tag[L.cell_off + c] & bits)) continue;
    const int e = atomicAdd(count, 1);
    if (e < cap) out[e] = make_int2(C.blk_ld[gb], (int)c);
    else atomicOr(C.err, ERR_LIST_OVF);
  }
}

// Restriction layer from a cell list (one thread per covered cell).
template <int Q, typename T>
__global__ void k_restrict_cells(Ctx C, const int2 *cells, int n) {
  LSB_GRID_WAIT();
  constexpr int D = Lat<Q>::D;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
    const int2 it = cells[e];
    const LevelDev &L = C.lds[it.x];
    const long long c = it.y;
    int x, y, z;
    cell_xyz(L, c, x, y, z);
    const LevelDev &F = C.lds[L.child_ld];
    const T *Af = fA<T, Q>(C, F);
    float f[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) f[i] = 0.f;
    const int nz = (D == 3) ? 2 : 1;
    for (int sz = 0; sz < nz; ++sz)
      for (int sy = 0; sy < 2; ++sy)
        for (int sx = 0; sx < 2; ++sx) {
          const long long cf = cidx(F, 2 * x + sx, 2 * y + sy, D == 3 ? 2 * z + sz : 0);
#pragma unroll
          for (int i = 0; i < Q; ++i) f[i] += Store<T>::ld(Af + i * F.ncell + cf, C.fp16_inv);
        }
    const float inv = 1.0f / (float)(4 * nz);
#pragma unroll
    for (int i = 0; i < Q; ++i) f[i] *= inv;
    const int ph = C.tag[L.cell_off + c] & TAG_GAS;
    rescale_neq<Q>(f, 2.0f * L.tau[ph] / F.tau[ph]);
    T *Ac = fA<T, Q>(C, L);
#pragma unroll
    for (int i = 0; i < Q; ++i) Store<T>::st(Ac + i * L.ncell + c, f[i], C.fp16_scale);
  }
}

// Ghost ring of level F (TAG_GHOST cells), one thread per listed cell: coarse
// interpolation at time weight theta, f^neq scaled by tau_f / (2 tau_c), a
// fine-level collision, pushed into the fine leaves that stream from it.
template <int Q, typename T>
__global__ void LSB_GHOST_LB k_ghost_cells(Ctx C, const int2 *cells, int n, float theta) {
  LSB_GRID_WAIT();
  using LT = Lat<Q>;
  constexpr int D = LT::D;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
    const int2 it = cells[e];
    const LevelDev &F = C.lds[it.x];
    const long long c = it.y;
    int x, y, z;
    cell_xyz(F, c, x, y, z);
    const LevelDev &Lc = C.lds[F.parent_ld];
    float f[Q];
    interp_coarse<Q, T>(C, Lc, x, y, z, theta, f);
    const long long cpar = cidx(Lc, x >> 1, y >> 1, D == 3 ? (z >> 1) : 0);
    const int ph = C.tag[Lc.cell_off + cpar] & TAG_GAS;
    rescale_neq<Q>(f, F.tau[ph] / (2.0f * Lc.tau[ph]));
    float drho, u[3];
    const float acc[3] = {F.acc[ph][0], F.acc[ph][1], F.acc[ph][2]};
    collide_phase<Q>(f, F.omega[ph], acc, drho, u, F.cumulant[ph]);
    T *Bf = fB<T, Q>(C, F);
    const unsigned N = (unsigned)F.ncell;
    const uint8_t *tagF = C.tag + F.cell_off;
    if (x > 0 && x + 1 < F.n[0] && y > 0 && y + 1 < F.n[1] && (D == 2 || (z > 0 && z + 1 < F.n[2]))) {
      // away from the box faces every target is c + c_i
      const int p0 = F.p[0], p01 = F.p[0] * F.p[1];
#pragma unroll
      for (int i = 0; i < Q; ++i) {
        if (i == LT::REST) continue;
        const unsigned ct = (unsigned)((int)c + LT::cx(i) + LT::cy(i) * p0 + LT::cz(i) * p01);
        if (tagF[ct] & TAG_LEAF) Store<T>::st(Bf + (i * N + ct), f[i], C.fp16_scale);
      }
      continue;
    }
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      if (i == LT::REST) continue;
      // through a slip wall the population comes back mirrored, moved on tangentially
      int t[3] = {x + LT::cx(i), y + LT::cy(i), z + LT::cz(i)};
      const int o[3] = {x, y, z};
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
      if (C.tag[F.cell_off + ct] & TAG_LEAF)
        Store<T>::st(Bf + mirror_dir<Q>(i, mm) * F.ncell + ct, f[i], C.fp16_scale);
    }
  }
}

// ------------------------------------------------------------------ restriction, one warp per cell
// The restriction update with the populations of one covered cell spread over the
// lanes of a group (population i on lane i; 16 lanes per cell on D2Q9, 32 on
// D3Q19): the 2^D children's loads of every lane are independent and in flight
// together instead of one thread walking Q x 2^D loads; the moments are summed
// over the group with shuffles.  (The ghost ring keeps one thread per cell: there
// neighbouring cells share their coarse sources, and loads coalesced over cells
// measured 2.4x faster than this layout.)
template <int Q>
struct GroupLanes {
  static constexpr int LPC = Q <= 16 ? 16 : 32;  // lanes per cell
  static constexpr int GPW = 32 / LPC;           // cells per warp
};
template <int Q>
__device__ __forceinline__ float group_sum(float v) {
#pragma unroll
  for (int o = GroupLanes<Q>::LPC / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
// drho and u of the group's populations (lanes past Q hold zero).
template <int Q>
__device__ __forceinline__ void group_moments(float f, int cxi, int cyi, int czi, float &drho, float u[3]) {
  const float d = group_sum<Q>(f), jx = group_sum<Q>(cxi * f), jy = group_sum<Q>(cyi * f);
  const float jz = Lat<Q>::D == 3 ? group_sum<Q>(czi * f) : 0.f;
  const float inv = 1.0f / (1.0f + d);
  drho = d;
  u[0] = jx * inv;
  u[1] = jy * inv;
  u[2] = jz * inv;
}
// Eq. feq deviation of one population, given its velocity and weight.
__device__ __forceinline__ float feq_lane(float wi, int cxi, int cyi, int czi, float drho, const float u[3]) {
  const float cu = cxi * u[0] + cyi * u[1] + czi * u[2];
  const float usq = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
  return wi * (drho + (1.0f + drho) * (3.0f * cu + 4.5f * cu * cu - 1.5f * usq));
}

template <int Q, typename T>
__global__ void k_restrict_cells_w(Ctx C, const int2 *cells, int n) {
  LSB_GRID_WAIT();
  using LT = Lat<Q>;
  constexpr int D = LT::D, LPC = GroupLanes<Q>::LPC, GPW = GroupLanes<Q>::GPW;
  const int lane = threadIdx.x & 31, sub = lane & (LPC - 1);
  const bool act = sub < Q;
  const int i = act ? sub : LT::REST;
  const int cxi = LT::cx(i), cyi = LT::cy(i), czi = LT::cz(i);
  const float wi = LT::w(i);
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int e0 = warp * GPW; e0 < n; e0 += nwarps * GPW) {
    const int e = min(e0 + lane / LPC, n - 1);  // a group past the end repeats the last cell and stores nothing
    const bool store = act && e0 + lane / LPC < n;
    const int2 it = cells[e];
    const LevelDev &L = C.lds[it.x];
    const unsigned c = (unsigned)it.y, p0 = (unsigned)L.p[0], p1 = (unsigned)L.p[1];
    const int x = (int)(c % p0), y = (int)((c / p0) % p1), z = (int)(c / (p0 * p1));
    const LevelDev &F = C.lds[L.child_ld];
    const T *Af = fA<T, Q>(C, F) + (size_t)i * F.ncell;
    const unsigned fp0 = (unsigned)F.p[0], fp01 = (unsigned)(F.p[0] * F.p[1]);
    const unsigned cf0 = 2u * x + fp0 * (2u * y) + (D == 3 ? fp01 * (2u * z) : 0u);
    float f = 0.f;
#pragma unroll
    for (int k = 0; k < (D == 3 ? 8 : 4); ++k)
      f += Store<T>::ld(Af + (cf0 + (k & 1) + ((k >> 1) & 1) * fp0 + ((k >> 2) & 1) * fp01), C.fp16_inv);
    f = act ? f * (1.0f / (float)(D == 3 ? 8 : 4)) : 0.f;
    const int ph = C.tag[L.cell_off + c] & TAG_GAS;
    float drho, u[3];
    group_moments<Q>(f, cxi, cyi, czi, drho, u);
    const float fe = feq_lane(wi, cxi, cyi, czi, drho, u);
    f = fe + (2.0f * L.tau[ph] / F.tau[ph]) * (f - fe);
    if (store) Store<T>::st(fA<T, Q>(C, L) + (size_t)i * L.ncell + c, f, C.fp16_scale);
  }
}

// ------------------------------------------------------------------ allocation-free export staging
// Fixed staging area for lsb_get_fields_noalloc: a file-scope device array, so
// callers that must not allocate device memory can still export fields.  Every
// GPU that loads the library holds it until the process exits.  In host code
// the name below is only a stand-in; its device address comes from
// cudaGetSymbolAddress, resolved once per device (with that device current).
static __device__ __align__(256) float g_export_scratch[kNoAllocFloats];

cudaError_t noalloc_scratch(float **ptr) {
  static std::mutex mu;
  static float *addr[kMaxDevices] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(mu);
  if (!addr[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_export_scratch);
    if (e != cudaSuccess) return e;
    addr[dev] = static_cast<float *>(p);
  }
  *ptr = addr[dev];
  return cudaSuccess;
}

// ------------------------------------------------------------------ host launchers
#define LSB_QT(Q, st, CALL)                                      \
  do {                                                           \
    if (Q == 9) {                                                \
      if (st == 0) { constexpr int Q_ = 9; using T_ = float; CALL; } \
      else { constexpr int Q_ = 9; using T_ = __half; CALL; }    \
    } else if (Q == 19) {                                        \
      if (st == 0) { constexpr int Q_ = 19; using T_ = float; CALL; } \
      else { constexpr int Q_ = 19; using T_ = __half; CALL; }   \
    } else if (st == 0) { /* D3Q27: FP32 storage only */        \
      constexpr int Q_ = 27; using T_ = float; CALL;             \
    } else {                                                     \
      return cudaErrorInvalidValue;                              \
    }                                                            \
    return cudaGetLastError();                                   \
  } while (0)

#define LK(kern) launcher(kern<Q_, T_>, L, 0)

cudaError_t run_init(int Q, int st, Launch L, Ctx C, BlockShape S, const int *list, int n) {
  LSB_QT(Q, st, (LK(k_init)(C, S, list, n)));
}
cudaError_t run_collide_stream(int Q, int st, Launch L, Ctx C, BlockShape S, const int *list, int n) {
  LSB_QT(Q, st, (LK(k_collide_stream)(C, S, list, n)));
}
// Dynamic shared memory of the TMA-staged kernel: two stages of Q x block cells.
size_t tma_smem_bytes(int Q, int st, int nthreads) {
  const size_t stage = ((size_t)Q * nthreads * (st == 0 ? 4 : 2) + 127) & ~size_t(127);
  return 2 * ((stage + nthreads + 127) & ~size_t(127));  // populations, then the block's tags
}
// Raise the kernel's dynamic shared-memory limit (once, outside any capture) and
// report how many CTAs of nthreads fit on one SM.
cudaError_t prepare_collide_stream_tma(int Q, int st, int nthreads, int *ctas_per_sm) {
  const size_t smem = tma_smem_bytes(Q, st, nthreads);
  cudaError_t e = cudaSuccess;
  int nb = 0;
  auto prep = [&](auto kern) {
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, nthreads, smem);
  };
  if (Q == 9) st == 0 ? prep(k_collide_stream_tma<9, float>) : prep(k_collide_stream_tma<9, __half>);
  else if (Q == 19) st == 0 ? prep(k_collide_stream_tma<19, float>) : prep(k_collide_stream_tma<19, __half>);
  else if (st == 0) prep(k_collide_stream_tma<27, float>);
  else e = cudaErrorInvalidValue;  // D3Q27: FP32 storage only
  *ctas_per_sm = nb;
  return e;
}
cudaError_t run_collide_stream_tma(int Q, int st, Launch L, Ctx C, BlockShape S, const int *list, int n,
                                   const CUtensorMap *tmaps, const CUtensorMap *tmaps_tag, int *work) {
  const size_t smem = tma_smem_bytes(Q, st, L.block);
  LSB_QT(Q, st,
         (launcher(k_collide_stream_tma<Q_, T_>, L, smem)(C, S, list, n, tmaps, tmaps_tag, work)));
}
cudaError_t run_interface_bc(int Q, int st, Launch L, Ctx C, int glevel) {
  LSB_QT(Q, st, (LK(k_interface_bc)(C, glevel)));
}
cudaError_t run_iface_init(int Q, int st, Launch L, Ctx C, int glevel, int gi) {
  LSB_QT(Q, st, (LK(k_iface_init)(C, glevel, gi)));
}
cudaError_t run_restrict(int Q, int st, Launch L, Ctx C, BlockShape S, const int *list, int n, int all_cells) {
  LSB_QT(Q, st, (LK(k_restrict)(C, S, list, n, all_cells)));
}
cudaError_t run_prolong(int Q, int st, Launch L, Ctx C, BlockShape S, const int *list, int n) {
  LSB_QT(Q, st, (LK(k_prolong)(C, S, list, n)));
}
cudaError_t run_observables(int Q, int st, Launch L, Ctx C, BlockShape S, const int *list, int n, double *out,
                            int stride, float eps, const CUtensorMap *tmaps, const CUtensorMap *tmaps_tag) {
  if (tmaps) {
    const size_t smem = tma_smem_bytes(Q, st, L.block);
    LSB_QT(Q, st,
           (launcher(k_observables_tma<Q_, T_>, L, smem)(C, S, list, n, out, stride, eps, tmaps, tmaps_tag)));
  }
  LSB_QT(Q, st, (LK(k_observables)(C, S, list, n, out, stride, eps)));
}
// Raise the TMA-staged observables kernel's dynamic shared-memory limit (once, outside
// any capture) and report how many CTAs of nthreads fit on one SM.
cudaError_t prepare_observables_tma(int Q, int st, int nthreads, int *ctas_per_sm) {
  const size_t smem = tma_smem_bytes(Q, st, nthreads);
  cudaError_t e = cudaSuccess;
  int nb = 0;
  auto prep = [&](auto kern) {
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, nthreads, smem);
  };
  if (Q == 9) st == 0 ? prep(k_observables_tma<9, float>) : prep(k_observables_tma<9, __half>);
  else if (Q == 19) st == 0 ? prep(k_observables_tma<19, float>) : prep(k_observables_tma<19, __half>);
  else if (st == 0) prep(k_observables_tma<27, float>);
  else e = cudaErrorInvalidValue;
  *ctas_per_sm = nb;
  return e;
}
cudaError_t run_export(int Q, int st, Launch L, Ctx C, int ld, int field, float *dst) {
  LSB_QT(Q, st, (LK(k_export)(C, ld, field, dst)));
}
cudaError_t run_export_noalloc(int Q, int st, Launch L, Ctx C, int ld, int field, float **staged) {
  float *dst = nullptr;
  cudaError_t e = noalloc_scratch(&dst);
  if (e != cudaSuccess) return e;
  *staged = dst;
  LSB_QT(Q, st, (LK(k_export)(C, ld, field, dst)));
}
cudaError_t run_collect(Launch L, Ctx C, BlockShape S, const int *list, int n, int bits, int2 *out, int *count,
                        int cap) {
  launcher(k_collect, L, 0)(C, S, list, n, bits, out, count, cap);
  return cudaGetLastError();
}
// One warp per GPW cells for the lattices with a group kernel (D2Q9, D3Q19); D3Q27 keeps
// one thread per cell on the grid it was given.
Launch group_launch(Launch L, int Q, int n) {
  const int gpw = Q <= 16 ? 2 : 1;
  const long long threads = (long long)((n + gpw - 1) / gpw) * 32;
  L.block = 128;
  L.grid = (int)std::max(1LL, (threads + 127) / 128);
  return L;
}
#define LSB_GROUP_Q(Q, st, KERN, ...)                                                              \
  do {                                                                                             \
    L = group_launch(L, Q, n);                                                                     \
    if (Q == 9) {                                                                                  \
      if (st == 0) launcher(KERN<9, float>, L, 0)(__VA_ARGS__);                \
      else launcher(KERN<9, __half>, L, 0)(__VA_ARGS__);                       \
    } else {                                                                                       \
      if (st == 0) launcher(KERN<19, float>, L, 0)(__VA_ARGS__);               \
      else launcher(KERN<19, __half>, L, 0)(__VA_ARGS__);                      \
    }                                                                                              \
    return cudaGetLastError();                                                                     \
  } while (0)
cudaError_t run_restrict_cells(int Q, int st, Launch L, Ctx C, const int2 *cells, int n) {
  if (Q == 27) LSB_QT(Q, st, (LK(k_restrict_cells)(C, cells, n)));
  LSB_GROUP_Q(Q, st, k_restrict_cells_w, C, cells, n);
}
cudaError_t run_ghost_cells(int Q, int st, Launch L, Ctx C, const int2 *cells, int n, float theta) {
  LSB_QT(Q, st, (LK(k_ghost_cells)(C, cells, n, theta)));
}
cudaError_t run_level_tags(int Q, Launch L, Ctx C, BlockShape S, const int *list, int n) {
  if (Q == 9) launcher(k_level_tags<9>, L, 0)(C, S, list, n);
  else if (Q == 19) launcher(k_level_tags<19>, L, 0)(C, S, list, n);
  else launcher(k_level_tags<27>, L, 0)(C, S, list, n);
  return cudaGetLastError();
}

}  // namespace lsb
