// Level-set kernels on the finest level (Sec. 2.2): phase classification and
// cut links (Sec. 2.3 radiation theorem), the narrow band, float64
// least-squares geometry, hyperbolic velocity extension (Eq.
// hyperbolicExtension), upwind-5 / TVD-RK3 transport, constrained
// reinitialisation (HJ-WENO5 Godunov, interface cells frozen), refill of cells
// that change phase (Sec. 2.4) and the refinement sensor (Sec. 2.6, 3.2.2).
//
// The narrow band is block granular: finest-level blocks holding an interface
// cell and their 3^D neighbours (active blocks only).  phi, the RK stage
// arrays and the extension velocity are dense finest-level arrays; stencil
// points outside the band read the committed fields.
#include <cooperative_groups.h>

#include <map>
#include <mutex>

#include "lsb_kernels.h"

namespace lsb {

__device__ __forceinline__ bool in_band(const Ctx &C, const LevelDev &L, const BlockShape &S, int x, int y, int z) {
  return (C.bflag[L.block_off + block_of(L, x, y, z, S)] & BF_BAND) != 0;
}

// ------------------------------------------------------------------ classification
// Pass 1: phase of every leaf cell from phi (liquid iff phi < 0); flipped cells
// are listed.  init = 1 (after creation or regrid): all blocks, no flips,
// previous = current.  Otherwise only blocks of the previous band (they keep the band
// flag the previous band pass set until the link pass rewrites the flags), and every
// block next to a flipped cell (or holding one) that is not in that band gets BF_CHECK
// and a place in the check list.
template <int Q>
__global__ void k_classify_phase(Ctx C, BlockShape S, const int *list, int nlist, int glevel, int init) {
  LSB_GRID_WAIT();
  using LT = Lat<Q>;
  constexpr int D = LT::D;
  // phi changes only on band cells, so outside the previous band no phase (and no stale
  // flip bit: flips happen next to the interface, inside the band) can change: unless
  // init, the blocks are those of the previous band list
  if (!init) {
    nlist = min(C.counters[glevel * NCOUNT + 5], C.band_cap);
    list = C.band_list + (long long)glevel * C.band_cap;
    // the band count starts again for the band pass (no pass before it reads it)
    if (blockIdx.x == 0 && threadIdx.x == 0) C.counters[glevel * NCOUNT + 3] = 0;
  }
  for (int w = blockIdx.x; w < nlist; w += gridDim.x) {
    const int gb = list[w];
    int x, y, z;
    const LevelDev &L = blk_cell(C, S, gb, threadIdx.x, x, y, z);
    if (x >= L.n[0] || y >= L.n[1] || z >= L.n[2]) continue;
    const long long c = cidx(L, x, y, z);
    const uint8_t tg = C.tag[L.cell_off + c];
    if (!(tg & TAG_LEAF)) continue;
    const float ph = C.phi[L.fine_off + c];
    // the transport and reinitialisation stages of this update wrote p1, p2 on band
    // cells: back to phi, as the mirrored passes expect outside the next band
    C.p1[L.fine_off + c] = ph;
    C.p2[L.fine_off + c] = ph;
    const int gas = ph >= 0.0f ? 1 : 0;
    const int prev = init ? gas : (tg & TAG_GAS);
    const bool flip = !init && (gas != prev);
    uint8_t nt = (tg & (TAG_LEAF | TAG_RLAYER | TAG_GHOST)) | (gas ? TAG_GAS : 0) | (prev ? TAG_PREVGAS : 0) |
                 (flip ? TAG_FLIP : 0);
    C.tag[L.cell_off + c] = nt;
    if (flip) {
      int e = atomicAdd(&C.counters[glevel * NCOUNT + 2], 1);
      if (e < C.list_cap) C.flip_list[(long long)glevel * C.list_cap + e] = make_int2(C.blk_ld[gb], (int)c);
      else atomicOr(C.err, ERR_LIST_OVF);
      // the blocks around the flip that the previous band does not hold: the band flags
      // tested here are those of the previous classification, which no thread of this pass
      // changes
      for (int k = 0; k < Q; ++k) {
        int sx = x + LT::cx(k), sy = y + LT::cy(k), sz = z + LT::cz(k);
        if (!(wrap(L, 0, sx) && wrap(L, 1, sy) && (D == 2 || wrap(L, 2, sz)))) continue;
        const int nb = L.block_off + block_of(L, sx, sy, sz, S);
        // set BF_CHECK once per block (compare-and-swap on the flag's word) and list it
        unsigned *wp = reinterpret_cast<unsigned *>(C.bflag + (nb & ~3));
        const int sh = (nb & 3) * 8;
        unsigned old = *reinterpret_cast<volatile unsigned *>(wp);
        while (!(((old >> sh) & 0xffu) & (BF_BAND | BF_CHECK))) {
          const unsigned seen = atomicCAS(wp, old, old | ((unsigned)BF_CHECK << sh));
          if (seen == old) {
            const int slot = atomicAdd(&C.counters[glevel * NCOUNT + 4], 1);
            if (slot < C.band_cap) C.check_list[(long long)glevel * C.band_cap + slot] = nb;
            else atomicOr(C.err, ERR_BAND_OVF);
            break;
          }
          old = seen;
        }
      }
    }
  }
}

// Pass 2: cut mask of every leaf cell (bit k: source x - c_k is a leaf of the
// other phase), link base, interface list, block interface flag.  Unless full,
// only blocks of the previous band and blocks next to a flipped cell are
// examined: phi changes only on band cells, so a cut link elsewhere would need a
// neighbour that flipped; every other block has no cut link now and, having left
// the band with none, an all-zero mask already.
template <int Q>
__global__ void k_classify_links(Ctx C, BlockShape S, const int *list, int nlist, int glevel, int full) {
  LSB_GRID_WAIT();
  using LT = Lat<Q>;
  constexpr int D = LT::D;
  // unless full: the previous band list, then the check list (every other block keeps
  // flag 0 and an all-zero mask)
  int nband = nlist;
  if (!full) {
    nband = min(C.counters[glevel * NCOUNT + 5], C.band_cap);
    nlist = nband + min(C.counters[glevel * NCOUNT + 4], C.band_cap);
    list = C.band_list + (long long)glevel * C.band_cap;
  }
  const int *chk = C.check_list + (long long)glevel * C.band_cap;
  for (int w = blockIdx.x; w < nlist; w += gridDim.x) {
    const int gb = w < nband ? list[w] : chk[w - nband];
    const bool work = full || (C.bflag[gb] & (BF_BAND | BF_CHECK));
    __syncthreads();  // every thread has read the flags before thread 0 rewrites them
    if (!work) {
      if (threadIdx.x == 0) C.bflag[gb] = 0;
      continue;
    }
    int x, y, z;
    const LevelDev &L = blk_cell(C, S, gb, threadIdx.x, x, y, z);
    uint32_t m = 0;
    long long c = 0;
    uint8_t tg = 0;
    if (x < L.n[0] && y < L.n[1] && z < L.n[2]) {
      c = cidx(L, x, y, z);
      tg = C.tag[L.cell_off + c];
      if (tg & TAG_LEAF) {
        const bool inner = x >= 1 && x + 1 < L.n[0] && y >= 1 && y + 1 < L.n[1] && (D == 2 || (z >= 1 && z + 1 < L.n[2]));
        if (inner) {  // every source inside the box: direct offsets
          const long long p0 = L.p[0], p01 = (long long)L.p[0] * L.p[1];
          const uint8_t *tc = C.tag + L.cell_off + c;
#pragma unroll
          for (int k = 0; k < Q; ++k) {
            if (k == LT::REST) continue;
            const uint8_t ts = tc[-(LT::cx(k) + LT::cy(k) * p0 + LT::cz(k) * p01)];
            if ((ts & TAG_LEAF) && ((ts & TAG_GAS) != (tg & TAG_GAS))) m |= 1u << k;
          }
        } else {
          for (int k = 0; k < Q; ++k) {
            if (k == LT::REST) continue;
            int sx = x - LT::cx(k), sy = y - LT::cy(k), sz = z - LT::cz(k);
            if (!(wrap(L, 0, sx) && wrap(L, 1, sy) && (D == 2 || wrap(L, 2, sz)))) continue;
            const uint8_t ts = C.tag[L.cell_off + cidx(L, sx, sy, sz)];
            if ((ts & TAG_LEAF) && ((ts & TAG_GAS) != (tg & TAG_GAS))) m |= 1u << k;
          }
        }
        C.cmask[L.fine_off + c] = m;
      }
    }
    // slots in the link list and the interface list, one atomic per warp (every lane
    // of the CTA is here: the block-level branch above is uniform)
    const int lane = threadIdx.x & 31;
    const int np = __popc(m);
    int incl = np;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    const int wlinks = __shfl_sync(0xffffffffu, incl, 31);
    const unsigned wcells = __ballot_sync(0xffffffffu, m != 0);
    int lbase = 0, cbase0 = 0;
    if (lane == 0 && wcells) {
      lbase = atomicAdd(&C.counters[glevel * NCOUNT + 0], wlinks);
      cbase0 = atomicAdd(&C.counters[glevel * NCOUNT + 1], __popc(wcells));
    }
    lbase = __shfl_sync(0xffffffffu, lbase, 0);
    cbase0 = __shfl_sync(0xffffffffu, cbase0, 0);
    if (m) {
      const int base = lbase + incl - np;
      if ((long long)base + np > C.link_cap) atomicOr(C.err, ERR_LINK_OVF);
      C.cbase[L.fine_off + c] = base;
      // the link list: one entry per cut link, in link-buffer order
      const int2 cell = make_int2(C.blk_ld[gb], (int)c);
      uint32_t mm = m;
      for (int r = 0; mm; ++r) {
        const int k = __ffs(mm) - 1;
        mm &= mm - 1u;
        if ((long long)base + r < C.link_cap) {
          C.link_cell[C.link_list_off[glevel] + base + r] = cell;
          C.link_dir[C.link_list_off[glevel] + base + r] = (uint8_t)k;
        }
      }
      C.tag[L.cell_off + c] = tg | TAG_IFACE;
      const int e = cbase0 + __popc(wcells & ((1u << lane) - 1u));
      if (e < C.list_cap) C.iface_list[(long long)glevel * C.list_cap + e] = make_int2(C.blk_ld[gb], (int)c);
      else atomicOr(C.err, ERR_LIST_OVF);
    }
    const bool any = __syncthreads_or(m != 0);
    if (threadIdx.x == 0) C.bflag[gb] = any ? BF_IFACE : 0;
  }
}

// Pass 3: band flag of every active finest block (itself or a 3^D neighbour
// holds an interface cell); band blocks are listed.  One warp per block, lane k
// reading the flags of neighbour k, so the 3^D loads are in flight together.
// On the CTAs [b0, b0 + nb) of the launch.
template <int Q>
__device__ __forceinline__ void d_band(const Ctx &C, const int *list, int nlist, int glevel, int b0, int nb) {
  constexpr int D = Lat<Q>::D;
  constexpr int NN = D == 3 ? 27 : 9;
  const int lane = threadIdx.x & 31;
  const int wpb = blockDim.x >> 5;
  for (int w = ((int)blockIdx.x - b0) * wpb + (threadIdx.x >> 5); w < nlist; w += nb * wpb) {
    const int gb = list[w];
    const LevelDev &L = C.lds[C.blk_ld[gb]];
    bool hot = false;
    if (lane < NN) {
      const int lb = gb - L.block_off;
      int nb3[3] = {lb % L.nb[0] + lane % 3 - 1, (lb / L.nb[0]) % L.nb[1] + (lane / 3) % 3 - 1,
                    lb / (L.nb[0] * L.nb[1]) + (D == 3 ? lane / 9 - 1 : 0)};
      bool ok = true;
      for (int a = 0; a < D; ++a) {
        if (nb3[a] < 0 || nb3[a] >= L.nb[a]) {
          if (L.per[a]) nb3[a] = (nb3[a] + L.nb[a]) % L.nb[a];
          else ok = false;
        }
      }
      if (ok) hot = (C.bflag[L.block_off + nb3[0] + L.nb[0] * (nb3[1] + L.nb[1] * nb3[2])] & BF_IFACE) != 0;
    }
    const bool band = __any_sync(0xffffffffu, hot);
    if (lane == 0 && band && C.bstat[gb] == BLK_LEAF) {
      C.bflag[gb] = C.bflag[gb] | BF_BAND;
      const int e = atomicAdd(&C.counters[glevel * NCOUNT + 3], 1);
      if (e < C.band_cap) {
        C.band_list[(long long)glevel * C.band_cap + e] = gb;
        C.band_info[(long long)glevel * C.band_cap + e] = C.blk_info[gb];
      } else {
        atomicOr(C.err, ERR_BAND_OVF);
      }
    }
  }
}

// ------------------------------------------------------------------ geometry (float64)
// Unweighted least-squares quadratic over the 3^D stencil.  With offsets in
// {-1,0,1}^D the odd basis functions decouple: grad_a = sum(o_a phi)/sum(o_a^2),
// H_ab = sum(o_a o_b phi)/sum(o_a^2 o_b^2) (a != b); the constant and pure
// quadratic coefficients solve the 1 + D even normal equations in closed form.
// n = g/|g|, kappa = (|g|^2 tr H - g.H.g)/|g|^3.
// which: 0 the interface list, 1 the flip list, 2 both (one index space, interface
// cells first; a cell on both lists gets the same values twice).
// On the CTAs [b0, b0 + nb) of the launch; post(it) runs after the fit of each flipped cell.
template <int D, typename Post>
__device__ __forceinline__ void d_geometry(const Ctx &C, int glevel, int which, int b0, int nb, Post post) {
  const int ni = which == 1 ? 0 : min(C.counters[glevel * NCOUNT + 1], (int)C.list_cap);
  const int nf = which == 0 ? 0 : min(C.counters[glevel * NCOUNT + 2], (int)C.list_cap);
  const int2 *li = C.iface_list + (long long)glevel * C.list_cap;
  const int2 *lf = C.flip_list + (long long)glevel * C.list_cap;
  for (int e = ((int)blockIdx.x - b0) * blockDim.x + threadIdx.x; e < ni + nf; e += nb * blockDim.x) {
    const int2 it = e < ni ? li[e] : lf[e - ni];
    const LevelDev &L = C.lds[it.x];
    const long long c = it.y;
    int x, y, z;
    cell_xyz(L, c, x, y, z);
    // Stencil sums exactly: phi (float) in fixed point with 30 fraction bits (exact
    // for |phi| >= 2^-6, within 2^-31 below), summed in 64-bit integers, then
    // converted to float64 (exact below 2^53).  This keeps the float64 work of the
    // fit to the closed-form solve; GB300 runs float64 at a small fraction of its
    // integer rate.
    long long iP = 0, isx[3] = {0, 0, 0}, isxx[3] = {0, 0, 0}, isxy[3] = {0, 0, 0};
    // cells whose 3^D stencil lies inside the box read it at direct offsets
    const bool inner = x >= 1 && x + 1 < L.n[0] && y >= 1 && y + 1 < L.n[1] && (D == 2 || (z >= 1 && z + 1 < L.n[2]));
    const long long p0 = L.p[0], p01 = (long long)L.p[0] * L.p[1];
#pragma unroll
    for (int oz = (D == 3 ? -1 : 0); oz <= (D == 3 ? 1 : 0); ++oz)
#pragma unroll
      for (int oy = -1; oy <= 1; ++oy)
#pragma unroll
        for (int ox = -1; ox <= 1; ++ox) {
          long long cc;
          if (inner) {
            cc = c + ox + oy * p0 + oz * p01;
          } else {
            const int xx = clampwrap(L, 0, x + ox), yy = clampwrap(L, 1, y + oy);
            const int zz = D == 3 ? clampwrap(L, 2, z + oz) : 0;
            cc = cidx(L, xx, yy, zz);
          }
          const long long v = __float2ll_rn(C.phi[L.fine_off + cc] * 1073741824.0f);
          const int o[3] = {ox, oy, oz};
          iP += v;
          for (int a = 0; a < D; ++a) {
            isx[a] += o[a] > 0 ? v : (o[a] < 0 ? -v : 0);
            isxx[a] += o[a] != 0 ? v : 0;
          }
          isxy[0] += ox * oy > 0 ? v : (ox * oy < 0 ? -v : 0);
          if (D == 3) {
            isxy[1] += ox * oz > 0 ? v : (ox * oz < 0 ? -v : 0);
            isxy[2] += oy * oz > 0 ? v : (oy * oz < 0 ? -v : 0);
          }
        }
    // The fit's coefficients are fixed rational combinations of the stencil sums.  In 2D
    // (9 points: sum o^2 = 6, sum o_x^2 o_y^2 = 4, sum o^4 = 6) g_a = S_a / 6, H_aa =
    // (3 S_aa - 2 P) / 3, H_xy = S_xy / 4; in 3D (27 points: 18, 12, 18) g_a = S_a / 18,
    // H_aa = (3 S_aa - 2 P) / 9, H_ab = S_ab / 12.  In the unit 1 / (12 * 2^30) (2D) or
    // 1 / (36 * 2^30) (3D) both read g = 2 G and H = K with the integers G_a = S_a,
    // K_aa = 4 (3 S_aa - 2 P), K_ab = 3 S_ab, and kappa, homogeneous of degree zero in
    // (g, H), is (|G|^2 tr K - G.K.G) / (2 |G|^3): float64 from exact integers, one
    // square root and two divisions.
    double G[3] = {0, 0, 0}, K[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    for (int a = 0; a < D; ++a) {
      G[a] = (double)isx[a];
      K[a][a] = (double)(4 * (3 * isxx[a] - 2 * iP));
    }
    K[0][1] = K[1][0] = (double)(3 * isxy[0]);
    if (D == 3) {
      K[0][2] = K[2][0] = (double)(3 * isxy[1]);
      K[1][2] = K[2][1] = (double)(3 * isxy[2]);
    }
    double g2 = 0, tr = 0, gKg = 0;
    for (int a = 0; a < D; ++a) {
      g2 += G[a] * G[a];
      tr += K[a][a];
      for (int b = 0; b < D; ++b) gKg += G[a] * K[a][b] * G[b];
    }
    const double mag = sqrt(g2);
    const long long fc = L.fine_off + c;
    // |grad phi| = |G| / (6 or 18) / 2^30
    if (mag > 1e-12 * (D == 2 ? 6.0 : 18.0) * 1073741824.0) {
      const double inv = 1.0 / mag;
      for (int a = 0; a < D; ++a) C.nvec[a * C.nfine + fc] = (float)(G[a] * inv);
      C.kappa[fc] = (float)((g2 * tr - gKg) / (2.0 * g2 * mag));
    } else {
      for (int a = 0; a < D; ++a) C.nvec[a * C.nfine + fc] = 0.f;
      C.kappa[fc] = 0.f;
    }
    if (e >= ni) post(it);
  }
}
template <int D>
__global__ void k_geometry(Ctx C, int glevel, int which) {
  LSB_GRID_WAIT();
  d_geometry<D>(C, glevel, which, 0, gridDim.x, [](int2) {});
}

// ------------------------------------------------------------------ velocity extension
// (d_ext_init, the interface cells' u~, is in lsb_device.cuh: the interface pass shares
// its launch)
template <int Q>
__global__ void k_ext_init(Ctx C, int glevel) {
  LSB_GRID_WAIT();
  d_ext_init<Q>(C, glevel, 0, gridDim.x);
}

// One Jacobi sweep of first-order upwind extension on the band (interface cells
// copy their value).  Neighbours outside the band read the committed field ut0.
// mode 0: sweep; 2: sweep and store the plan (velocity S(phi) n, upwind side and
// band membership of each upwind neighbour, interface / boundary bits), which phi
// fixes for all sweeps of a step; 3: sweep from the plan; 1: copy uin into ut0 on
// the band (commit).
template <int D>
__device__ __forceinline__ void d_ext_iter(const Ctx &C, BlockShape S, int glevel, const float *uin, float *uout, int mode) {
  const int nl = min(C.counters[glevel * NCOUNT + 3], C.band_cap);
  const int *lst = C.band_list + (long long)glevel * C.band_cap;
  for (int w = blockIdx.x; w < nl; w += gridDim.x) {
    const int gb = lst[w];
    int x, y, z;
    const LevelDev &L = band_cell(C, S, glevel, w, threadIdx.x, x, y, z);
    if (!L.ls_active) continue;  // frozen level set in this case
    if (x >= L.n[0] || y >= L.n[1] || z >= L.n[2]) continue;
    const long long fo = L.fine_off, NF = C.nfine;
    const long long c = cidx(L, x, y, z);
    if (mode == 1) {
      for (int a = 0; a < D; ++a) C.ut0[a * NF + fo + c] = uin[a * NF + fo + c];
      continue;
    }
    const int crd[3] = {x, y, z};
    const int str[3] = {1, L.p[0], L.p[0] * L.p[1]};
    if (mode == 3) {
      // sweep from the plan of the first sweep: same values, no normal, no band lookups
      const uint8_t pf = C.plan_f[fo + c];
      if (pf & 64) {
        for (int a = 0; a < D; ++a) uout[a * NF + fo + c] = uin[a * NF + fo + c];
        continue;
      }
      float u0[3];
      for (int b = 0; b < D; ++b) u0[b] = uin[b * NF + fo + c];
      float acc[3] = {0.f, 0.f, 0.f};
      for (int a = 0; a < D; ++a) {
        const float va = C.plan_v[a * NF + fo + c];
        const int dir = (pf >> a) & 1 ? -1 : 1;
        long long cn;
        if (pf & 128) {
          int nb[3] = {x, y, z};
          nb[a] = clampwrap(L, a, crd[a] + dir);
          cn = cidx(L, nb[0], nb[1], nb[2]);
        } else {
          cn = c + dir * str[a];
        }
        const float *src = (pf >> (3 + a)) & 1 ? uin : C.ut0;
        for (int b = 0; b < D; ++b) {
          const float un = src[b * NF + fo + cn];
          acc[b] += va * (va > 0.f ? (u0[b] - un) : (un - u0[b]));
        }
      }
      for (int b = 0; b < D; ++b) uout[b * NF + fo + c] = u0[b] - L.dtau_ext * acc[b];
      continue;
    }
    const uint8_t tg = C.tag[L.cell_off + c];
    if (tg & TAG_IFACE) {
      for (int a = 0; a < D; ++a) uout[a * NF + fo + c] = uin[a * NF + fo + c];
      if (mode == 2) C.plan_f[fo + c] = 64;
      continue;
    }
    // interior: all +-1 neighbours inside the box (direct offsets, face-neighbour band flags)
    bool inner = true;
    for (int a = 0; a < D; ++a) inner = inner && crd[a] >= 1 && crd[a] + 1 < L.n[a];
    const float *phiL = C.phi + fo;
    float nvec[3], gm = 0.f;
    uint8_t pf = inner ? 0 : 128;
    for (int a = 0; a < D; ++a) {
      if (inner) {
        nvec[a] = 0.5f * (phiL[(unsigned)c + str[a]] - phiL[(unsigned)c - str[a]]);
      } else {
        int p[3] = {x, y, z}, m[3] = {x, y, z};
        p[a] = clampwrap(L, a, crd[a] + 1);
        m[a] = clampwrap(L, a, crd[a] - 1);
        nvec[a] = 0.5f * (phiL[cidx(L, p[0], p[1], p[2])] - phiL[cidx(L, m[0], m[1], m[2])]);
      }
      gm += nvec[a] * nvec[a];
    }
    gm = sqrtf(gm);
    const float ph = phiL[c];
    const float sg = ph / sqrtf(ph * ph + 1.0f);
    float u0[3];
    for (int b = 0; b < D; ++b) u0[b] = uin[b * NF + fo + c];
    float acc[3] = {0.f, 0.f, 0.f};
    for (int a = 0; a < D; ++a) {
      const float va = gm > 0.f ? sg * nvec[a] / gm : 0.f;
      const int dir = va > 0.f ? -1 : 1;
      long long cn;
      bool inb;
      if (inner) {
        cn = c + dir * str[a];
        const int s0 = (crd[a] >> S.lg[a]) << S.lg[a];
        const int q = crd[a] + dir;
        if (q >= s0 && q < s0 + S.bs[a]) {
          inb = true;  // own block (a band block)
        } else {
          const int bstr = a == 0 ? 1 : (a == 1 ? L.nb[0] : L.nb[0] * L.nb[1]);
          inb = (C.bflag[gb + dir * bstr] & BF_BAND) != 0;
        }
      } else {
        int nb[3] = {x, y, z};
        nb[a] = clampwrap(L, a, crd[a] + dir);
        cn = cidx(L, nb[0], nb[1], nb[2]);
        inb = in_band(C, L, S, nb[0], nb[1], nb[2]);
      }
      const float *src = inb ? uin : C.ut0;
      for (int b = 0; b < D; ++b) {
        const float un = src[b * NF + fo + cn];
        acc[b] += va * (va > 0.f ? (u0[b] - un) : (un - u0[b]));
      }
      if (mode == 2) {
        C.plan_v[a * NF + fo + c] = va;
        pf |= (dir < 0 ? 1 : 0) << a;
        pf |= (inb ? 1 : 0) << (3 + a);
      }
    }
    for (int b = 0; b < D; ++b) uout[b * NF + fo + c] = u0[b] - L.dtau_ext * acc[b];
    if (mode == 2) C.plan_f[fo + c] = pf;
  }
}
template <int D>
__global__ void k_ext_iter(Ctx C, BlockShape S, int glevel, const float *uin, float *uout, int mode) {
  LSB_GRID_WAIT();
  d_ext_iter<D>(C, S, glevel, uin, uout, mode);
}

#ifndef LSB_EXT_MINB
#define LSB_EXT_MINB 3  // CTAs of 512 threads per SM the sweep is built for
#endif
#ifndef LSB_EXT_U
#define LSB_EXT_U 1  // band blocks a thread carries at once
#endif
// The sweeps after the first (mode 3 of d_ext_iter: the same arithmetic in the same order)
// as a lean kernel of its own.  Its chain of dependent loads (band list, block coordinates,
// plan, values, upwind neighbours) is latency-bound and the band holds only a few blocks
// per resident CTA: one cell per thread (LSB_EXT_U blocks at once) at three CTAs per SM
// measured faster than two blocks per thread at two CTAs per SM (more CTAs in flight).
// MIRROR: the forward step's stage arrays equal ut0 outside the band, so every
// upwind neighbour reads uin (no band bit of the plan consulted).
template <int D, bool MIRROR = false>
__global__ void __launch_bounds__(512, LSB_EXT_MINB) k_ext_plan(Ctx C, BlockShape S, int glevel, const float *__restrict__ uin,
                                                     float *__restrict__ uout) {
  LSB_GRID_WAIT();
  const int nl = min(C.counters[glevel * NCOUNT + 3], C.band_cap);
  const int *lst = C.band_list + (long long)glevel * C.band_cap;
  const long long NF = C.nfine;
  const int G = gridDim.x;
  // each thread takes its cell in U band blocks per pass, with the blocks' dependent loads
  // (list entry, block coordinates, plan, neighbours) issued side by side
  constexpr int U = LSB_EXT_U;
  for (int w0 = blockIdx.x; w0 < nl; w0 += U * G) {
    int gb[U];
#pragma unroll
    for (int k = 0; k < U; ++k) gb[k] = w0 + k * G < nl ? __ldg(lst + w0 + k * G) : -1;
    int4 bi[U];
#pragma unroll
    for (int k = 0; k < U; ++k)
      bi[k] = gb[k] >= 0 ? __ldg(C.band_info + (long long)glevel * C.band_cap + w0 + k * G) : make_int4(-1, 0, 0, 0);
    bool act[U];
    long long fo[U], c[U];
    int x[U], y[U], z[U];
    uint8_t pf[U];
#pragma unroll
    for (int k = 0; k < U; ++k) {
      act[k] = bi[k].x >= 0;
      fo[k] = 0;
      c[k] = 0;
      x[k] = y[k] = z[k] = 0;
      pf[k] = 64;
      if (!act[k]) continue;
      const LevelDev &L = C.lds[bi[k].x];
      x[k] = (bi[k].y << S.lg[0]) + (threadIdx.x & (S.bs[0] - 1));
      y[k] = (bi[k].z << S.lg[1]) + ((threadIdx.x >> S.lg[0]) & (S.bs[1] - 1));
      z[k] = (bi[k].w << S.lg[2]) + (threadIdx.x >> (S.lg[0] + S.lg[1]));
      act[k] = L.ls_active && x[k] < L.n[0] && y[k] < L.n[1] && z[k] < L.n[2];
      if (!act[k]) continue;
      fo[k] = L.fine_off;
      c[k] = cidx(L, x[k], y[k], z[k]);
      pf[k] = __ldg(C.plan_f + fo[k] + c[k]);
    }
    float u0[U][3], un[U][D][3], va[U][3];
#pragma unroll
    for (int k = 0; k < U; ++k) {
      if (!act[k]) continue;
      const float *ui = uin + fo[k];
#pragma unroll
      for (int b = 0; b < D; ++b) u0[k][b] = __ldg(ui + b * NF + c[k]);
      if (pf[k] & 64) continue;
      const LevelDev &L = C.lds[bi[k].x];
#pragma unroll
      for (int a = 0; a < D; ++a) {
        va[k][a] = __ldg(C.plan_v + a * NF + fo[k] + c[k]);
        const int dir = (pf[k] >> a) & 1 ? -1 : 1;
        long long cn;
        if (pf[k] & 128) {  // box-boundary cell: the neighbour clamped or wrapped
          const int nx = a == 0 ? clampwrap(L, 0, x[k] + dir) : x[k];
          const int ny = a == 1 ? clampwrap(L, 1, y[k] + dir) : y[k];
          const int nz = a == 2 ? clampwrap(L, 2, z[k] + dir) : z[k];
          cn = cidx(L, nx, ny, nz);
        } else {
          cn = c[k] + dir * (a == 0 ? 1LL : (a == 1 ? (long long)L.p[0] : (long long)L.p[0] * L.p[1]));
        }
        const float *src = (MIRROR || ((pf[k] >> (3 + a)) & 1)) ? ui : C.ut0 + fo[k];
#pragma unroll
        for (int b = 0; b < D; ++b) un[k][a][b] = __ldg(src + b * NF + cn);
      }
    }
#pragma unroll
    for (int k = 0; k < U; ++k) {
      if (!act[k]) continue;
      float *uo = uout + fo[k];
      if (pf[k] & 64) {  // outside the band: carried over
#pragma unroll
        for (int b = 0; b < D; ++b) uo[b * NF + c[k]] = u0[k][b];
        continue;
      }
      float acc[3] = {0.f, 0.f, 0.f};
#pragma unroll
      for (int a = 0; a < D; ++a)
#pragma unroll
        for (int b = 0; b < D; ++b)
          acc[b] += va[k][a] * (va[k][a] > 0.f ? (u0[k][b] - un[k][a][b]) : (un[k][a][b] - u0[k][b]));
      const float dt = C.lds[bi[k].x].dtau_ext;
#pragma unroll
      for (int b = 0; b < D; ++b) uo[b * NF + c[k]] = u0[k][b] - dt * acc[b];
    }
  }
}

// ------------------------------------------------------------------ transport
// Gather phi along axis a at offsets -3..+3; points in the band (and, for the
// reinitialisation, not frozen) read the stage array, others the committed phi.
template <int D>
__device__ __forceinline__ void gather7(const Ctx &C, const LevelDev &L, const BlockShape &S, const float *pin,
                                        bool use_frozen, int x, int y, int z, int a, float v[7]) {
  const int crd[3] = {x, y, z};
  for (int m = 0; m < 7; ++m) {
    int p[3] = {x, y, z};
    p[a] = clampwrap(L, a, crd[a] + m - 3);
    const long long cc = L.fine_off + cidx(L, p[0], p[1], p[2]);
    bool upd = pin != C.phi && in_band(C, L, S, p[0], p[1], p[2]);
    if (upd && use_frozen) upd = !C.frozen[cc];
    v[m] = upd ? pin[cc] : C.phi[cc];
  }
}

// gather7 for a cell of band block gb (global id) at level offset c.  When the
// seven points lie inside the box on axis a (no clamping or wrapping), they are
// read at direct offsets, and a point's band membership is its own block's
// (always in the band) or that of the face neighbour it falls into; otherwise the
// general path above.  Same values as gather7.
template <int D>
__device__ __forceinline__ void gather7f(const Ctx &C, const LevelDev &L, const BlockShape &S, int gb,
                                         const float *pin, bool use_frozen, int x, int y, int z, unsigned c, int a,
                                         float v[7]) {
  const int crd = a == 0 ? x : (a == 1 ? y : z);
  if (crd < 3 || crd + 3 >= L.n[a] || S.bs[a] < 4) {  // the fast path assumes at most one block crossed
    gather7<D>(C, L, S, pin, use_frozen, x, y, z, a, v);
    return;
  }
  const float *phiL = C.phi + L.fine_off;
  const float *pinL = pin + L.fine_off;
  const uint8_t *frzL = C.frozen + L.fine_off;
  const bool merged = pin != C.phi;
  const int str = a == 0 ? 1 : (a == 1 ? L.p[0] : L.p[0] * L.p[1]);
  const int s0 = (crd >> S.lg[a]) << S.lg[a], s1 = s0 + S.bs[a];
  const int bstr = a == 0 ? 1 : (a == 1 ? L.nb[0] : L.nb[0] * L.nb[1]);
  bool fm = false, fp = false;
  if (merged) {
    if (crd - 3 < s0) fm = (C.bflag[gb - bstr] & BF_BAND) != 0;
    if (crd + 3 >= s1) fp = (C.bflag[gb + bstr] & BF_BAND) != 0;
  }
#pragma unroll
  for (int m = 0; m < 7; ++m) {
    const int q = crd + m - 3;
    const unsigned off = c + (m - 3) * str;
    bool upd = merged && (q < s0 ? fm : (q >= s1 ? fp : true));
    if (upd && use_frozen) upd = !frzL[off];
    const float *src = upd ? pinL : phiL;  // one load from the selected array
    v[m] = src[off];
  }
}

__device__ __forceinline__ float d5m(const float v[7]) {  // left-biased, offsets -3..+2
  return (-2.f * v[0] + 15.f * v[1] - 60.f * v[2] + 20.f * v[3] + 30.f * v[4] - 3.f * v[5]) / 60.f;
}
__device__ __forceinline__ float d5p(const float v[7]) {  // mirror image
  return -(-2.f * v[6] + 15.f * v[5] - 60.f * v[4] + 20.f * v[3] + 30.f * v[2] - 3.f * v[1]) / 60.f;
}

// TVD-RK3 stage of d phi/dt = -u~ . grad phi on the band (dt = 1):
// stage 1: p1 = phi + L(phi); 2: p2 = 3/4 phi + 1/4 (p1 + L(p1)); 3: phi = 1/3 phi + 2/3 (p2 + L(p2)).
template <int D>
__device__ __forceinline__ void d_adv_stage(const Ctx &C, BlockShape S, int glevel, int stage) {
  const int nl = min(C.counters[glevel * NCOUNT + 3], C.band_cap);
  const float *pin = stage == 1 ? C.phi : (stage == 2 ? C.p1 : C.p2);
  for (int w = blockIdx.x; w < nl; w += gridDim.x) {
    int x, y, z;
    const LevelDev &L = band_cell(C, S, glevel, w, threadIdx.x, x, y, z);
    if (!L.ls_active) continue;  // frozen level set in this case
    if (x >= L.n[0] || y >= L.n[1] || z >= L.n[2]) continue;
    const long long fc = L.fine_off + cidx(L, x, y, z);
    float rhs = 0.f;
    for (int a = 0; a < D; ++a) {
      float v[7];
      gather7<D>(C, L, S, pin, false, x, y, z, a, v);  // measured faster here than gather7f
      const float ua = C.ut0[a * C.nfine + fc];
      rhs -= ua * (ua >= 0.f ? d5m(v) : d5p(v));
    }
    const float p0 = C.phi[fc];
    if (stage == 1) C.p1[fc] = p0 + rhs;
    else if (stage == 2) C.p2[fc] = 0.75f * p0 + 0.25f * (C.p1[fc] + rhs);
    else C.phi[fc] = p0 / 3.0f + (2.0f / 3.0f) * (C.p2[fc] + rhs);
  }
}
template <int D>
__global__ void k_adv_stage(Ctx C, BlockShape S, int glevel, int stage) {
  LSB_GRID_WAIT();
  d_adv_stage<D>(C, S, glevel, stage);
}

// ------------------------------------------------------------------ reinitialisation
// Frozen cells (sign change to any lattice neighbour in the box) and S(phi0).
template <int Q>
__device__ __forceinline__ void d_reinit_prep(const Ctx &C, BlockShape S, int glevel) {
  using LT = Lat<Q>;
  constexpr int D = LT::D;
  const int nl = min(C.counters[glevel * NCOUNT + 3], C.band_cap);
  for (int w = blockIdx.x; w < nl; w += gridDim.x) {
    int x, y, z;
    const LevelDev &L = band_cell(C, S, glevel, w, threadIdx.x, x, y, z);
    if (!L.ls_active) continue;  // frozen level set in this case
    if (x >= L.n[0] || y >= L.n[1] || z >= L.n[2]) continue;
    const long long fc = L.fine_off + cidx(L, x, y, z);
    const float p = C.phi[fc];
    const bool g = p >= 0.f;
    bool fr = false;
    const bool inner = x >= 1 && x + 1 < L.n[0] && y >= 1 && y + 1 < L.n[1] && (D == 2 || (z >= 1 && z + 1 < L.n[2]));
    if (inner) {  // every lattice neighbour inside the box: direct offsets
      const int p0 = L.p[0], p01 = L.p[0] * L.p[1];
#pragma unroll
      for (int i = 0; i < Q; ++i) {
        if (i == LT::REST) continue;
        if ((C.phi[fc + LT::cx(i) + LT::cy(i) * p0 + LT::cz(i) * p01] >= 0.f) != g) fr = true;
      }
    } else {
      for (int i = 0; i < Q; ++i) {
        if (i == LT::REST) continue;
        int tx = x + LT::cx(i), ty = y + LT::cy(i), tz = z + LT::cz(i);
        if (!(wrap(L, 0, tx) && wrap(L, 1, ty) && (D == 2 || wrap(L, 2, tz)))) continue;
        if ((C.phi[L.fine_off + cidx(L, tx, ty, tz)] >= 0.f) != g) fr = true;
      }
    }
    C.frozen[fc] = fr ? 1 : 0;
    C.s0[fc] = p / sqrtf(p * p + 1.0f);
  }
}
template <int Q>
__global__ void k_reinit_prep(Ctx C, BlockShape S, int glevel) {
  LSB_GRID_WAIT();
  d_reinit_prep<Q>(C, S, glevel);
}

// HJ-WENO5 one-sided derivative (Jiang & Peng 2000) from the five differences.
// Constant divisions are multiplications by the reciprocals, and the three weights
// gamma_k / (s_k + eps)^2 are formed as gamma_k prod_{j != k} (s_j + eps)^2 (the
// same normalised weights, one division instead of four).
__device__ __forceinline__ float weno5(float v1, float v2, float v3, float v4, float v5) {
  const float eps = 1e-6f;
  const float r3 = 1.f / 3.f, r6 = 1.f / 6.f;
  const float d1 = v1 * r3 - 7.f * r6 * v2 + 11.f * r6 * v3;
  const float d2 = -v2 * r6 + 5.f * r6 * v3 + v4 * r3;
  const float d3 = v3 * r3 + 5.f * r6 * v4 - v5 * r6;
  const float b1 = v1 - 2.f * v2 + v3, c1 = v1 - 4.f * v2 + 3.f * v3;
  const float b2 = v2 - 2.f * v3 + v4, c2 = v2 - v4;
  const float b3 = v3 - 2.f * v4 + v5, c3 = 3.f * v3 - 4.f * v4 + v5;
  const float t1 = 13.f / 12.f * b1 * b1 + 0.25f * c1 * c1 + eps;
  const float t2 = 13.f / 12.f * b2 * b2 + 0.25f * c2 * c2 + eps;
  const float t3 = 13.f / 12.f * b3 * b3 + 0.25f * c3 * c3 + eps;
  const float q1 = t1 * t1, q2 = t2 * t2, q3 = t3 * t3;
  const float a1 = 0.1f * q2 * q3, a2 = 0.6f * q1 * q3, a3 = 0.3f * q1 * q2;
  return (a1 * d1 + a2 * d2 + a3 * d3) / (a1 + a2 + a3);
}

// TVD-RK3 stage of phi_tau = -S(phi0)(|grad phi|_G - 1) on band cells that are not frozen.
template <int D>
__device__ __forceinline__ void d_reinit_stage(const Ctx &C, BlockShape S, int glevel, int stage) {
  const int nl = min(C.counters[glevel * NCOUNT + 3], C.band_cap);
  const int *lst = C.band_list + (long long)glevel * C.band_cap;
  const float *pin = stage == 1 ? C.phi : (stage == 2 ? C.p1 : C.p2);
  for (int w = blockIdx.x; w < nl; w += gridDim.x) {
    const int gb = lst[w];
    int x, y, z;
    const LevelDev &L = band_cell(C, S, glevel, w, threadIdx.x, x, y, z);
    if (!L.ls_active) continue;  // frozen level set in this case
    if (x >= L.n[0] || y >= L.n[1] || z >= L.n[2]) continue;
    const unsigned cl = (unsigned)cidx(L, x, y, z);
    const long long fc = L.fine_off + cl;
    if (C.frozen[fc]) continue;
    const float s0 = C.s0[fc];
    float g2 = 0.f;
    for (int a = 0; a < D; ++a) {
      float v[7];
      gather7f<D>(C, L, S, gb, pin, true, x, y, z, cl, a, v);
      const float dm = weno5(v[1] - v[0], v[2] - v[1], v[3] - v[2], v[4] - v[3], v[5] - v[4]);
      const float dp = weno5(v[6] - v[5], v[5] - v[4], v[4] - v[3], v[3] - v[2], v[2] - v[1]);
      float ga;
      if (s0 > 0.f) ga = fmaxf(fmaxf(dm, 0.f) * fmaxf(dm, 0.f), fminf(dp, 0.f) * fminf(dp, 0.f));
      else ga = fmaxf(fminf(dm, 0.f) * fminf(dm, 0.f), fmaxf(dp, 0.f) * fmaxf(dp, 0.f));
      g2 += ga;
    }
    const float rhs = L.dtau_reinit * (-s0 * (sqrtf(g2) - 1.0f));
    const float p0 = C.phi[fc];
    if (stage == 1) C.p1[fc] = p0 + rhs;
    else if (stage == 2) C.p2[fc] = 0.75f * p0 + 0.25f * (C.p1[fc] + rhs);
    else C.phi[fc] = p0 / 3.0f + (2.0f / 3.0f) * (C.p2[fc] + rhs);
  }
}
template <int D>
__global__ void k_reinit_stage(Ctx C, BlockShape S, int glevel, int stage) {
  LSB_GRID_WAIT();
  d_reinit_stage<D>(C, S, glevel, stage);
}

// ------------------------------------------------------------------ forward passes on mirrored stage arrays
// The forward step keeps the stage arrays equal to the committed fields at every
// finest cell outside the band when a level-set update starts: p1 = p2 = phi and
// ut1 = ut2 = ut0.  Band cells restore this at the end of each update (u~ in the
// first transport stage, which also commits the extension; phi in the phase pass
// of the classification), and the host copies the arrays in full after creation
// and after every restore of phi or u~.  A stencil point then reads the stage
// array wherever it lies, so the passes below need no band or frozen-cell lookups;
// frozen cells of the reinitialisation write phi into the stage arrays their
// neighbours read.  The arithmetic and its order are those of the passes above,
// so the results are the same bit for bit.

// Resident CTAs of 512 threads per SM the mirrored stage kernels are compiled for (their
// registers capped to fit): the passes are latency-bound, so more warps in flight pay.
#ifndef LSB_LS_MINB
#define LSB_LS_MINB 3
#endif
#ifndef LSB_EF_MINB
#define LSB_EF_MINB LSB_LS_MINB  // the first extension sweep
#endif
#ifndef LSB_ADV_MINB
#define LSB_ADV_MINB LSB_LS_MINB  // the transport stages
#endif
#ifndef LSB_RE_MINB
#define LSB_RE_MINB LSB_LS_MINB  // the reinitialisation stages
#endif

// seven values of the stage array along axis a at offsets -3..+3 (clamped or
// wrapped at the box faces like gather7)
__device__ __forceinline__ void gather7m(const LevelDev &L, const float *__restrict__ pinL, int x, int y, int z,
                                         unsigned c, int a, float v[7]) {
  const int crd = a == 0 ? x : (a == 1 ? y : z);
  if (crd >= 3 && crd + 3 < L.n[a]) {
    const int str = a == 0 ? 1 : (a == 1 ? L.p[0] : L.p[0] * L.p[1]);
#pragma unroll
    for (int m = 0; m < 7; ++m) v[m] = pinL[c + (m - 3) * str];
  } else {
#pragma unroll
    for (int m = 0; m < 7; ++m) {
      int p[3] = {x, y, z};
      p[a] = clampwrap(L, a, crd + m - 3);
      v[m] = pinL[cidx(L, p[0], p[1], p[2])];
    }
  }
}

// First extension sweep of a step (mode 2 of d_ext_iter): sweep from uin = ut0 and
// store the plan (S(phi) n, upwind sides, interface and box-boundary bits).
template <int D>
// turn: also start the classification's counters (the band count into the previous-band
// slot, the other slots but the band count to zero; no pass between here and the
// classification reads them).
__global__ void __launch_bounds__(512, LSB_EF_MINB) k_ext_first(Ctx C, BlockShape S, int glevel, const float *__restrict__ uin,
                            float *__restrict__ uout, int turn) {
  LSB_GRID_WAIT();
  const int nl = min(C.counters[glevel * NCOUNT + 3], C.band_cap);
  if (turn && blockIdx.x == 0 && threadIdx.x == 0) {
    int *cnt = C.counters + glevel * NCOUNT;
    cnt[5] = cnt[3];
    cnt[0] = cnt[1] = cnt[2] = cnt[4] = 0;
  }
  const long long NF = C.nfine;
  // the next entry of the band list is loaded while this one is processed
  const int4 *info = C.band_info + (long long)glevel * C.band_cap;
  int4 next = blockIdx.x < nl ? __ldg(info + blockIdx.x) : make_int4(0, 0, 0, 0);
  for (int w = blockIdx.x; w < nl; w += gridDim.x) {
    const int4 bi = next;
    if (w + gridDim.x < nl) next = __ldg(info + w + gridDim.x);
    int x, y, z;
    const LevelDev &L = band_cell_at(C, S, bi, threadIdx.x, x, y, z);
    if (!L.ls_active) continue;
    if (x >= L.n[0] || y >= L.n[1] || z >= L.n[2]) continue;
    const long long fo = L.fine_off;
    const long long c = cidx(L, x, y, z);
    if (C.tag[L.cell_off + c] & TAG_IFACE) {
      for (int a = 0; a < D; ++a) uout[a * NF + fo + c] = uin[a * NF + fo + c];
      C.plan_f[fo + c] = 64;
      continue;
    }
    const int crd[3] = {x, y, z};
    const int str[3] = {1, L.p[0], L.p[0] * L.p[1]};
    bool inner = true;
    for (int a = 0; a < D; ++a) inner = inner && crd[a] >= 1 && crd[a] + 1 < L.n[a];
    const float *phiL = C.phi + fo;
    float nvec[3], gm = 0.f;
    uint8_t pf = inner ? 0 : 128;
    for (int a = 0; a < D; ++a) {
      if (inner) {
        nvec[a] = 0.5f * (phiL[(unsigned)c + str[a]] - phiL[(unsigned)c - str[a]]);
      } else {
        int p[3] = {x, y, z}, m[3] = {x, y, z};
        p[a] = clampwrap(L, a, crd[a] + 1);
        m[a] = clampwrap(L, a, crd[a] - 1);
        nvec[a] = 0.5f * (phiL[cidx(L, p[0], p[1], p[2])] - phiL[cidx(L, m[0], m[1], m[2])]);
      }
      gm += nvec[a] * nvec[a];
    }
    gm = sqrtf(gm);
    const float ph = phiL[c];
    const float sg = ph / sqrtf(ph * ph + 1.0f);
    float u0[3];
    for (int b = 0; b < D; ++b) u0[b] = uin[b * NF + fo + c];
    float acc[3] = {0.f, 0.f, 0.f};
    for (int a = 0; a < D; ++a) {
      const float va = gm > 0.f ? sg * nvec[a] / gm : 0.f;
      const int dir = va > 0.f ? -1 : 1;
      long long cn;
      if (inner) {
        cn = c + dir * str[a];
      } else {
        int nb[3] = {x, y, z};
        nb[a] = clampwrap(L, a, crd[a] + dir);
        cn = cidx(L, nb[0], nb[1], nb[2]);
      }
      for (int b = 0; b < D; ++b) {
        const float un = uin[b * NF + fo + cn];
        acc[b] += va * (va > 0.f ? (u0[b] - un) : (un - u0[b]));
      }
      C.plan_v[a * NF + fo + c] = va;
      pf |= (dir < 0 ? 1 : 0) << a;
    }
    for (int b = 0; b < D; ++b) uout[b * NF + fo + c] = u0[b] - L.dtau_ext * acc[b];
    C.plan_f[fo + c] = pf;
  }
}

// TVD-RK3 transport stage (as d_adv_stage).  Stage 1 takes u~ from the last
// extension sweep (ufin) and commits it to ut0, ut1 and ut2 at the cell.
template <int D>
__global__ void __launch_bounds__(512, LSB_ADV_MINB) k_adv_mirror(Ctx C, BlockShape S, int glevel, int stage,
                                                                 const float *__restrict__ ufin) {
  LSB_GRID_WAIT();
  const int nl = min(C.counters[glevel * NCOUNT + 3], C.band_cap);
  const float *pin = stage == 1 ? C.phi : (stage == 2 ? C.p1 : C.p2);
  const long long NF = C.nfine;
  // the next entry of the band list is loaded while this one is processed
  const int4 *info = C.band_info + (long long)glevel * C.band_cap;
  int4 next = blockIdx.x < nl ? __ldg(info + blockIdx.x) : make_int4(0, 0, 0, 0);
  for (int w = blockIdx.x; w < nl; w += gridDim.x) {
    const int4 bi = next;
    if (w + gridDim.x < nl) next = __ldg(info + w + gridDim.x);
    int x, y, z;
    const LevelDev &L = band_cell_at(C, S, bi, threadIdx.x, x, y, z);
    if (!L.ls_active) continue;
    if (x >= L.n[0] || y >= L.n[1] || z >= L.n[2]) continue;
    const unsigned c = (unsigned)cidx(L, x, y, z);
    const long long fc = L.fine_off + c;
    float ua[3];
    if (stage == 1) {
      for (int a = 0; a < D; ++a) {
        const float u = ufin[a * NF + fc];
        ua[a] = u;
        C.ut0[a * NF + fc] = u;
        C.ut1[a * NF + fc] = u;
        C.ut2[a * NF + fc] = u;
      }
    } else {
      for (int a = 0; a < D; ++a) ua[a] = C.ut0[a * NF + fc];
    }
    const float *pinL = pin + L.fine_off;
    float rhs = 0.f;
    for (int a = 0; a < D; ++a) {
      float v[7];
      gather7m(L, pinL, x, y, z, c, a, v);
      rhs -= ua[a] * (ua[a] >= 0.f ? d5m(v) : d5p(v));
    }
    const float p0 = C.phi[fc];
    if (stage == 1) C.p1[fc] = p0 + rhs;
    else if (stage == 2) C.p2[fc] = 0.75f * p0 + 0.25f * (C.p1[fc] + rhs);
    else C.phi[fc] = p0 / 3.0f + (2.0f / 3.0f) * (C.p2[fc] + rhs);
  }
}

// Reinitialisation stage (as d_reinit_stage); with prep set (first stage of the first
// pseudo step) it also finds the frozen cells and S(phi0) as d_reinit_prep does.
// Frozen cells leave phi as it is and write it into the stage array of stages 1, 2.
template <int Q>
__global__ void __launch_bounds__(512, LSB_RE_MINB) k_reinit_mirror(Ctx C, BlockShape S, int glevel, int stage,
                                                                    int prep) {
  LSB_GRID_WAIT();
  using LT = Lat<Q>;
  constexpr int D = LT::D;
  const int nl = min(C.counters[glevel * NCOUNT + 3], C.band_cap);
  const float *pin = stage == 1 ? C.phi : (stage == 2 ? C.p1 : C.p2);
  // the next entry of the band list is loaded while this one is processed
  const int4 *info = C.band_info + (long long)glevel * C.band_cap;
  int4 next = blockIdx.x < nl ? __ldg(info + blockIdx.x) : make_int4(0, 0, 0, 0);
  for (int w = blockIdx.x; w < nl; w += gridDim.x) {
    const int4 bi = next;
    if (w + gridDim.x < nl) next = __ldg(info + w + gridDim.x);
    int x, y, z;
    const LevelDev &L = band_cell_at(C, S, bi, threadIdx.x, x, y, z);
    if (!L.ls_active) continue;
    if (x >= L.n[0] || y >= L.n[1] || z >= L.n[2]) continue;
    const unsigned cl = (unsigned)cidx(L, x, y, z);
    const long long fc = L.fine_off + cl;
    const float p0 = C.phi[fc];
    bool fr;
    float s0;
    if (prep) {
      const bool g = p0 >= 0.f;
      fr = false;
      const bool inner = x >= 1 && x + 1 < L.n[0] && y >= 1 && y + 1 < L.n[1] && (D == 2 || (z >= 1 && z + 1 < L.n[2]));
      if (inner) {
        const int q0 = L.p[0], q01 = L.p[0] * L.p[1];
#pragma unroll
        for (int i = 0; i < Q; ++i) {
          if (i == LT::REST) continue;
          if ((C.phi[fc + LT::cx(i) + LT::cy(i) * q0 + LT::cz(i) * q01] >= 0.f) != g) fr = true;
        }
      } else {
        for (int i = 0; i < Q; ++i) {
          if (i == LT::REST) continue;
          int tx = x + LT::cx(i), ty = y + LT::cy(i), tz = z + LT::cz(i);
          if (!(wrap(L, 0, tx) && wrap(L, 1, ty) && (D == 2 || wrap(L, 2, tz)))) continue;
          if ((C.phi[L.fine_off + cidx(L, tx, ty, tz)] >= 0.f) != g) fr = true;
        }
      }
      s0 = p0 / sqrtf(p0 * p0 + 1.0f);
      C.frozen[fc] = fr ? 1 : 0;
      C.s0[fc] = s0;
    } else {
      fr = C.frozen[fc] != 0;
      s0 = C.s0[fc];
    }
    if (fr) {
      if (stage == 1) C.p1[fc] = p0;
      else if (stage == 2) C.p2[fc] = p0;
      continue;
    }
    const float *pinL = pin + L.fine_off;
    float g2 = 0.f;
    for (int a = 0; a < D; ++a) {
      float v[7];
      gather7m(L, pinL, x, y, z, cl, a, v);
      const float dm = weno5(v[1] - v[0], v[2] - v[1], v[3] - v[2], v[4] - v[3], v[5] - v[4]);
      const float dp = weno5(v[6] - v[5], v[5] - v[4], v[4] - v[3], v[3] - v[2], v[2] - v[1]);
      float ga;
      if (s0 > 0.f) ga = fmaxf(fmaxf(dm, 0.f) * fmaxf(dm, 0.f), fminf(dp, 0.f) * fminf(dp, 0.f));
      else ga = fmaxf(fminf(dm, 0.f) * fminf(dm, 0.f), fmaxf(dp, 0.f) * fmaxf(dp, 0.f));
      g2 += ga;
    }
    const float rhs = L.dtau_reinit * (-s0 * (sqrtf(g2) - 1.0f));
    if (stage == 1) C.p1[fc] = p0 + rhs;
    else if (stage == 2) C.p2[fc] = 0.75f * p0 + 0.25f * (C.p1[fc] + rhs);
    else C.phi[fc] = p0 / 3.0f + (2.0f / 3.0f) * (C.p2[fc] + rhs);
  }
}

// ------------------------------------------------------------------ persistent level-set phase
// The whole level-set update of a finest level (extension, transport,
// reinitialisation: up to 16 dependent passes over the band list) as one
// cooperative launch, with a grid barrier between passes.  The barrier spins
// with an iteration limit: on expiry the block sets ERR_TIMEOUT and returns, so
// a barrier that cannot complete ends the kernel instead of hanging it (the
// cooperative launch makes every CTA resident, so this does not happen in
// normal operation).  bar: two words, arrival count and generation, zero at rest
// (cleared before every launch).  limit: sleeps of ~64 ns before giving up (the
// handle's wait limit, 2^22 ~ 0.3 s by default; 0 gives up at the first wait).
__device__ __forceinline__ bool grid_barrier(unsigned *bar, int *err, long long limit) {
  __shared__ int abort_flag;
  __syncthreads();
  if (threadIdx.x == 0) {
    abort_flag = 0;
    volatile unsigned *vgen = bar + 1;
    const unsigned gen = *vgen;
    __threadfence();
    const unsigned arrived = atomicAdd(bar, 1u) + 1u;
    if (arrived == gridDim.x) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      long long it = 0;
      while (*vgen == gen) {
        if (++it > limit) {
          atomicOr(err, ERR_TIMEOUT);
          abort_flag = 1;
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
  }
  __syncthreads();
  return abort_flag == 0;
}

template <int Q>
__global__ void k_levelset_persistent(Ctx C, BlockShape S, int glevel, int n_ext, int reinit, int n_reinit,
                                      unsigned *bar, long long limit) {
  LSB_GRID_WAIT();
  constexpr int D = Lat<Q>::D;
  d_ext_init<Q>(C, glevel, 0, gridDim.x);
  if (!grid_barrier(bar, C.err, limit)) return;
  const float *uin = C.ut0;
  for (int it = 0; it < n_ext; ++it) {
    float *uout = (it & 1) ? C.ut2 : C.ut1;
    d_ext_iter<D>(C, S, glevel, uin, uout, it == 0 ? 2 : 3);
    if (!grid_barrier(bar, C.err, limit)) return;
    uin = uout;
  }
  if (n_ext > 0) {
    d_ext_iter<D>(C, S, glevel, uin, nullptr, 1);
    if (!grid_barrier(bar, C.err, limit)) return;
  }
  for (int st = 1; st <= 3; ++st) {
    d_adv_stage<D>(C, S, glevel, st);
    if (!grid_barrier(bar, C.err, limit)) return;
  }
  if (reinit) {
    d_reinit_prep<Q>(C, S, glevel);
    if (!grid_barrier(bar, C.err, limit)) return;
    for (int r = 0; r < n_reinit; ++r)
      for (int st = 1; st <= 3; ++st) {
        d_reinit_stage<D>(C, S, glevel, st);
        if (!grid_barrier(bar, C.err, limit)) return;
      }
  }
}

// ------------------------------------------------------------------ refill (Sec. 2.4)
template <int Q>
__device__ __forceinline__ void moments_q(const float *f, float &drho, float u[3]) {
  using LT = Lat<Q>;
  float d = 0.f, jx = 0.f, jy = 0.f, jz = 0.f;
  for (int i = 0; i < Q; ++i) {
    d += f[i];
    jx += LT::cx(i) * f[i];
    jy += LT::cy(i) * f[i];
    jz += LT::cz(i) * f[i];
  }
  drho = d;
  const float inv = 1.0f / (1.0f + d);
  u[0] = jx * inv; u[1] = jy * inv; u[2] = jz * inv;
}

template <int Q>
__device__ __forceinline__ float feq_q(int i, float drho, const float u[3]) {
  using LT = Lat<Q>;
  const float cu = LT::cx(i) * u[0] + LT::cy(i) * u[1] + LT::cz(i) * u[2];
  const float usq = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
  return LT::w(i) * (drho + (1.0f + drho) * (3.0f * cu + 4.5f * cu * cu - 1.5f * usq));
}

// Refill of one flipped cell (its normal and curvature already fitted).
template <int Q, typename T>
__device__ __forceinline__ void refill_cell(const Ctx &C, int2 it) {
  using LT = Lat<Q>;
  constexpr int D = LT::D;
  {
    const LevelDev &L = C.lds[it.x];
    const long long c = it.y;
    int x, y, z;
    cell_xyz(L, c, x, y, z);
    const long long fo = L.fine_off, NF = C.nfine, N = L.ncell;
    T *Bf = fB<T, Q>(C, L);
    const uint8_t tg = C.tag[L.cell_off + c];
    const int Pn = tg & TAG_GAS;
    const int Po = (tg & TAG_PREVGAS) ? 1 : 0;
    const float sg = Pn == 0 ? 1.0f : -1.0f;
    float mvec[3] = {0.f, 0.f, 0.f};
    for (int a = 0; a < D; ++a) mvec[a] = -sg * C.nvec[a * NF + fo + c];  // into the new phase
    auto valid_new = [&](int tx, int ty, int tz, long long &ct) -> bool {
      if (!(wrap(L, 0, tx) && wrap(L, 1, ty) && (D == 2 || wrap(L, 2, tz)))) return false;
      ct = cidx(L, tx, ty, tz);
      const uint8_t tt = C.tag[L.cell_off + ct];
      const int g = tt & TAG_GAS, pg = (tt & TAG_PREVGAS) ? 1 : 0;
      return (tt & TAG_LEAF) && g == Pn && pg == Pn;
    };
    int best = -1;
    float bestv = -1e30f;
    for (int i = 0; i < Q; ++i) {
      if (i == LT::REST) continue;
      long long ct;
      if (!valid_new(x + LT::cx(i), y + LT::cy(i), z + LT::cz(i), ct)) continue;
      const float nrm = sqrtf((float)(LT::cx(i) * LT::cx(i) + LT::cy(i) * LT::cy(i) + LT::cz(i) * LT::cz(i)));
      const float v = (LT::cx(i) * mvec[0] + LT::cy(i) * mvec[1] + LT::cz(i) * mvec[2]) / nrm;
      if (v > bestv) {
        bestv = v;
        best = i;
      }
    }
    if (best < 0) {
      for (int i = 0; i < Q; ++i) Store<T>::st(Bf + i * N + c, 0.0f, C.fp16_scale);
      return;
    }
    const int ex = LT::cx(best), ey = LT::cy(best), ez = LT::cz(best);
    const float phr = C.phi[fo + c];
    float q = 0.5f;
    {
      int bx = x - ex, by = y - ey, bz = z - ez;
      if (wrap(L, 0, bx) && wrap(L, 1, by) && (D == 2 || wrap(L, 2, bz))) {
        const long long cb = cidx(L, bx, by, bz);
        if ((C.tag[L.cell_off + cb] & TAG_GAS) != Pn) q = phr / (phr - C.phi[fo + cb]);
      }
    }
    long long c1 = 0, c2 = 0;
    valid_new(x + ex, y + ey, z + ez, c1);
    const bool quad = valid_new(x + 2 * ex, y + 2 * ey, z + 2 * ez, c2);
    float w0, w1, w2;
    if (quad) {
      w0 = 2.0f / ((q + 1.0f) * (q + 2.0f));
      w1 = 2.0f * q / (q + 1.0f);
      w2 = -q / (q + 2.0f);
    } else {
      w0 = 1.0f / (1.0f + q);
      w1 = q / (1.0f + q);
      w2 = 0.0f;
    }
    float fo_[Q], f1[Q];
    for (int i = 0; i < Q; ++i) {
      fo_[i] = Store<T>::ld(Bf + i * N + c, C.fp16_inv);
      f1[i] = Store<T>::ld(Bf + i * N + c1, C.fp16_inv);
    }
    float r_old, u_old[3], r1, u1[3];
    moments_q<Q>(fo_, r_old, u_old);
    moments_q<Q>(f1, r1, u1);
    const float p_gamma = L.rho_phys[Po] * CS2 * r_old + L.sigma * sg * C.kappa[fo + c];
    const float r_g = p_gamma / (L.rho_phys[Pn] * CS2);
    float rr = w0 * r_g + w1 * r1;
    float ur[3];
    for (int a = 0; a < 3; ++a) ur[a] = w0 * u_old[a] + w1 * u1[a];
    if (quad) {
      float f2[Q], r2, u2[3];
      for (int i = 0; i < Q; ++i) f2[i] = Store<T>::ld(Bf + i * N + c2, C.fp16_inv);
      moments_q<Q>(f2, r2, u2);
      rr += w2 * r2;
      for (int a = 0; a < 3; ++a) ur[a] += w2 * u2[a];
    }
    for (int i = 0; i < Q; ++i) {
      const float v = feq_q<Q>(i, rr, ur) + (f1[i] - feq_q<Q>(i, r1, u1));
      Store<T>::st(Bf + i * N + c, v, C.fp16_scale);
    }
  }
}

// The classification's last passes in one launch: the curvature fit of the interface and
// flipped cells (CTAs [0, gg): the longer chain per thread, scheduled first) and the band
// (the rest, a warp per finest block), which read nothing of each other's; with refill
// set, each flipped cell is refilled by the thread that fitted it (the refill reads the
// fit at its own cell only, and neighbours of the new phase that did not flip).
template <int Q, typename T>
__global__ void k_post_classify(Ctx C, const int *list, int nlist, int glevel, int gg, int refill) {
  LSB_GRID_WAIT();
  constexpr int D = Lat<Q>::D;
  if ((int)blockIdx.x >= gg) {
    d_band<Q>(C, list, nlist, glevel, gg, (int)gridDim.x - gg);
  } else if (refill) {
    d_geometry<D>(C, glevel, 2, 0, gg, [&](int2 it) { refill_cell<Q, T>(C, it); });
  } else {
    d_geometry<D>(C, glevel, 2, 0, gg, [](int2) {});
  }
}

// ------------------------------------------------------------------ refinement sensor
// Per listed coarse block: min |phi| (mode 0) or max phi (mode 1) over the
// finest cells under it.
__global__ void k_sensor(Ctx C, BlockShape S, const int *list, int nlist, int mode, float *out) {
  LSB_GRID_WAIT();
  __shared__ float red[32];
  for (int w = blockIdx.x; w < nlist; w += gridDim.x) {
    const int gb = list[w];
    const LevelDev &L = C.lds[C.blk_ld[gb]];
    const LevelDev &F = C.lds[L.fine_ld];
    const int lb = gb - L.block_off;
    const int b[3] = {lb % L.nb[0], (lb / L.nb[0]) % L.nb[1], lb / (L.nb[0] * L.nb[1])};
    int lo[3], hi[3];
    for (int a = 0; a < 3; ++a) {
      lo[a] = b[a] * S.bs[a] * L.scale;
      hi[a] = min((b[a] + 1) * S.bs[a], L.n[a]) * L.scale;
      hi[a] = min(hi[a], F.n[a]);
    }
    const long long cnt = (long long)(hi[0] - lo[0]) * (hi[1] - lo[1]) * (hi[2] - lo[2]);
    float acc = mode == 0 ? 3.0e38f : -3.0e38f;
    for (long long e = threadIdx.x; e < cnt; e += blockDim.x) {
      const int sx = hi[0] - lo[0], sy = hi[1] - lo[1];
      const int x = lo[0] + (int)(e % sx);
      const int y = lo[1] + (int)((e / sx) % sy);
      const int z = lo[2] + (int)(e / ((long long)sx * sy));
      const float p = C.phi[F.fine_off + cidx(F, x, y, z)];
      acc = mode == 0 ? fminf(acc, fabsf(p)) : fmaxf(acc, p);
    }
    for (int off = 16; off > 0; off >>= 1) {
      const float o = __shfl_down_sync(0xffffffffu, acc, off);
      acc = mode == 0 ? fminf(acc, o) : fmaxf(acc, o);
    }
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
      float r = red[0];
      for (int k = 1; k < (int)(blockDim.x + 31) / 32; ++k) r = mode == 0 ? fminf(r, red[k]) : fmaxf(r, red[k]);
      out[w] = r;
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------------ host launchers
#define LQ(kern, ...)                                                          \
  do {                                                                         \
    if (Q == 9) launcher(kern<9>, L, 0)(__VA_ARGS__);        \
    else if (Q == 19) launcher(kern<19>, L, 0)(__VA_ARGS__); \
    else launcher(kern<27>, L, 0)(__VA_ARGS__);              \
    return cudaGetLastError();                                                 \
  } while (0)
#define LD(kern, ...)                                                          \
  do {                                                                         \
    if (D == 2) launcher(kern<2>, L, 0)(__VA_ARGS__);        \
    else launcher(kern<3>, L, 0)(__VA_ARGS__);               \
    return cudaGetLastError();                                                 \
  } while (0)
// Same for a band-list kernel, with the grid capped at the resident CTAs.
#define LDP(kern, ...)                                                                             \
  do {                                                                                             \
    if (D == 2) launcher(kern<2>, with_grid(L, resident_grid(kern<2>, L.block, L.grid)))(__VA_ARGS__); \
    else launcher(kern<3>, with_grid(L, resident_grid(kern<3>, L.block, L.grid)))(__VA_ARGS__);        \
    return cudaGetLastError();                                                                     \
  } while (0)
#define LQP(kern, ...)                                                                             \
  do {                                                                                             \
    if (Q == 9) launcher(kern<9>, with_grid(L, resident_grid(kern<9>, L.block, L.grid)))(__VA_ARGS__); \
    else if (Q == 19) launcher(kern<19>, with_grid(L, resident_grid(kern<19>, L.block, L.grid)))(__VA_ARGS__); \
    else launcher(kern<27>, with_grid(L, resident_grid(kern<27>, L.block, L.grid)))(__VA_ARGS__);      \
    return cudaGetLastError();                                                                     \
  } while (0)

// Band-list kernels walk a device-sized list with a block-stride loop; their grid
// is capped at the CTAs resident at once (152 SMs x CTAs per SM for this kernel and
// block size), so no wave of CTAs starts only to find the list exhausted.
template <typename K>
int resident_grid(K kern, int block, int want) {
  static std::mutex mu;
  static std::map<std::pair<const void *, int>, int> cache;  // (kernel, block) -> resident CTAs
  const std::pair<const void *, int> key{reinterpret_cast<const void *>(kern), block};
  std::lock_guard<std::mutex> lock(mu);
  auto it = cache.find(key);
  if (it == cache.end()) {
    int n = 1, dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, block, 0) != cudaSuccess || n < 1) n = 1;
    it = cache.emplace(key, n * sms).first;
  }
  return want < it->second ? want : it->second;
}

cudaError_t run_classify_phase(int Q, Launch L, Ctx C, BlockShape S, const int *list, int n, int glevel, int init) {
  LQ(k_classify_phase, C, S, list, n, glevel, init);
}
cudaError_t run_classify_links(int Q, Launch L, Ctx C, BlockShape S, const int *list, int n, int glevel, int full) {
  LQ(k_classify_links, C, S, list, n, glevel, full);
}
cudaError_t run_geometry(int D, Launch L, Ctx C, int glevel, int which) { LD(k_geometry, C, glevel, which); }
cudaError_t run_ext_init(int Q, Launch L, Ctx C, int glevel) { LQ(k_ext_init, C, glevel); }
cudaError_t run_ext_iter(int D, Launch L, Ctx C, BlockShape S, int glevel, const float *uin, float *uout, int mode) {
  if (mode == 3) LDP(k_ext_plan, C, S, glevel, uin, uout);
  LDP(k_ext_iter, C, S, glevel, uin, uout, mode);
}
cudaError_t run_adv_stage(int D, Launch L, Ctx C, BlockShape S, int glevel, int stage) {
  LDP(k_adv_stage, C, S, glevel, stage);
}
cudaError_t run_ext_first(int D, Launch L, Ctx C, BlockShape S, int glevel, const float *uin, float *uout,
                          int turn) {
  LDP(k_ext_first, C, S, glevel, uin, uout, turn);
}
cudaError_t run_ext_sweep_mirror(int D, Launch L, Ctx C, BlockShape S, int glevel, const float *uin, float *uout) {
  if (D == 2)
    launcher(k_ext_plan<2, true>, with_grid(L, resident_grid(k_ext_plan<2, true>, L.block, L.grid)))(C, S, glevel, uin,
                                                                                                      uout);
  else
    launcher(k_ext_plan<3, true>, with_grid(L, resident_grid(k_ext_plan<3, true>, L.block, L.grid)))(C, S, glevel, uin,
                                                                                                      uout);
  return cudaGetLastError();
}
cudaError_t run_adv_mirror(int D, Launch L, Ctx C, BlockShape S, int glevel, int stage, const float *ufin) {
  LDP(k_adv_mirror, C, S, glevel, stage, ufin);
}
cudaError_t run_reinit_mirror(int Q, Launch L, Ctx C, BlockShape S, int glevel, int stage, int prep) {
  LQP(k_reinit_mirror, C, S, glevel, stage, prep);
}
cudaError_t run_reinit_prep(int Q, Launch L, Ctx C, BlockShape S, int glevel) { LQP(k_reinit_prep, C, S, glevel); }
cudaError_t run_reinit_stage(int D, Launch L, Ctx C, BlockShape S, int glevel, int stage) {
  LDP(k_reinit_stage, C, S, glevel, stage);
}
cudaError_t run_post_classify(int Q, int st, Launch L, Ctx C, const int *list, int n, int glevel, int gg,
                              int refill) {
  if (Q == 9) {
    if (st == 0) launcher(k_post_classify<9, float>, L, 0)(C, list, n, glevel, gg, refill);
    else launcher(k_post_classify<9, __half>, L, 0)(C, list, n, glevel, gg, refill);
  } else if (Q == 19) {
    if (st == 0) launcher(k_post_classify<19, float>, L, 0)(C, list, n, glevel, gg, refill);
    else launcher(k_post_classify<19, __half>, L, 0)(C, list, n, glevel, gg, refill);
  } else {
    if (st != 0) return cudaErrorInvalidValue;  // D3Q27: FP32 storage only
    launcher(k_post_classify<27, float>, L, 0)(C, list, n, glevel, gg, refill);
  }
  return cudaGetLastError();
}
cudaError_t run_sensor(Launch L, Ctx C, BlockShape S, const int *list, int n, int mode, float *out) {
  launcher(k_sensor, L, 0)(C, S, list, n, mode, out);
  return cudaGetLastError();
}

// One cooperative launch of the level-set phase; grid = resident CTAs (required
// for a cooperative launch, which fails rather than oversubscribe).
cudaError_t run_levelset_persistent(int Q, Launch L, Ctx C, BlockShape S, int glevel, int n_ext, int reinit,
                                    int n_reinit, unsigned *bar, long long limit) {
  void *args[] = {&C, &S, &glevel, &n_ext, &reinit, &n_reinit, &bar, &limit};
  if (Q == 9) {
    const int grid = resident_grid(k_levelset_persistent<9>, L.block, L.grid);
    return cudaLaunchCooperativeKernel((const void *)k_levelset_persistent<9>, grid, L.block, args, 0, L.stream);
  }
  if (Q == 19) {
    const int grid = resident_grid(k_levelset_persistent<19>, L.block, L.grid);
    return cudaLaunchCooperativeKernel((const void *)k_levelset_persistent<19>, grid, L.block, args, 0, L.stream);
  }
  const int grid = resident_grid(k_levelset_persistent<27>, L.block, L.grid);
  return cudaLaunchCooperativeKernel((const void *)k_levelset_persistent<27>, grid, L.block, args, 0, L.stream);
}

}  // namespace lsb
