// Device-side definitions shared by the lsb kernels: velocity sets (Sec. 2.1,
// Fig. 1), level descriptors of the block-structured grid, storage of the
// populations as deviations from the rest weights (FP32 or scaled FP16).
#pragma once
#include <cuda_fp16.h>
#include <stdint.h>

namespace lsb {

constexpr float CS2 = 1.0f / 3.0f;

// ---------------------------------------------------------------- lattices
// D2Q9 ordering of Fig. 1a: -x, +x, -y, +y, (-1,-1), (-1,1), (1,1), (1,-1), rest.
// D3Q19: the axis and edge velocities of Fig. 1b in that order, rest last.
// First statement of every kernel of the step: wait for the grid the kernel depends
// on (and its memory) when it was launched as a programmatic dependent, then let the
// next kernel on the stream be scheduled.  Both are no-ops for an ordinary launch.
#define LSB_GRID_WAIT() asm volatile("griddepcontrol.wait;\n\tgriddepcontrol.launch_dependents;" ::: "memory")

template <int Q> struct Lat;

template <> struct Lat<9> {
  static constexpr int D = 2;
  static constexpr int REST = 8;
  __host__ __device__ static constexpr int cx(int i) {
    return (i == 0 || i == 4 || i == 5) ? -1 : ((i == 1 || i == 6 || i == 7) ? 1 : 0);
  }
  __host__ __device__ static constexpr int cy(int i) {
    return (i == 2 || i == 4 || i == 7) ? -1 : ((i == 3 || i == 5 || i == 6) ? 1 : 0);
  }
  __host__ __device__ static constexpr int cz(int) { return 0; }
  __host__ __device__ static constexpr float w(int i) {
    return i < 4 ? 1.0f / 9.0f : (i < 8 ? 1.0f / 36.0f : 4.0f / 9.0f);
  }
  __host__ __device__ static constexpr int opp(int i) {
    return i == 8 ? 8 : (i < 4 ? (i ^ 1) : (i < 6 ? i + 2 : i - 2));
  }
};

template <> struct Lat<19> {
  static constexpr int D = 3;
  static constexpr int REST = 18;
  // axis: 0 -x, 1 +x, 2 -y, 3 +y, 4 -z, 5 +z
  // edges: 6 (-1,-1,0) 7 (-1,1,0) 8 (1,-1,0) 9 (1,1,0)
  //        10 (-1,0,-1) 11 (-1,0,1) 12 (1,0,-1) 13 (1,0,1)
  //        14 (0,-1,-1) 15 (0,-1,1) 16 (0,1,-1) 17 (0,1,1)
  __host__ __device__ static constexpr int cx(int i) {
    return (i == 0 || (i >= 6 && i <= 7) || (i >= 10 && i <= 11)) ? -1
         : ((i == 1 || (i >= 8 && i <= 9) || (i >= 12 && i <= 13)) ? 1 : 0);
  }
  __host__ __device__ static constexpr int cy(int i) {
    return (i == 2 || i == 6 || i == 8 || i == 14 || i == 15) ? -1
         : ((i == 3 || i == 7 || i == 9 || i == 16 || i == 17) ? 1 : 0);
  }
  __host__ __device__ static constexpr int cz(int i) {
    return (i == 4 || i == 10 || i == 12 || i == 14 || i == 16) ? -1
         : ((i == 5 || i == 11 || i == 13 || i == 15 || i == 17) ? 1 : 0);
  }
  __host__ __device__ static constexpr float w(int i) {
    return i < 6 ? 1.0f / 18.0f : (i < 18 ? 1.0f / 36.0f : 1.0f / 3.0f);
  }
  __host__ __device__ static constexpr int opp(int i) {
    return i == 18 ? 18
         : (i < 6 ? (i ^ 1)
         : (i < 10 ? 15 - i : (i < 14 ? 23 - i : 31 - i)));
  }
};

template <> struct Lat<27> {
  static constexpr int D = 3;
  static constexpr int REST = 26;
  // axis and edge velocities as D3Q19 (0..17); corners 18..25: 18 + 4 [cx > 0] + 2 [cy > 0] + [cz > 0]
  __host__ __device__ static constexpr int cx(int i) {
    return i < 18 ? Lat<19>::cx(i) : (i < 26 ? (((i - 18) & 4) ? 1 : -1) : 0);
  }
  __host__ __device__ static constexpr int cy(int i) {
    return i < 18 ? Lat<19>::cy(i) : (i < 26 ? (((i - 18) & 2) ? 1 : -1) : 0);
  }
  __host__ __device__ static constexpr int cz(int i) {
    return i < 18 ? Lat<19>::cz(i) : (i < 26 ? (((i - 18) & 1) ? 1 : -1) : 0);
  }
  __host__ __device__ static constexpr float w(int i) {
    return i < 6 ? 2.0f / 27.0f : (i < 18 ? 1.0f / 54.0f : (i < 26 ? 1.0f / 216.0f : 8.0f / 27.0f));
  }
  __host__ __device__ static constexpr int opp(int i) { return i < 18 ? Lat<19>::opp(i) : (i < 26 ? 43 - i : 26); }
};

// The direction c_i with the components of the axes in bit mask m negated: the
// direction a population leaves a slip wall with (specular reflection).
template <int Q>
__host__ __device__ __forceinline__ int mirror_dir(int i, int m) {
  using LT = Lat<Q>;
  const int x = (m & 1) ? -LT::cx(i) : LT::cx(i);
  const int y = (m & 2) ? -LT::cy(i) : LT::cy(i);
  const int z = (m & 4) ? -LT::cz(i) : LT::cz(i);
  int r = i;
#pragma unroll
  for (int j = 0; j < Q; ++j)
    if (LT::cx(j) == x && LT::cy(j) == y && LT::cz(j) == z) r = j;
  return r;
}

// ---------------------------------------------------------------- moments and equilibrium
// Eq. macro on deviations f~ = f - w: drho = sum f~, u = sum c f~ / (1 + drho).
template <int Q>
__device__ __forceinline__ void lb_moments(const float *f, float &drho, float u[3]) {
  using LT = Lat<Q>;
  float d = 0.f, jx = 0.f, jy = 0.f, jz = 0.f;
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    d += f[i];
    jx += LT::cx(i) * f[i];
    jy += LT::cy(i) * f[i];
    if (LT::D == 3) jz += LT::cz(i) * f[i];
  }
  float inv = 1.0f / (1.0f + d);
  drho = d;
  u[0] = jx * inv;
  u[1] = jy * inv;
  u[2] = jz * inv;
}

// Deviation of Eq. feq from the rest weights: f~eq_i = feq_i - w_i.
template <int Q>
__device__ __forceinline__ float feq_dev(int i, float drho, const float u[3], float usq) {
  using LT = Lat<Q>;
  float cu = LT::cx(i) * u[0] + LT::cy(i) * u[1] + LT::cz(i) * u[2];
  return LT::w(i) * (drho + (1.0f + drho) * (3.0f * cu + 4.5f * cu * cu - 1.5f * usq));
}

// ---------------------------------------------------------------- grid descriptors
enum : int8_t { BLK_INACTIVE = 0, BLK_LEAF = 1, BLK_REFINED = 2 };

// per-cell tag bits
enum : uint8_t {
  TAG_GAS = 1,      // current phase (1 gas, 0 liquid)
  TAG_IFACE = 2,    // finest level: has a cut incoming link
  TAG_FLIP = 4,     // changed phase at the last classification
  TAG_PREVGAS = 8,  // phase before the last classification
  TAG_RLAYER = 16,  // covered cell a leaf streams from (fine-to-coarse target)
  TAG_GHOST = 32,   // inactive cell a leaf streams from (coarse-to-fine target)
  TAG_LEAF = 64,    // cell of a leaf block inside the box
  TAG_CCUT = 128    // coarser level: a lattice neighbour (not a ghost cell) has the other phase;
                    // pushes towards it bounce back into the cell's own opposite population
};

// per-block flag bits (finest level)
// BF_CHECK lives only between the phase and link passes of a classification: blocks
// next to a cell that flipped outside the previous band (whose blocks still hold BF_BAND
// until the link pass rewrites the flags).
enum : uint8_t { BF_IFACE = 1, BF_BAND = 2, BF_CHECK = 8 };

struct LevelDev {
  int case_id, level, n_levels, finest;
  int n[3];        // true cells per axis (n[2] = 1 in 2D)
  int p[3];        // padded to whole blocks
  int nb[3];       // blocks per axis
  int per[3];      // periodic axis flags
  int slip[3];     // walled axes with slip walls (specular reflection)
  int cumulant[2]; // per phase: cumulant collision (D3Q27) instead of BGK
  long long ncell; // p0*p1*p2
  long long cell_off;  // offset in per-cell arrays of all levels (f uses *Q)
  long long fine_off;  // offset in finest-level arrays, -1 if not finest
  int block_off, nblock;
  int parent_ld, child_ld;
  int scale;       // finest cells per cell edge of this level: 2^(n_levels-1-level)
  int fine_ld;     // level descriptor of this case's finest level
  float omega[2], tau[2];
  float acc[2][3];     // lattice acceleration per phase at this level
  float wall_u[6][3];  // face velocities
  // case physics needed on the finest level
  float rho_phys[2], eta[2], sigma;
  float dtau_ext, dtau_reinit;
  float x_ref[3], grav[3];
  float p_gas0;
  int ls_active;
};

struct Ctx {
  const LevelDev *lds;
  const int *blk_ld;       // global block id -> level descriptor
  const int4 *blk_info;    // global block id -> (level descriptor, block x, y, z)
  int8_t *bstat;           // block status (per global block)
  int8_t *bstat_old;       // previous status during regrid
  uint8_t *bflag;          // finest-level block flags
  uint8_t *tag;            // per cell, all levels
  void *buf[2];            // two population buffers; level l reads buf[par[l]] (state A)
  int par[4];              // and writes buf[1 - par[l]] (state B); SoA by q at cell_off*Q
  // finest-level arrays (indexed fine_off + cell)
  float *phi, *p1, *p2, *s0;
  uint8_t *frozen;
  float *ut0, *ut1, *ut2;  // extension velocity (D planes of nfine each)
  float *plan_v;           // extension plan: upwind velocity (D planes of nfine)
  uint8_t *plan_f;         // extension plan: side / band / interface / boundary bits
  uint32_t *cmask;
  int *cbase;
  float *macro;            // MF planes of nfine: drho, u[D], S (sym, D(D+1)/2)
  float *nvec, *kappa;     // geometry at interface cells (D planes + 1)
  float *linkbuf;          // 2 floats per cut link
  int2 *link_cell;         // per cut link: (level descriptor, cell) of x
  uint8_t *link_dir;       // per cut link: incoming direction k
  long long link_list_off[4];  // start of each finest global level's region of the link list
  long long nfine;         // finest-level cells over all cases
  long long link_cap;
  int *counters;           // per global level: [0] links, [1] iface cells, [2] flipped, [3] band blocks
  int2 *iface_list, *flip_list;   // (ld, cell)
  int *band_list;          // global block ids
  int *check_list;         // blocks next to a flipped cell outside the previous band
  int4 *band_info;         // beside each band-list entry: its block coordinates (as blk_info)
  long long list_cap;      // capacity of iface/flip lists per global level
  int band_cap;
  int *err;                // latched error bits
  float fp16_scale, fp16_inv;
};

enum : int { ERR_LINK_OVF = 1, ERR_LIST_OVF = 2, ERR_NONFINITE = 4, ERR_BAND_OVF = 8, ERR_TIMEOUT = 16 };
// device counters per global level: [0] cut links, [1] interface cells, [2] flipped cells,
// [3] band blocks, [4] blocks next to a flipped cell outside the previous band (check
// list), [5] band blocks of the previous classification (the band list it left)
constexpr int NCOUNT = 6;

// ---------------------------------------------------------------- storage
template <typename T> struct Store;
template <> struct Store<float> {
  __device__ static __forceinline__ float ld(const float *p, float) { return __ldg(p); }
  __device__ static __forceinline__ void st(float *p, float v, float) { *p = v; }
};
template <> struct Store<__half> {
  __device__ static __forceinline__ float ld(const __half *p, float inv) {
    return __half2float(__ldg(p)) * inv;
  }
  __device__ static __forceinline__ void st(__half *p, float v, float scale) {
    *p = __float2half_rn(v * scale);
  }
};

struct BlockShape {
  int bs[3];  // block edge per axis (powers of two)
  int lg[3];  // log2 of the edges
};

// Population state A (pre-collision, time t) and B (destination of the push) of a level.
template <typename T, int Q>
__device__ __forceinline__ T *fA(const Ctx &C, const LevelDev &L) {
  return reinterpret_cast<T *>(C.buf[C.par[L.level]]) + L.cell_off * Q;
}
template <typename T, int Q>
__device__ __forceinline__ T *fB(const Ctx &C, const LevelDev &L) {
  return reinterpret_cast<T *>(C.buf[1 - C.par[L.level]]) + L.cell_off * Q;
}

// ---------------------------------------------------------------- indexing helpers
__device__ __forceinline__ void block_cell(const LevelDev &L, int lb, int t, const int bs[3], int &x,
                                           int &y, int &z) {
  int bx = lb % L.nb[0];
  int by = (lb / L.nb[0]) % L.nb[1];
  int bz = lb / (L.nb[0] * L.nb[1]);
  int tx = t % bs[0];
  int ty = (t / bs[0]) % bs[1];
  int tz = t / (bs[0] * bs[1]);
  x = bx * bs[0] + tx;
  y = by * bs[1] + ty;
  z = bz * bs[2] + tz;
}

// Same with power-of-two block edges (shifts and masks for the thread part).
__device__ __forceinline__ void block_cell2(const LevelDev &L, int lb, int t, const BlockShape &S, int &x,
                                            int &y, int &z) {
  const int nb0 = L.nb[0], nb1 = L.nb[1];
  const int q0 = lb / nb0;
  const int bx = lb - q0 * nb0;
  const int bz = q0 / nb1;
  const int by = q0 - bz * nb1;
  x = (bx << S.lg[0]) + (t & (S.bs[0] - 1));
  y = (by << S.lg[1]) + ((t >> S.lg[0]) & (S.bs[1] - 1));
  z = (bz << S.lg[2]) + (t >> (S.lg[0] + S.lg[1]));
}

__device__ __forceinline__ long long cidx(const LevelDev &L, int x, int y, int z) {
  return (long long)x + (long long)L.p[0] * ((long long)y + (long long)L.p[1] * z);
}

__device__ __forceinline__ int block_of(const LevelDev &L, int x, int y, int z, const BlockShape &S) {
  return (x >> S.lg[0]) + L.nb[0] * ((y >> S.lg[1]) + L.nb[1] * (z >> S.lg[2]));
}

// Level descriptor and cell coordinates of thread t of global block gb.
__device__ __forceinline__ const LevelDev &blk_cell(const Ctx &C, const BlockShape &S, int gb, int t, int &x, int &y,
                                                    int &z) {
  const int4 bi = __ldg(C.blk_info + gb);
  x = (bi.y << S.lg[0]) + (t & (S.bs[0] - 1));
  y = (bi.z << S.lg[1]) + ((t >> S.lg[0]) & (S.bs[1] - 1));
  z = (bi.w << S.lg[2]) + (t >> (S.lg[0] + S.lg[1]));
  return C.lds[bi.x];
}

// Cell (x, y, z) of thread t in band-list entry w of global level glevel: the block
// coordinates come from the copy the band pass stores beside the list, so they do not wait
// on the list entry.
__device__ __forceinline__ const LevelDev &band_cell(const Ctx &C, const BlockShape &S, int glevel, int w, int t,
                                                     int &x, int &y, int &z) {
  const int4 bi = __ldg(C.band_info + (long long)glevel * C.band_cap + w);
  x = (bi.y << S.lg[0]) + (t & (S.bs[0] - 1));
  y = (bi.z << S.lg[1]) + ((t >> S.lg[0]) & (S.bs[1] - 1));
  z = (bi.w << S.lg[2]) + (t >> (S.lg[0] + S.lg[1]));
  return C.lds[bi.x];
}

// The same from a band-list entry already loaded (prefetched one iteration ahead).
__device__ __forceinline__ const LevelDev &band_cell_at(const Ctx &C, const BlockShape &S, int4 bi, int t, int &x,
                                                        int &y, int &z) {
  x = (bi.y << S.lg[0]) + (t & (S.bs[0] - 1));
  y = (bi.z << S.lg[1]) + ((t >> S.lg[0]) & (S.bs[1] - 1));
  z = (bi.w << S.lg[2]) + (t >> (S.lg[0] + S.lg[1]));
  return C.lds[bi.x];
}

// Smoothed gas indicator of the adjoint objective (Sec. 3.2's integrals weighted so
// that they depend smoothly on phi): H(phi) = 1/2 (1 + t + sin(pi t)/pi), t = phi/eps on
// |phi| <= eps, 0 below, 1 above; and its derivative.
__device__ __forceinline__ float smooth_h(float phi, float eps) {
  if (phi >= eps) return 1.0f;
  if (phi <= -eps) return 0.0f;
  const float t = phi / eps;
  return 0.5f * (1.0f + t + sinpif(t) * 0.318309886183790672f);
}
__device__ __forceinline__ float smooth_dh(float phi, float eps) {
  if (phi >= eps || phi <= -eps) return 0.0f;
  return 0.5f / eps * (1.0f + cospif(phi / eps));
}
// phi of the finest cell a leaf of level L reads its indicator at (its first finest child).
__device__ __forceinline__ long long corner_phi_index(const Ctx &C, const LevelDev &L, int x, int y, int z) {
  const LevelDev &F = C.lds[L.fine_ld];
  const int s = L.scale;
  return F.fine_off + cidx(F, x * s, y * s, z * s);
}

// (x, y, z) of level-local cell index c, in 32-bit arithmetic: every level holds fewer
// than 2^32 / (Q + 1) cells (checked when the grid is created).
__device__ __forceinline__ void cell_xyz(const LevelDev &L, long long c, int &x, int &y, int &z) {
  const unsigned u = (unsigned)c, p0 = (unsigned)L.p[0], p1 = (unsigned)L.p[1];
  const unsigned q = u / p0;
  x = (int)(u - q * p0);
  y = (int)(q % p1);
  z = (int)(q / p1);
}

// Wrap a coordinate on a periodic axis; returns false if it leaves through a wall.
__device__ __forceinline__ bool wrap(const LevelDev &L, int a, int &v) {
  int n = L.n[a];
  if (v >= 0 && v < n) return true;
  if (!L.per[a]) return false;
  v = (v % n + n) % n;
  return true;
}

// Clamp (walled axes) or wrap (periodic axes): zero-gradient ghost values.
__device__ __forceinline__ int clampwrap(const LevelDev &L, int a, int v) {
  int n = L.n[a];
  if (L.per[a]) return (v % n + n) % n;
  return v < 0 ? 0 : (v >= n ? n - 1 : v);
}


// ------------------------------------------------------------------ interface velocity
// Interface cells: mean of u_I = (1-q) u(x) + q u(x + c_i) over their cut links, on the
// CTAs [b0, b0 + nb) of the launch (the rest of a shared launch does other work).
template <int Q>
__device__ __forceinline__ void d_ext_init(const Ctx &C, int glevel, int b0, int nb) {
  using LT = Lat<Q>;
  constexpr int D = LT::D;
  const int n = min(C.counters[glevel * NCOUNT + 1], (int)C.list_cap);
  const int2 *lst = C.iface_list + (long long)glevel * C.list_cap;
  for (int e = ((int)blockIdx.x - b0) * blockDim.x + threadIdx.x; e < n; e += nb * blockDim.x) {
    const int2 it = lst[e];
    const LevelDev &L = C.lds[it.x];
    if (!L.ls_active) continue;  // frozen level set in this case
    const long long c = it.y;
    int x, y, z;
    cell_xyz(L, c, x, y, z);
    const long long fo = L.fine_off, NF = C.nfine;
    const uint32_t m = C.cmask[fo + c];
    const float phx = C.phi[fo + c];
    float ux[3];
    for (int a = 0; a < D; ++a) ux[a] = C.macro[(1 + a) * NF + fo + c];
    // the cut links' partners, loaded in groups of four with every load of a group in
    // flight together (a dependent chain per link otherwise), summed in link order
    float acc[3] = {0.f, 0.f, 0.f};
    int cnt = 0;
    uint32_t mm = m;
    while (mm) {
      constexpr int G = 4;
      long long cy[G];
      bool on[G];
#pragma unroll
      for (int j = 0; j < G; ++j) {
        on[j] = mm != 0;
        cy[j] = fo + c;
        if (!on[j]) continue;
        const int k = __ffs(mm) - 1;
        mm &= mm - 1u;
        const int i = LT::opp(k);
        int yx = x + LT::cx(i), yy = y + LT::cy(i), yz = z + LT::cz(i);
        wrap(L, 0, yx); wrap(L, 1, yy); if (D == 3) wrap(L, 2, yz);
        cy[j] = fo + cidx(L, yx, yy, yz);
      }
      float py[G], uy[G][3];
#pragma unroll
      for (int j = 0; j < G; ++j) {
        py[j] = C.phi[cy[j]];
#pragma unroll
        for (int a = 0; a < D; ++a) uy[j][a] = C.macro[(1 + a) * NF + cy[j]];
      }
#pragma unroll
      for (int j = 0; j < G; ++j) {
        if (!on[j]) continue;
        const float q = phx / (phx - py[j]);
        for (int a = 0; a < D; ++a) acc[a] += (1.0f - q) * ux[a] + q * uy[j][a];
        ++cnt;
      }
    }
    for (int a = 0; a < D; ++a) C.ut0[a * NF + fo + c] = acc[a] / (float)cnt;
  }
}

}  // namespace lsb
