// Host launchers of the lsb kernels.  Each is defined in the translation unit
// that defines its kernel (lsb_lb.cu, lsb_ls.cu, lsb_adj.cu), so the launch and the kernel
// registration live together; (Q, storage) pick the template instance.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>

#include "lsb_device.cuh"

namespace lsb {

// Size of the fixed staging array behind lsb_get_fields_noalloc (floats, 16 MiB).
constexpr size_t kNoAllocFloats = size_t(4) << 20;
constexpr int kMaxDevices = 64;

struct Launch {
  int grid, block;
  cudaStream_t stream;
  int pdl = 0;   // programmatic dependent launch: may overlap the previous kernel's tail
  int prio = 0;  // launch priority (0: the stream's; lower numbers are scheduled first)
};

// Launch kern on L's grid and stream.  With L.pdl the launch carries the
// programmatic-stream-serialization attribute: the kernel may be scheduled while
// the kernel before it on the stream finishes, and waits for it (and for its
// memory) in LSB_GRID_WAIT at its start.
template <typename... P, typename... A>
inline void lsb_launch(void (*kern)(P...), const Launch &L, size_t smem, A... args) {
  if (!L.pdl && !L.prio) {
    kern<<<L.grid, L.block, smem, L.stream>>>(args...);
    return;
  }
  cudaLaunchAttribute at[2];
  unsigned na = 0;
  if (L.pdl) {
    at[na].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[na++].val.programmaticStreamSerializationAllowed = 1;
  }
  if (L.prio) {
    at[na].id = cudaLaunchAttributePriority;
    at[na++].val.priority = L.prio;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)L.grid);
  cfg.blockDim = dim3((unsigned)L.block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = L.stream;
  cfg.attrs = at;
  cfg.numAttrs = na;
  cudaLaunchKernelEx(&cfg, kern, args...);
}
template <typename K>
struct Launcher {
  K kern;
  Launch L;
  size_t smem;
  template <typename... A>
  void operator()(A... args) const { lsb_launch(kern, L, smem, args...); }
};
template <typename K>
inline Launcher<K> launcher(K kern, const Launch &L, size_t smem = 0) { return Launcher<K>{kern, L, smem}; }
inline Launch with_grid(Launch L, int grid) {
  L.grid = grid;
  return L;
}

// lsb_lb.cu: lattice Boltzmann, interface bounce-back, level transfers
cudaError_t run_init(int Q, int st, Launch L, Ctx C, BlockShape S, const int *list, int n);
cudaError_t run_collide_stream(int Q, int st, Launch L, Ctx C, BlockShape S, const int *list, int n);
// work: nullptr, or two zeroed counters of this launch's own (dynamic block taking)
cudaError_t run_collide_stream_tma(int Q, int st, Launch L, Ctx C, BlockShape S, const int *list, int n,
                                   const CUtensorMap *tmaps, const CUtensorMap *tmaps_tag, int *work);
size_t tma_smem_bytes(int Q, int st, int nthreads);
cudaError_t prepare_collide_stream_tma(int Q, int st, int nthreads, int *ctas_per_sm);
cudaError_t run_interface_bc(int Q, int st, Launch L, Ctx C, int glevel);
// the interface cells' u~ on CTAs [0, gi) and the interface pass on the rest, one launch
cudaError_t run_iface_init(int Q, int st, Launch L, Ctx C, int glevel, int gi);
cudaError_t run_restrict(int Q, int st, Launch L, Ctx C, BlockShape S, const int *list, int n, int all_cells);
cudaError_t run_prolong(int Q, int st, Launch L, Ctx C, BlockShape S, const int *list, int n);
cudaError_t run_level_tags(int Q, Launch L, Ctx C, BlockShape S, const int *list, int n);
cudaError_t run_collect(Launch L, Ctx C, BlockShape S, const int *list, int n, int bits, int2 *out, int *count,
                        int cap);
cudaError_t run_restrict_cells(int Q, int st, Launch L, Ctx C, const int2 *cells, int n);
cudaError_t run_ghost_cells(int Q, int st, Launch L, Ctx C, const int2 *cells, int n, float theta);
#ifndef LSB_OBS_MINB
#define LSB_OBS_MINB 2  // CTAs of 512 threads per SM k_observables is built for (its grid)
#endif
// tmaps (population maps as for the TMA-staged collide; tmaps_tag optional): the
// TMA-staged kernel (grid at most its resident CTAs); nullptr: per-thread loads
cudaError_t run_observables(int Q, int st, Launch L, Ctx C, BlockShape S, const int *list, int n, double *out,
                            int stride, float eps, const CUtensorMap *tmaps, const CUtensorMap *tmaps_tag);
cudaError_t prepare_observables_tma(int Q, int st, int nthreads, int *ctas_per_sm);
cudaError_t run_export(int Q, int st, Launch L, Ctx C, int ld, int field, float *dst);
// Export into the file-scope staging array; *staged receives its device address.
cudaError_t run_export_noalloc(int Q, int st, Launch L, Ctx C, int ld, int field, float **staged);

// lsb_ls.cu: level set, classification, geometry, refill, sensor
cudaError_t run_classify_phase(int Q, Launch L, Ctx C, BlockShape S, const int *list, int n, int glevel, int init);
cudaError_t run_classify_links(int Q, Launch L, Ctx C, BlockShape S, const int *list, int n, int glevel, int full);
cudaError_t run_geometry(int D, Launch L, Ctx C, int glevel, int which);
cudaError_t run_ext_init(int Q, Launch L, Ctx C, int glevel);
cudaError_t run_ext_iter(int D, Launch L, Ctx C, BlockShape S, int glevel, const float *uin, float *uout, int mode);
cudaError_t run_adv_stage(int D, Launch L, Ctx C, BlockShape S, int glevel, int stage);
cudaError_t run_reinit_prep(int Q, Launch L, Ctx C, BlockShape S, int glevel);
cudaError_t run_reinit_stage(int D, Launch L, Ctx C, BlockShape S, int glevel, int stage);
// forward passes on mirrored stage arrays (no band lookups; see lsb_ls.cu)
cudaError_t run_ext_first(int D, Launch L, Ctx C, BlockShape S, int glevel, const float *uin, float *uout,
                          int turn);
cudaError_t run_ext_sweep_mirror(int D, Launch L, Ctx C, BlockShape S, int glevel, const float *uin, float *uout);
cudaError_t run_adv_mirror(int D, Launch L, Ctx C, BlockShape S, int glevel, int stage, const float *ufin);
cudaError_t run_reinit_mirror(int Q, Launch L, Ctx C, BlockShape S, int glevel, int stage, int prep);
// the curvature fit of the interface and flipped cells on CTAs [0, gg) (each flipped cell
// then refilled when refill is set) and the band pass on the rest, one launch
cudaError_t run_post_classify(int Q, int st, Launch L, Ctx C, const int *list, int n, int glevel, int gg,
                              int refill);
cudaError_t run_levelset_persistent(int Q, Launch L, Ctx C, BlockShape S, int glevel, int n_ext, int reinit,
                                    int n_reinit, unsigned *bar, long long limit);
cudaError_t run_sensor(Launch L, Ctx C, BlockShape S, const int *list, int n, int mode, float *out);

// lsb_adj.cu: adjoint of the frozen-interface step
constexpr int NG_ADJ = 13;  // parameter partials per case accumulated on the device
// Adjoints of the frozen geometry, finest-level arrays (nullptr: not computed):
// phi (nfine), interface cells' normal (D planes of nfine) and curvature (nfine).
struct GeoAdj {
  float *phi, *n, *kappa;
};
cudaError_t run_adj_seed(int Q, Launch L, Ctx C, BlockShape S, const int *list, int n, const float *F, float *lam,
                         const double *wobs, const double *obs, int stride, float eps, float *lphi);
cudaError_t run_adj_links(int Q, Launch L, Ctx C, int glevel, const float *F, float *lamN, float *LA, float *MA,
                          double *grad, int ncase, GeoAdj G);
cudaError_t run_adj_geometry(int D, Launch L, Ctx C, int glevel, GeoAdj G);
cudaError_t run_adj_collide(int Q, Launch L, Ctx C, BlockShape S, const int *list, int n, const float *F,
                            const float *lamN, float *lamO, const float *LA, double *grad);
cudaError_t run_adj_macro(int Q, Launch L, Ctx C, int glevel, const float *F, float *lamO, float *MA, double *grad,
                          int ncase);
// Multi-level grids: transposes of the ghost-ring transfer (per ghost cell of a
// fine level, coarse states at t and t + 1 blended by theta), of its coarse
// share's hand-over after the coarse sub-step, and of the restriction (per
// restriction-layer cell of a coarse level).
cudaError_t run_copy_blocks(int Q, Launch L, Ctx C, BlockShape S, const int *list, int n, const float *src,
                            float *dst);
cudaError_t run_adj_ghost(int Q, Launch L, Ctx C, const int2 *cells, int n, float theta, const float *Fold,
                          const float *Fnew, const float *lamNf, float *lamX, float *lamNc, double *grad, int ncase);
cudaError_t run_adj_ghost_apply(int Q, Launch L, Ctx C, const int2 *cells, int n, float *lamX, float *lamOc);
cudaError_t run_adj_restrict(int Q, Launch L, Ctx C, const int2 *cells, int n, const float *Ff, float *lamOc,
                             float *lamF, double *grad, int ncase);

// lsb_adj_ls.cu: adjoint of the level-set passes of a step with a moving interface
cudaError_t run_lsa_init(int Q, Launch L, Ctx C, int glevel, const float *F, float *U0);
cudaError_t run_lsa_init_T(int Q, Launch L, Ctx C, int glevel, const float *F, float *LS0, float *MA, float *LPHI);
cudaError_t run_lsa_mix(int D, Launch L, Ctx C, BlockShape S, int glevel, int mode, int use_frozen, const float *L3,
                        float *L0, float *L1, float *L2, const float *Ls0);
cudaError_t run_lsa_reinit_rt(int D, Launch L, Ctx C, BlockShape S, int glevel, const float *pin, const float *MU,
                              float scale, float *Lt, float *L0, float *Ls0);
cudaError_t run_lsa_adv_rt(int D, Launch L, Ctx C, BlockShape S, int glevel, const float *pin, const float *MU,
                           float scale, float *Lt, float *L0, float *LU);
cudaError_t run_lsa_ext_T(int D, Launch L, Ctx C, BlockShape S, int glevel, const float *Sk, const float *S0,
                          const float *Lin, float *Lout, float *LOFF, float *LV);
cudaError_t run_lsa_ext_v(int D, Launch L, Ctx C, BlockShape S, int glevel, float *LV, float *LPHI);
cudaError_t run_lsa_axpy(Launch L, long long n, const float *x, float *y);
cudaError_t run_lsa_flipflag(Launch L, const int *counters, int glevel, int *flag);

}  // namespace lsb
