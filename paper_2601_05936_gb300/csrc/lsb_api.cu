// Host runtime and C ABI of the lsb library (include/lsb.h).
//
// Owns every device buffer, builds the per-level block work lists, drives the
// Dupuis-Chopard recursion over levels (Sec. 2.1 last paragraph) with the
// finest-level interface, level-set and refill kernels, runs the refinement
// sensor and regrid (Sec. 2.6) with host-side grading, and exports fields.
// All cases of a handle (an ensemble) advance together: every launch covers
// the blocks of all cases that own the level it works on.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <functional>
#include <string>
#include <vector>

#include "lsb.h"
#include "lsb_kernels.h"

using namespace lsb;

namespace {

constexpr int MAXL = 4;
const char *const KNAMES[] = {"k_collide_stream", "k_interface_bc", "k_restrict", "k_ghost", "k_prolong", "k_level_tags", "k_observables", "k_export", "k_classify_phase", "k_classify_links", "k_post_classify", "k_geometry", "k_ext_init", "k_ext_iter", "k_adv_stage", "k_reinit_prep", "k_reinit_stage", "k_refill", "k_sensor", "k_init", "k_collect",
                               "k_collide_stream_l1", "k_collide_stream_l2", "k_collide_stream_l3", "k_adj_seed",
                               "k_adj_links", "k_adj_collide", "k_adj_macro", "k_adj_geometry",
                               "k_levelset_persistent", "k_lsa", "k_adj_ghost", "k_adj_ghost_apply",
                               "k_adj_restrict", "k_tape"};
constexpr int KADJ_SEED = 24, KADJ_LINKS = 25, KADJ_COLLIDE = 26, KADJ_MACRO = 27, KADJ_GEOM = 28, KLS_PERSIST = 29,
              KLSA = 30, KADJ_GHOST = 31, KADJ_GAPPLY = 32, KADJ_RESTRICT = 33, KTAPE = 34;
constexpr int NKERN = sizeof(KNAMES) / sizeof(KNAMES[0]);

struct ProfRec {
  int kid;
  cudaEvent_t a, b;
  double bytes;
};

struct WorkList {
  int *d = nullptr;
  int n = 0;
  int cap = 0;
  std::vector<int> h;
};

struct CellList {
  int2 *d = nullptr;
  int n = 0;
  int cap = 0;
};

struct CaseHost {
  lsb_grid_desc d;
  lsb_params p;
  int L = 1;
  int ld0 = 0;  // first level descriptor of this case
};

thread_local std::string g_create_error;

}  // namespace

struct lsb_grid {
  int ncase = 0, Q = 9, D = 2, storage = LSB_FP32, Lmax = 1;
  int bs[3] = {1, 1, 1};
  int nthreads = 0;
  float fp16_scale = 1.f;
  std::vector<CaseHost> cases;
  std::vector<LevelDev> lds;
  std::vector<std::vector<int8_t>> status;  // per ld
  long long ncell_total = 0, nfine = 0;
  int nblock_total = 0;
  // device buffers
  LevelDev *d_lds = nullptr;
  int *d_blk_ld = nullptr;
  int4 *d_blk_info = nullptr;
  int8_t *d_bstat = nullptr, *d_bstat_old = nullptr;
  uint8_t *d_bflag = nullptr, *d_tag = nullptr, *d_frozen = nullptr;
  void *d_buf[2] = {nullptr, nullptr};
  float *d_phi = nullptr, *d_p1 = nullptr, *d_p2 = nullptr, *d_s0 = nullptr;
  float *d_ut[3] = {nullptr, nullptr, nullptr};
  float *d_plan_v = nullptr;
  uint8_t *d_plan_f = nullptr;
  uint32_t *d_cmask = nullptr;
  int *d_cbase = nullptr;
  float *d_macro = nullptr, *d_nvec = nullptr, *d_kappa = nullptr, *d_linkbuf = nullptr;
  int2 *d_linkcell = nullptr;
  uint8_t *d_linkdir = nullptr;
  long long link_list_off[MAXL] = {0, 0, 0, 0};
  // pinned host words the synchronising calls read back into: the error word, then the
  // observables of every case (allocated at the first use)
  int *h_err = nullptr;
  double *h_obs = nullptr;
  int *d_work = nullptr;  // per level: the collide-and-stream's block counters (next, finished)
  int *d_counters = nullptr, *d_err = nullptr, *d_band = nullptr, *d_check = nullptr;
  int4 *d_band_info = nullptr;
  unsigned *d_bar = nullptr;  // grid barrier of the persistent level-set kernel
  long long wait_limit = 1LL << 22;  // sleeps of ~64 ns before a device-side wait gives up
  bool ls_dirty = false;  // stage arrays no longer mirror phi / u~ outside the band (driver 1 ran)
  float obj_eps = 0.f;    // > 0: observables and objective with the smoothed gas indicator H_eps
  int driver = 0;             // 0: one launch per level-set pass, 1: one persistent launch
  int2 *d_iface = nullptr, *d_flip = nullptr;
  double *d_obs = nullptr;
  float *d_sens = nullptr;
  long long link_cap = 0, list_cap = 0;
  int band_cap = 0;
  std::vector<void *> allocs;
  // work lists per global level
  WorkList cs[MAXL], rst[MAXL], ghost[MAXL], finest[MAXL], leaf, tags, sens, all_active;
  std::vector<int> tags_prev;
  CellList ghost_cells[MAXL], rl_cells[MAXL];
  int *d_count = nullptr;
  int par[MAXL] = {0, 0, 0, 0};
  long long fine_steps[MAXL] = {0, 0, 0, 0};
  long long coarse_steps = 0;
  // method parameters shared by all cases
  int n_ext = 8, reinit_every = 1, n_reinit = 1, regrid_every = 0;
  cudaStream_t stream = nullptr;
  uint64_t launches = 0;
  std::string err;
  int latched = 0;
  // kernel timing
  int prof_mode = 0;
  std::vector<cudaEvent_t> ev_pool;
  std::vector<ProfRec> prof;
  double leaf_cells[MAXL] = {0, 0, 0, 0};
  double updates_done = 0;
  // CUDA graphs of two coarse steps, one per starting parity of level 0
  int use_graphs = 0;
  // TMA tensor maps of every level's population buffers (2 per level descriptor)
  CUtensorMap *d_tmaps = nullptr;
  int tma_grid = 0;
  int prio_hi = 0;                // the device's highest launch priority
  int obs_tma_grid = 0;           // resident CTAs of the TMA-staged observables pass (0: not built)
  int tma_tags = 0;               // d_tmaps also holds one cell-tag map per level descriptor
  cudaGraphExec_t gexec[2][2] = {};  // [coarse steps per replay - 1][level-0 parity at the start]
  cudaStream_t side[MAXL] = {};        // per level: its collide-and-stream beside the first fine sub-step
  cudaEvent_t ev_fork[MAXL] = {}, ev_join[MAXL] = {};
  // per level: its second sub-step's ghost ring, filled beside the first sub-step's
  // interface, level-set, classification and refill passes
  cudaStream_t side2[MAXL] = {};
  cudaEvent_t ev_free[MAXL] = {}, ev_fill[MAXL] = {}, ev_ring0[MAXL] = {}, ev_ring0_done[MAXL] = {};
  int early_fill = -1;  // level whose next ghost ring fills right after its collide
  bool counters_turned[MAXL] = {};  // the level's classification counters already started
  bool init_done[MAXL] = {};        // the level's interface u~ came with the interface pass
  uint64_t gnodes[2][2] = {};
  // adjoint of the frozen-interface step: recording and reverse sweep
  int rec_on = 0, rec_every = 0;
  int no_tma = 0;                 // recomputation writes into segment slots: plain collide kernel
  long long rec_steps = 0;
  std::vector<float *> rec_ckpt;  // state at the start of steps 0, every, 2 every, ...
  float *d_seg = nullptr;         // states of one recomputed segment
  int seg_cap = 0;
  CUtensorMap *d_seg_tmaps = nullptr;  // per slot and level descriptor: that slot's populations
  const CUtensorMap *tma_a = nullptr;  // population maps the next collide launches read (default d_tmaps)
  void *encode_fn = nullptr;           // cuTensorMapEncodeTiled
  size_t seg_slot = 0;            // bytes per stored state
  float *d_adj[2] = {nullptr, nullptr};
  int adj_cur = -1;               // >= 0 once lsb_backward has run: dJ/df_0 is held in d_adj
  int apar[MAXL] = {0, 0, 0, 0};  // level l's adjoint is d_adj[apar[l]] (its region of the buffer)
  // multi-level grids: the step is replayed with every level's populations recorded per
  // call of the level recursion (preorder), input of the transposed transfers
  int tape_on = 0, tape_call = 0;
  std::vector<float *> tape_old, tape_new;  // state at the call's start (after restriction), after its sub-step
  std::vector<float *> tape_ls;             // moving level set: phi and u~ at each finest call's start
  int lspar = 0;                            // moving level set: its adjoints are in LP[lspar], LU[lspar]
  float *d_adjx = nullptr;                  // coarse adjoint shares of the ghost rings (kept zero)
  float *d_fsave = nullptr, *d_madj = nullptr, *d_linkadj = nullptr;
  float *d_gphi = nullptr, *d_gn = nullptr, *d_gk = nullptr;  // level-set adjoint (finest level)
  // moving level set: the state is (f, phi, u~); scratch of the level-set replay and transposes
  int rec_moving = 0;
  int *d_recflip = nullptr;  // set when a recorded step flipped a cell
  float *d_lsa = nullptr;    // one allocation, carved by lsa_ptrs()
  size_t lsa_floats = 0;
  float *d_phisave = nullptr, *d_utsave = nullptr;
  double *d_grad = nullptr, *d_wobs = nullptr;
};

namespace {

lsb_status fail(lsb_grid *g, lsb_status s, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (g) g->err = buf;
  else g_create_error = buf;
  return s;
}

#define CU(call)                                                                           \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess) return fail(g, LSB_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

template <typename P>
lsb_status dalloc(lsb_grid *g, P **ptr, size_t bytes) {
  void *p = nullptr;
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMalloc(&p, bytes);
  if (e != cudaSuccess) return fail(g, LSB_ENOMEM, "cudaMalloc(%zu): %s", bytes, cudaGetErrorString(e));
  g->allocs.push_back(p);
  *ptr = reinterpret_cast<P *>(p);
  return LSB_OK;
}

lsb_status upload_list(lsb_grid *g, WorkList &w) {
  w.n = (int)w.h.size();
  if (w.n > w.cap) {
    int cap = std::max(w.n, 64);
    int *p = nullptr;
    lsb_status s = dalloc(g, &p, sizeof(int) * (size_t)cap);
    if (s) return s;
    w.d = p;
    w.cap = cap;
  }
  if (w.n) CU(cudaMemcpyAsync(w.d, w.h.data(), sizeof(int) * w.n, cudaMemcpyHostToDevice, g->stream));
  return LSB_OK;
}

Ctx make_ctx(lsb_grid *g) {
  Ctx C;
  memset(&C, 0, sizeof C);
  C.lds = g->d_lds;
  C.blk_ld = g->d_blk_ld;
  C.blk_info = g->d_blk_info;
  C.bstat = g->d_bstat;
  C.bstat_old = g->d_bstat_old;
  C.bflag = g->d_bflag;
  C.tag = g->d_tag;
  C.buf[0] = g->d_buf[0];
  C.buf[1] = g->d_buf[1];
  for (int l = 0; l < MAXL; ++l) C.par[l] = g->par[l];
  C.phi = g->d_phi;
  C.p1 = g->d_p1;
  C.p2 = g->d_p2;
  C.s0 = g->d_s0;
  C.frozen = g->d_frozen;
  C.ut0 = g->d_ut[0];
  C.ut1 = g->d_ut[1];
  C.ut2 = g->d_ut[2];
  C.plan_v = g->d_plan_v;
  C.plan_f = g->d_plan_f;
  C.cmask = g->d_cmask;
  C.cbase = g->d_cbase;
  C.macro = g->d_macro;
  C.nvec = g->d_nvec;
  C.kappa = g->d_kappa;
  C.linkbuf = g->d_linkbuf;
  C.nfine = g->nfine;
  C.link_cap = g->link_cap;
  C.link_cell = g->d_linkcell;
  C.link_dir = g->d_linkdir;
  for (int l = 0; l < MAXL; ++l) C.link_list_off[l] = g->link_list_off[l];
  C.counters = g->d_counters;
  C.iface_list = g->d_iface;
  C.flip_list = g->d_flip;
  C.band_list = g->d_band;
  C.check_list = g->d_check;
  C.band_info = g->d_band_info;
  C.list_cap = g->list_cap;
  C.band_cap = g->band_cap;
  C.err = g->d_err;
  C.fp16_scale = g->fp16_scale;
  C.fp16_inv = 1.0f / g->fp16_scale;
  return C;
}

BlockShape shape(const lsb_grid *g) {
  BlockShape S;
  for (int a = 0; a < 3; ++a) {
    S.bs[a] = g->bs[a];
    int lg = 0;
    while ((1 << lg) < g->bs[a]) ++lg;
    S.lg[a] = lg;
  }
  return S;
}

// Count a launch and turn its error into a status.
lsb_status launched(lsb_grid *g, cudaError_t e) {
  g->launches++;
  if (e != cudaSuccess) return fail(g, LSB_ECUDA, "kernel launch: %s", cudaGetErrorString(e));
  return LSB_OK;
}

// Kernels of a handle with a stream of its own launch as programmatic dependents of the
// kernel before them (off while kernel timing is on, so that each launch's events
// bracket that launch alone).
#ifndef LSB_PDL
#define LSB_PDL 1
#endif
// ... and at the device's highest priority: the coarser level's collide-and-stream on its
// side stream (default priority) then fills the slots the step's own chain leaves free
#ifndef LSB_PRIO
#define LSB_PRIO 1
#endif
Launch LN(const lsb_grid *g, int grid, int block) {
  return Launch{grid, block, g->stream, LSB_PDL && g->stream != nullptr && g->prof_mode == 0 ? 1 : 0,
                LSB_PRIO ? g->prio_hi : 0};
}

cudaEvent_t take_event(lsb_grid *g) {
  if (!g->ev_pool.empty()) {
    cudaEvent_t e = g->ev_pool.back();
    g->ev_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// Collide-and-stream launches carry one timing class per level (0, then 21..23).
int collide_kid(int level) { return level == 0 ? 0 : 20 + level; }
bool is_collide_kid(int kid) { return kid == 0 || (kid >= 21 && kid <= 23); }
bool profiled(const lsb_grid *g, int kid) { return g->prof_mode == 2 || (g->prof_mode == 1 && is_collide_kid(kid)); }

// Launch through a host launcher; with profiling on, bracket it with events.
#define RUN(kid, bytes, grid, block, fn, ...)                         \
  do {                                                                \
    if ((grid) > 0) {                                                 \
      ProfRec pr_{kid, nullptr, nullptr, (double)(bytes)};            \
      const bool on_ = profiled(g, kid);                              \
      if (on_) {                                                      \
        pr_.a = take_event(g);                                        \
        pr_.b = take_event(g);                                        \
        cudaEventRecord(pr_.a, g->stream);                            \
      }                                                               \
      cudaError_t e_ = fn(__VA_ARGS__);                               \
      if (on_) {                                                      \
        cudaEventRecord(pr_.b, g->stream);                            \
        g->prof.push_back(pr_);                                       \
      }                                                               \
      TRY(launched(g, e_));                                           \
    }                                                                 \
  } while (0)

constexpr int DYN_GRID = 152 * 8;  // CTAs for kernels over device-sized lists
// CTAs of a shared launch for the interface cells' u~ and for the curvature fit (of 128
// threads; the cell lists are a few ten thousand long and loop beyond)
#ifndef LSB_INIT_CTAS
#define LSB_INIT_CTAS 512
#endif
#ifndef LSB_IFACE_CTAS
#define LSB_IFACE_CTAS DYN_GRID  // and for the cut links of the interface pass beside them
#endif
#ifndef LSB_GEO_CTAS
#define LSB_GEO_CTAS 512
#endif

#define TRY(x)                   \
  do {                           \
    lsb_status s_ = (x);         \
    if (s_ != LSB_OK) return s_; \
  } while (0)

// ------------------------------------------------------------------ block topology helpers
void block_coords(const LevelDev &L, int lb, int b[3]) {
  b[0] = lb % L.nb[0];
  b[1] = (lb / L.nb[0]) % L.nb[1];
  b[2] = lb / (L.nb[0] * L.nb[1]);
}

template <typename F>
void for_block_neighbors(const lsb_grid *g, const LevelDev &L, int lb, F fn) {
  int b[3];
  block_coords(L, lb, b);
  const int zr = g->D == 3 ? 1 : 0;
  for (int dz = -zr; dz <= zr; ++dz)
    for (int dy = -1; dy <= 1; ++dy)
      for (int dx = -1; dx <= 1; ++dx) {
        int c[3] = {b[0] + dx, b[1] + dy, b[2] + dz};
        bool ok = true;
        for (int a = 0; a < g->D; ++a) {
          if (c[a] < 0 || c[a] >= L.nb[a]) {
            if (L.per[a]) c[a] = (c[a] + L.nb[a]) % L.nb[a];
            else ok = false;
          }
        }
        if (ok) fn(c[0] + L.nb[0] * (c[1] + L.nb[1] * c[2]));
      }
}

int parent_block(const LevelDev &Lc, const LevelDev &Lf, int lbf) {
  int b[3];
  block_coords(Lf, lbf, b);
  return (b[0] / 2) + Lc.nb[0] * ((b[1] / 2) + Lc.nb[1] * (b[2] / 2));
}

// Grading from the finest level down, then statuses top-down (mirrors the oracle's reading).
void grade_case(const lsb_grid *g, const CaseHost &ch, std::vector<std::vector<char>> &want,
                std::vector<std::vector<int8_t>> &st) {
  const int L = ch.L;
  for (int l = L - 2; l >= 1; --l) {
    const LevelDev &Lf = g->lds[ch.ld0 + l];
    const LevelDev &Lc = g->lds[ch.ld0 + l - 1];
    for (int b = 0; b < Lf.nblock; ++b) {
      if (!want[l][b]) continue;
      for_block_neighbors(g, Lf, b, [&](int nb) { want[l - 1][parent_block(Lc, Lf, nb)] = 1; });
      want[l - 1][parent_block(Lc, Lf, b)] = 1;
    }
  }
  st.assign(L, {});
  for (int l = 0; l < L; ++l) {
    const LevelDev &Ll = g->lds[ch.ld0 + l];
    st[l].assign(Ll.nblock, BLK_INACTIVE);
    for (int b = 0; b < Ll.nblock; ++b) {
      bool act = l == 0 ? true : st[l - 1][parent_block(g->lds[ch.ld0 + l - 1], Ll, b)] == BLK_REFINED;
      int8_t s = act ? BLK_LEAF : BLK_INACTIVE;
      if (l < L - 1 && act && want[l][b]) s = BLK_REFINED;
      st[l][b] = s;
    }
  }
}

bool any_neighbor(const lsb_grid *g, const LevelDev &L, const std::vector<int8_t> &st, int lb, int8_t what,
                  bool active_any) {
  bool r = false;
  for_block_neighbors(g, L, lb, [&](int nb) {
    if (active_any ? (st[nb] != BLK_INACTIVE) : (st[nb] == what)) r = true;
  });
  return r;
}

// Rebuild every host work list from the statuses and upload them.
lsb_status build_lists(lsb_grid *g) {
  for (int l = 0; l < MAXL; ++l) {
    g->cs[l].h.clear();
    g->rst[l].h.clear();
    g->ghost[l].h.clear();
    g->finest[l].h.clear();
  }
  g->leaf.h.clear();
  g->all_active.h.clear();
  for (int l = 0; l < MAXL; ++l) g->leaf_cells[l] = 0;
  std::vector<int> tl;
  for (size_t ld = 0; ld < g->lds.size(); ++ld) {
    const LevelDev &L = g->lds[ld];
    const std::vector<int8_t> &st = g->status[ld];
    const int l = L.level;
    for (int b = 0; b < L.nblock; ++b) {
      const int gb = L.block_off + b;
      const int8_t s = st[b];
      bool near_leaf = any_neighbor(g, L, st, b, BLK_LEAF, false);
      bool near_active = any_neighbor(g, L, st, b, 0, true);
      if (s == BLK_LEAF) {
        int bc[3];
        block_coords(L, b, bc);
        double cnt = 1;
        for (int a = 0; a < 3; ++a) cnt *= std::min(g->bs[a], L.n[a] - bc[a] * g->bs[a]);
        g->leaf_cells[l] += cnt;
        g->cs[l].h.push_back(gb);
        g->leaf.h.push_back(gb);
        if (L.finest) g->finest[l].h.push_back(gb);
      }
      if (s != BLK_INACTIVE) g->all_active.h.push_back(gb);
      if (s == BLK_REFINED && near_leaf) {
        g->cs[l].h.push_back(gb);
        g->rst[l].h.push_back(gb);
      }
      if (s == BLK_INACTIVE && near_active && l > 0) g->ghost[l].h.push_back(gb);
      if (s != BLK_INACTIVE || near_active) tl.push_back(gb);
    }
  }
  // tags: current relevant blocks plus the previous ones (stale bits get cleared)
  std::vector<int> u = tl;
  u.insert(u.end(), g->tags_prev.begin(), g->tags_prev.end());
  std::sort(u.begin(), u.end());
  u.erase(std::unique(u.begin(), u.end()), u.end());
  g->tags.h = u;
  g->tags_prev = tl;
  for (int l = 0; l < MAXL; ++l) {
    TRY(upload_list(g, g->cs[l]));
    TRY(upload_list(g, g->rst[l]));
    TRY(upload_list(g, g->ghost[l]));
    TRY(upload_list(g, g->finest[l]));
  }
  TRY(upload_list(g, g->leaf));
  TRY(upload_list(g, g->tags));
  TRY(upload_list(g, g->all_active));
  return LSB_OK;
}

lsb_status upload_status(lsb_grid *g, const std::vector<std::vector<int8_t>> &st) {
  std::vector<int8_t> flat(g->nblock_total);
  for (size_t ld = 0; ld < g->lds.size(); ++ld)
    std::copy(st[ld].begin(), st[ld].end(), flat.begin() + g->lds[ld].block_off);
  CU(cudaMemcpyAsync(g->d_bstat, flat.data(), flat.size(), cudaMemcpyHostToDevice, g->stream));
  CU(cudaStreamSynchronize(g->stream));  // flat is a host temporary
  return LSB_OK;
}

lsb_status level_tags(lsb_grid *g) {
  Ctx C = make_ctx(g);
  BlockShape S = shape(g);
  RUN(5, 0, g->tags.n, g->nthreads, run_level_tags, g->Q, LN(g, g->tags.n, g->nthreads), C, S, (const int *)g->tags.d,
      g->tags.n);
  return LSB_OK;
}

bool has_finest(const lsb_grid *g, int l) {
  for (const CaseHost &c : g->cases)
    if (c.L - 1 == l) return true;
  return false;
}

// Classification of the finest level l: phases, flips, cut links, band; then geometry.
// refill: the step's classification, whose curvature-fit threads also refill the flipped
// cells (the refill pass of the step); otherwise no refill runs here.
#ifndef LSB_CLS_CTAS
#define LSB_CLS_CTAS 32  // CTAs per SM (at most) of the phase and link passes: a CTA per listed block
                         // (8: 0.769 ms per step, 16-32: 0.759)
#endif
lsb_status classify(lsb_grid *g, int l, int init, bool refill = false) {
  if (!has_finest(g, l)) return LSB_OK;
  // the band list the previous classification left is the set of blocks whose phases can
  // change (phi moves on band cells only): keep its length, then clear the counters
  // (the first extension sweep of this sub-step did it already; the phase pass clears the
  // band count)
  int *cnt = g->d_counters + l * NCOUNT;
  if (init || !g->counters_turned[l]) {
    CU(cudaMemcpyAsync(cnt + 5, cnt + 3, sizeof(int), cudaMemcpyDeviceToDevice, g->stream));
    CU(cudaMemsetAsync(cnt, 0, sizeof(int) * 5, g->stream));
  }
  g->counters_turned[l] = false;
  Ctx C = make_ctx(g);
  BlockShape S = shape(g);
  WorkList &F = g->finest[l];
  const int *fl = F.d;
  const int Q = g->Q, D = g->D, nt = g->nthreads;
  // after creation or a regrid every finest block; otherwise the previous band's blocks
  // (and, for the cut links, the blocks next to a flipped cell), walked from the lists
  const int nlist = init ? F.n : std::max(1, std::min(F.n, 152 * LSB_CLS_CTAS));
  RUN(8, 0, F.n, nt, run_classify_phase, Q, LN(g, nlist, nt), C, S, fl, F.n, l, init);
  RUN(9, 0, F.n, nt, run_classify_links, Q, LN(g, nlist, nt), C, S, fl, F.n, l, init);
  // the band pass (a warp per block) and the curvature fit at the interface and the
  // flipped cells (and the refill of the flipped cells) share a launch
  const int gband = (F.n + 3) / 4;
  RUN(10, 0, F.n, 128, run_post_classify, Q, g->storage, LN(g, LSB_GEO_CTAS + gband, 128), C, fl, F.n, l,
      LSB_GEO_CTAS, refill ? 1 : 0);
  (void)D;
  return LSB_OK;
}

// The precondition of the mirrored level-set passes, set in full: p1 = p2 = phi and
// ut1 = ut2 = ut0 at every finest cell (after creation and after phi or u~ were
// restored from a stored state).
lsb_status ls_mirror(lsb_grid *g) {
  const size_t b1 = sizeof(float) * (size_t)g->nfine, bD = b1 * g->D;
  CU(cudaMemcpyAsync(g->d_p1, g->d_phi, b1, cudaMemcpyDeviceToDevice, g->stream));
  CU(cudaMemcpyAsync(g->d_p2, g->d_phi, b1, cudaMemcpyDeviceToDevice, g->stream));
  CU(cudaMemcpyAsync(g->d_ut[1], g->d_ut[0], bD, cudaMemcpyDeviceToDevice, g->stream));
  CU(cudaMemcpyAsync(g->d_ut[2], g->d_ut[0], bD, cudaMemcpyDeviceToDevice, g->stream));
  g->ls_dirty = false;
  return LSB_OK;
}

// Level-set update of the finest level l (extension, transport, reinitialisation).
lsb_status levelset(lsb_grid *g, int l) {
  Ctx C = make_ctx(g);
  BlockShape S = shape(g);
  const int nb = std::max(1, std::min(g->band_cap, 152 * 16));
  const int nt = g->nthreads;
  const int Q = g->Q, D = g->D;
  if (g->driver == 1) {
    g->ls_dirty = true;  // its passes keep no mirror of u~ in the sweep buffers
    const bool due = g->reinit_every > 0 && ((g->fine_steps[l] + 1) % g->reinit_every == 0) && g->n_reinit > 0;
    // a barrier that gave up leaves its count behind: start every launch from zero
    CU(cudaMemsetAsync(g->d_bar, 0, 2 * sizeof(unsigned), g->stream));
    RUN(KLS_PERSIST, 0, 1, nt, run_levelset_persistent, Q, LN(g, nb, nt), C, S, l, g->n_ext, due ? 1 : 0,
        g->n_reinit, g->d_bar, g->wait_limit);
    return LSB_OK;
  }
  // passes on mirrored stage arrays: the first sweep stores the plan, the others reuse
  // it; the first transport stage commits u~; the first reinitialisation stage finds
  // the frozen cells
  if (!g->init_done[l]) RUN(12, 0, 1, 128, run_ext_init, Q, LN(g, DYN_GRID, 128), C, l);
  g->init_done[l] = false;
  const float *uin = g->d_ut[0];
  for (int it = 0; it < g->n_ext; ++it) {
    float *uout = g->d_ut[1 + (it & 1)];
    if (it == 0) {
      RUN(13, 0, nb, nt, run_ext_first, D, LN(g, nb, nt), C, S, l, uin, uout, 1);
      g->counters_turned[l] = true;  // the classification of this sub-step finds them started
    }
    else RUN(13, 0, nb, nt, run_ext_sweep_mirror, D, LN(g, nb, nt), C, S, l, uin, uout);
    uin = uout;
  }
  for (int st = 1; st <= 3; ++st) {
    RUN(14, 0, nb, nt, run_adv_mirror, D, LN(g, nb, nt), C, S, l, st, uin);
  }
  const bool due = g->reinit_every > 0 && ((g->fine_steps[l] + 1) % g->reinit_every == 0);
  if (due && g->n_reinit > 0) {
    for (int r = 0; r < g->n_reinit; ++r)
      for (int st = 1; st <= 3; ++st) {
        RUN(16, 0, nb, nt, run_reinit_mirror, Q, LN(g, nb, nt), C, S, l, st, r == 0 && st == 1 ? 1 : 0);
      }
  }
  return LSB_OK;
}

bool ls_active_any(const lsb_grid *g, int l) {
  for (const CaseHost &c : g->cases)
    if (c.L - 1 == l && c.p.ls_active) return true;
  return false;
}

// Copy every case's level-l populations from src to dst (same offsets: each level's
// region of a Q x ncell_total array): the cells of the level's leaf blocks and of the
// covered blocks leaves stream from, the only ones a step reads.
lsb_status copy_level(lsb_grid *g, float *dst, const float *src, int l) {
  const WorkList &w = g->cs[l];
  RUN(KTAPE, 2.0 * sizeof(float) * g->Q * g->nthreads * (double)w.n, w.n, g->nthreads, run_copy_blocks, g->Q,
      LN(g, std::min(w.n, DYN_GRID), g->nthreads), make_ctx(g), shape(g), (const int *)w.d, w.n, src, dst);
  return LSB_OK;
}

// The populations of every level (each level's current buffer) into one
// Q x ncell_total array, and back.
lsb_status snapshot(lsb_grid *g, float *dst) {
  for (int l = 0; l < g->Lmax; ++l) TRY(copy_level(g, dst, (const float *)g->d_buf[g->par[l]], l));
  return LSB_OK;
}
lsb_status restore(lsb_grid *g, const float *src) {
  for (int l = 0; l < g->Lmax; ++l) TRY(copy_level(g, (float *)g->d_buf[g->par[l]], src, l));
  return LSB_OK;
}

// The side stream's collide gets 1 / LSB_SIDE_DIV of the resident CTAs: all of them measured
// fastest (0.8179 ms per step against 0.8257 at half and 0.94 at a quarter), the main
// stream's kernels taking the slots it frees first by their priority.
#ifndef LSB_SIDE_DIV
#define LSB_SIDE_DIV 1
#endif

// The collide-and-stream's block counters of level l (two words, zero between launches;
// one launch of a level at a time), or none (static assignment).
#ifndef LSB_DYN
#define LSB_DYN 1
#endif
int *work_counters(lsb_grid *g, int l) { return LSB_DYN && g->d_work ? g->d_work + 2 * l : nullptr; }

// Restriction and collide-and-stream of level l on its side stream, after the main
// stream's work so far.
lsb_status coarse_side(lsb_grid *g, int l) {
  const BlockShape S = shape(g);
  const Ctx C = make_ctx(g);
  const int Q = g->Q, st = g->storage, nt = g->nthreads;
  if (!g->side[l]) {
    CU(cudaStreamCreateWithFlags(&g->side[l], cudaStreamNonBlocking));
    CU(cudaEventCreateWithFlags(&g->ev_fork[l], cudaEventDisableTiming));
    CU(cudaEventCreateWithFlags(&g->ev_join[l], cudaEventDisableTiming));
  }
  CU(cudaEventRecord(g->ev_fork[l], g->stream));
  CU(cudaStreamWaitEvent(g->side[l], g->ev_fork[l], 0));
  const CellList &rc = g->rl_cells[l];
  RUN(2, 0, rc.n, 128, run_restrict_cells, Q, st, (Launch{(rc.n + 127) / 128, 128, g->side[l]}), C,
      (const int2 *)rc.d, rc.n);
  const double cs_bytes = 2.0 * g->Q * (g->storage == LSB_FP32 ? 4 : 2) * g->leaf_cells[l];
  const int grid = std::min(g->cs[l].n, std::max(1, g->tma_grid / LSB_SIDE_DIV));
  const CUtensorMap *tm = (const CUtensorMap *)g->d_tmaps;
  RUN(collide_kid(l), cs_bytes, g->cs[l].n, nt, run_collide_stream_tma, Q, st, Launch{grid, nt, g->side[l]}, C, S,
      (const int *)g->cs[l].d, g->cs[l].n, tm, g->tma_tags ? tm + 2 * g->lds.size() : nullptr, work_counters(g, l));
  CU(cudaEventRecord(g->ev_join[l], g->side[l]));
  return LSB_OK;
}

// The first sub-step's ghost ring of the deepest level on its side stream beside that
// sub-step's collide (which takes its blocks dynamically, so the ring's CTAs cost it only
// their share): 0.803 -> 0.799 ms per step.
#ifndef LSB_RING0_SIDE
#define LSB_RING0_SIDE 1
#endif
// One advance of global level l (recursive over finer levels).
lsb_status advance(lsb_grid *g, int l) {
  BlockShape S = shape(g);
  const int nt = g->nthreads;
  Ctx C = make_ctx(g);
  const int Q = g->Q, st = g->storage;
  // A coarser level's collide-and-stream writes only its own B buffer, and the first fine
  // sub-step reads only its A buffer at leaf cells (ghost ring at theta = 0): with no case
  // finishing at this level, the restriction (it writes A at covered cells from the finer
  // level's A, which that sub-step only reads) and the collide run on a side stream beside
  // that sub-step (the sub-step's own kernels launch at a higher priority, so they take the
  // slots the collide's CTAs free first), joined before anything of the second sub-step
  // writes the finer A buffer or reads this B.
  const bool fork = g->stream && g->prof_mode == 0 && !g->tape_on && l + 1 < g->Lmax && !has_finest(g, l) &&
                    g->d_tmaps && !g->no_tma && !g->tma_a;
  const CellList &rc = g->rl_cells[l];
  if (fork) {
    TRY(coarse_side(g, l));
  } else {
    RUN(2, 0, rc.n, 128, run_restrict_cells, Q, st, LN(g, (rc.n + 127) / 128, 128), C, (const int2 *)rc.d, rc.n);
  }
  const int call = g->tape_on ? g->tape_call++ : -1;
  if (call >= 0) TRY(copy_level(g, g->tape_old[call], (const float *)g->d_buf[g->par[l]], l));
  if (call >= 0 && g->rec_moving && l == g->Lmax - 1) {  // the level set at the finest sub-step's start
    float *t = g->tape_ls[call];
    CU(cudaMemcpyAsync(t, g->d_phi, sizeof(float) * g->nfine, cudaMemcpyDeviceToDevice, g->stream));
    CU(cudaMemcpyAsync(t + g->nfine, g->d_ut[0], sizeof(float) * g->D * g->nfine, cudaMemcpyDeviceToDevice,
                       g->stream));
  }
  const double cs_bytes = 2.0 * g->Q * (g->storage == LSB_FP32 ? 4 : 2) * g->leaf_cells[l];
  if (fork) {
    // on the side stream (coarse_side, above)
  } else if (g->d_tmaps && !g->no_tma) {
    const int grid = std::min(g->cs[l].n, g->tma_grid);
    const CUtensorMap *tm = (const CUtensorMap *)g->d_tmaps;
    RUN(collide_kid(l), cs_bytes, g->cs[l].n, nt, run_collide_stream_tma, Q, st, LN(g, grid, nt), C, S,
        (const int *)g->cs[l].d, g->cs[l].n, g->tma_a ? g->tma_a : tm, g->tma_tags ? tm + 2 * g->lds.size() : nullptr,
        work_counters(g, l));
  } else {
    RUN(collide_kid(l), cs_bytes, g->cs[l].n, nt, run_collide_stream, Q, st, LN(g, g->cs[l].n, nt), C, S, (const int *)g->cs[l].d,
        g->cs[l].n);
  }
  if (g->early_fill == l) {
    // the second sub-step's ghost ring (theta = 1/2): its pushes go to the buffer that
    // sub-step streams into, which is this sub-step's A buffer (the collide has finished
    // reading it, and the interface, level-set, classification and refill passes that
    // follow touch only B); it reads the coarser level's A and B buffers, so it also waits
    // for that level's collide on side[l - 1]
    g->early_fill = -1;  // (the side stream and its events are made by the coarser level)
    CU(cudaEventRecord(g->ev_free[l], g->stream));
    if (LSB_RING0_SIDE) CU(cudaStreamWaitEvent(g->stream, g->ev_ring0_done[l], 0));  // this sub-step's ring
    CU(cudaStreamWaitEvent(g->side2[l], g->ev_free[l], 0));
    CU(cudaStreamWaitEvent(g->side2[l], g->ev_join[l - 1], 0));
    Ctx C2 = make_ctx(g);
    C2.par[l] ^= 1;  // the buffers of the next sub-step
    const CellList &gc = g->ghost_cells[l];
    RUN(3, 0, gc.n, 128, run_ghost_cells, Q, st, (Launch{(gc.n + 127) / 128, 128, g->side2[l]}), C2,
        (const int2 *)gc.d, gc.n, 0.5f);
    CU(cudaEventRecord(g->ev_fill[l], g->side2[l]));
  }
  if (has_finest(g, l)) {
    if (ls_active_any(g, l) && g->driver == 0) {
      // the interface pass and the level set's first pass (u~ at the interface cells) share
      // a launch; the level-set update then starts from its first extension sweep
      RUN(1, 0, 1, 128, run_iface_init, Q, st, LN(g, LSB_INIT_CTAS + LSB_IFACE_CTAS, 128), C, l, LSB_INIT_CTAS);
      g->init_done[l] = true;
    } else {
      RUN(1, 0, 1, 128, run_interface_bc, Q, st, LN(g, DYN_GRID, 128), C, l);
    }
    if (ls_active_any(g, l)) {
      TRY(levelset(g, l));
      TRY(classify(g, l, 0, true));  // with the refill of the flipped cells
    }  // a frozen level set leaves phases, cut links and geometry as they are
    g->fine_steps[l]++;
  }
  if (call >= 0 && l + 1 < g->Lmax) TRY(copy_level(g, g->tape_new[call], (const float *)g->d_buf[1 - g->par[l]], l));
  if (l + 1 < g->Lmax) {
    // with the next level the deepest (no sub-steps below it read its buffers), its ghost
    // rings fill on a side stream: the first beside its first sub-step's collide, the
    // second beside that sub-step's interface, level-set, classification and refill passes
    const bool early = fork && l + 2 == g->Lmax;
    if (early && !g->side2[l + 1]) {
      CU(cudaStreamCreateWithFlags(&g->side2[l + 1], cudaStreamNonBlocking));
      for (cudaEvent_t *e : {&g->ev_free[l + 1], &g->ev_fill[l + 1], &g->ev_ring0[l + 1], &g->ev_ring0_done[l + 1]})
        CU(cudaEventCreateWithFlags(e, cudaEventDisableTiming));
    }
    for (int sub = 0; sub < 2; ++sub) {
      if (sub == 0 && early && LSB_RING0_SIDE) {
        // the first sub-step's ring (theta = 0) reads only the coarser level's A buffer at
        // leaf cells and writes pushes into the finer B buffer that no leaf pushes to: it
        // runs beside that sub-step's collide-and-stream, joined before its interface pass
        CU(cudaEventRecord(g->ev_ring0[l + 1], g->stream));
        CU(cudaStreamWaitEvent(g->side2[l + 1], g->ev_ring0[l + 1], 0));
        C = make_ctx(g);
        const CellList &gc = g->ghost_cells[l + 1];
        RUN(3, 0, gc.n, 128, run_ghost_cells, Q, st, (Launch{(gc.n + 127) / 128, 128, g->side2[l + 1]}), C,
            (const int2 *)gc.d, gc.n, 0.0f);
        CU(cudaEventRecord(g->ev_ring0_done[l + 1], g->side2[l + 1]));
      } else if (sub == 1 && early) {
        CU(cudaStreamWaitEvent(g->stream, g->ev_fill[l + 1], 0));  // after the coarse collide, too
      } else {
        if (sub == 1 && fork) CU(cudaStreamWaitEvent(g->stream, g->ev_join[l], 0));  // theta = 1/2 reads B
        C = make_ctx(g);
        const float theta = sub == 0 ? 0.0f : 0.5f;
        const CellList &gc = g->ghost_cells[l + 1];
        RUN(3, 0, gc.n, 128, run_ghost_cells, Q, st, LN(g, (gc.n + 127) / 128, 128), C, (const int2 *)gc.d, gc.n,
            theta);
      }
      if (sub == 0 && early) g->early_fill = l + 1;
      const lsb_status r = advance(g, l + 1);
      g->early_fill = -1;
      if (r != LSB_OK) return r;
    }
  }
  g->par[l] ^= 1;
  return LSB_OK;
}

lsb_status regrid(lsb_grid *g, bool initial);
// Pinned read-back words (one allocation: the error word, then room for the observables).
lsb_status pin_host(lsb_grid *g) {
  if (g->h_err) return LSB_OK;
  const size_t nobs = (size_t)(4 + 2 * g->D) * g->ncase;
  void *p = nullptr;
  CU(cudaMallocHost(&p, 16 + sizeof(double) * nobs));
  g->h_err = static_cast<int *>(p);
  g->h_obs = reinterpret_cast<double *>(static_cast<char *>(p) + 16);
  return LSB_OK;
}


// Leaf cell updates of one coarse step: sum over levels of leaf cells x 2^level.
double updates_per_step(const lsb_grid *g) {
  double t = 0;
  for (int l = 0; l < MAXL; ++l) t += g->leaf_cells[l] * (double)(1 << l);
  return t;
}

lsb_status check_params(const lsb_params &p, const lsb_grid_desc &d, std::string &why) {
  char b[256];
  for (int k = 0; k < 2; ++k) {
    if (!(p.rho[k] > 0) || !(p.nu[k] > 0) || !std::isfinite(p.rho[k]) || !std::isfinite(p.nu[k])) {
      snprintf(b, sizeof b, "rho and nu must be positive (phase %d)", k);
      why = b;
      return LSB_EINVAL;
    }
  }
  if (p.n_ext < 0 || p.reinit_every < 0 || p.n_reinit < 0 || p.regrid_every < 0) {
    why = "negative iteration count";
    return LSB_EINVAL;
  }
  if (!(p.sigma >= 0)) { why = "sigma must be >= 0"; return LSB_EINVAL; }
  if (p.sensor != LSB_SENSOR_BAND && p.sensor != LSB_SENSOR_SIGNED) { why = "unknown sensor"; return LSB_EINVAL; }
  (void)d;
  return LSB_OK;
}

void fill_physics(lsb_grid *g, LevelDev &L, const CaseHost &ch) {
  const lsb_params &p = ch.p;
  const float scale = (float)L.scale;
  for (int k = 0; k < 2; ++k) {
    const double nu = p.nu[k] / L.scale;
    L.tau[k] = (float)(3.0 * nu + 0.5);
    L.omega[k] = (float)(1.0 / (3.0 * nu + 0.5));
    for (int a = 0; a < 3; ++a) L.acc[k][a] = (float)((p.gravity[a] + p.body_force[a] / p.rho[k]) * scale);
    L.rho_phys[k] = (float)p.rho[k];
    L.eta[k] = (float)(p.rho[k] * p.nu[k]);
  }
  for (int f = 0; f < 6; ++f)
    for (int a = 0; a < 3; ++a) L.wall_u[f][a] = (float)ch.d.wall_u[f][a];
  L.sigma = (float)p.sigma;
  L.dtau_ext = (float)p.dtau_ext;
  L.dtau_reinit = (float)p.dtau_reinit;
  for (int a = 0; a < 3; ++a) {
    L.x_ref[a] = (float)p.x_ref[a];
    L.grav[a] = (float)p.gravity[a];
  }
  L.ls_active = p.ls_active;
  L.p_gas0 = (float)p.p_gas0;
  for (int k = 0; k < 2; ++k) L.cumulant[k] = ch.d.collision[k] == LSB_CUMULANT;
  (void)g;
}

// Tensor maps for the TMA-staged collide kernel: per level descriptor and
// buffer, a (x, y, [z,] q) view of that level's populations with a box of one
// block x all Q populations; then, when a block row of tags is whole 16-byte
// units, per level descriptor an (x, y, [z]) view of its cell tags with a box
// of one block.  Leaves d_tmaps NULL when the driver entry point is
// unavailable; the plain kernel is used then.
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// The (x, y, [z,] q) view of level L's populations in the state array at buf, with a box of
// one block x all Q populations.
bool encode_pop_map(const lsb_grid *g, EncodeTiledFn encode, void *buf, const LevelDev &L, CUtensorMap *out) {
  const size_t es = g->storage == LSB_FP32 ? 4 : 2;
  const CUtensorMapDataType dt =
      g->storage == LSB_FP32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
  char *base = static_cast<char *>(buf) + (size_t)L.cell_off * g->Q * es;
  cuuint64_t dims[4], strides[3];
  cuuint32_t box[4], estr[4] = {1, 1, 1, 1};
  cuuint32_t rank;
  if (g->D == 3) {
    rank = 4;
    dims[0] = L.p[0]; dims[1] = L.p[1]; dims[2] = L.p[2]; dims[3] = g->Q;
    strides[0] = (cuuint64_t)L.p[0] * es;
    strides[1] = (cuuint64_t)L.p[0] * L.p[1] * es;
    strides[2] = (cuuint64_t)L.ncell * es;
    box[0] = g->bs[0]; box[1] = g->bs[1]; box[2] = g->bs[2]; box[3] = g->Q;
  } else {
    rank = 3;
    dims[0] = L.p[0]; dims[1] = L.p[1]; dims[2] = g->Q;
    strides[0] = (cuuint64_t)L.p[0] * es;
    strides[1] = (cuuint64_t)L.ncell * es;
    box[0] = g->bs[0]; box[1] = g->bs[1]; box[2] = g->Q;
  }
  return encode(out, dt, rank, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

lsb_status build_tensor_maps(lsb_grid *g) {
  void *fn = nullptr;
  cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
  if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
      q != cudaDriverEntryPointSuccess || !fn) {
    cudaGetLastError();
    return LSB_OK;
  }
  EncodeTiledFn encode = reinterpret_cast<EncodeTiledFn>(fn);
  const size_t es = g->storage == LSB_FP32 ? 4 : 2;
  // A box row must be whole 16-byte units: then every block's x origin is 16-byte aligned too.
  if ((g->bs[0] * es) % 16 != 0 || g->bs[0] > 256 || g->bs[1] > 256 || g->bs[2] > 256) return LSB_OK;
  const bool tags = g->bs[0] % 16 == 0;  // tag rows of whole 16-byte units (cell_off, p[0] follow)
  std::vector<CUtensorMap> maps((tags ? 3 : 2) * g->lds.size());
  for (size_t ld = 0; ld < g->lds.size(); ++ld) {
    const LevelDev &L = g->lds[ld];
    for (int b = 0; b < 2; ++b)
      if (!encode_pop_map(g, encode, g->d_buf[b], L, &maps[2 * ld + b])) return LSB_OK;  // keep the plain kernel
    if (tags) {
      cuuint64_t dims[3] = {(cuuint64_t)L.p[0], (cuuint64_t)L.p[1], (cuuint64_t)L.p[2]};
      cuuint64_t strides[2] = {(cuuint64_t)L.p[0], (cuuint64_t)L.p[0] * L.p[1]};
      cuuint32_t box[3] = {(cuuint32_t)g->bs[0], (cuuint32_t)g->bs[1], (cuuint32_t)g->bs[2]}, estr[3] = {1, 1, 1};
      CUresult r = encode(&maps[2 * g->lds.size() + ld], CU_TENSOR_MAP_DATA_TYPE_UINT8, g->D == 3 ? 3 : 2,
                          g->d_tag + L.cell_off, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                          CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
      if (r != CUDA_SUCCESS) return LSB_OK;
    }
  }
  int per_sm = 0, nsm = 0, dev = 0;
  CU(cudaGetDevice(&dev));
  CU(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  if (prepare_collide_stream_tma(g->Q, g->storage, g->nthreads, &per_sm) != cudaSuccess || per_sm < 1) {
    cudaGetLastError();
    return LSB_OK;
  }
  TRY(dalloc(g, &g->d_tmaps, sizeof(CUtensorMap) * maps.size()));
  CU(cudaMemcpy(g->d_tmaps, maps.data(), sizeof(CUtensorMap) * maps.size(), cudaMemcpyHostToDevice));
  g->tma_grid = per_sm * nsm;
  g->tma_tags = tags;
  int obs_sm = 0;
  if (prepare_observables_tma(g->Q, g->storage, g->nthreads, &obs_sm) == cudaSuccess && obs_sm >= 1)
    g->obs_tma_grid = obs_sm * nsm;
  else
    cudaGetLastError();
  g->encode_fn = fn;
  return LSB_OK;
}

void drop_graphs(lsb_grid *g) {
  for (int k = 0; k < 2; ++k)
    for (int p = 0; p < 2; ++p)
      if (g->gexec[k][p]) {
        cudaGraphExecDestroy(g->gexec[k][p]);
        g->gexec[k][p] = nullptr;
      }
}

// Graph replay needs a non-default stream, no kernel timing, and a fixed
// launch sequence (reinitialisation every finest step or never).
bool graphs_usable(const lsb_grid *g) {
  return g->use_graphs && g->stream && g->prof_mode == 0 && g->reinit_every <= 1;
}

// One or two coarse steps as one CUDA graph, one graph per starting parity of
// level 0.  A coarse step advances level l 2^l times, so every finer level's
// parity is the same at the start of every coarse step and level 0's alone
// alternates: the graph for (steps, level-0 parity) always meets the buffers it
// was captured with, until the next regrid rebuilds the work lists.
lsb_status replay_steps(lsb_grid *g, int nsteps) {
  const int p0 = g->par[0], ks = nsteps - 1;
  if (!g->gexec[ks][p0]) {
    int par[MAXL];
    long long fs[MAXL];
    std::copy(g->par, g->par + MAXL, par);
    std::copy(g->fine_steps, g->fine_steps + MAXL, fs);
    const uint64_t l0 = g->launches;
    CU(cudaStreamBeginCapture(g->stream, cudaStreamCaptureModeThreadLocal));
    lsb_status s = LSB_OK;
    for (int k = 0; k < nsteps && s == LSB_OK; ++k) s = advance(g, 0);
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(g->stream, &graph);
    std::copy(par, par + MAXL, g->par);
    std::copy(fs, fs + MAXL, g->fine_steps);
    g->gnodes[ks][p0] = g->launches - l0;
    g->launches = l0;
    if (s != LSB_OK) {
      if (graph) cudaGraphDestroy(graph);
      return s;
    }
    if (e != cudaSuccess) return fail(g, LSB_ECUDA, "graph capture: %s", cudaGetErrorString(e));
    e = cudaGraphInstantiate(&g->gexec[ks][p0], graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return fail(g, LSB_ECUDA, "graph instantiate: %s", cudaGetErrorString(e));
  }
  CU(cudaGraphLaunch(g->gexec[ks][p0], g->stream));
  g->launches += g->gnodes[ks][p0];
  for (int l = 0; l < MAXL; ++l) {
    // level l advances 2^l times per coarse step; its parity flips that often
    const long long adv = (long long)nsteps << l;
    if (l < g->Lmax) {
      if (adv & 1) g->par[l] ^= 1;
      if (has_finest(g, l)) g->fine_steps[l] += adv;
    }
  }
  for (int k = 0; k < nsteps; ++k) {
    g->updates_done += updates_per_step(g);
    g->coarse_steps++;
  }
  return LSB_OK;
}

// Populations of every level (floats; the adjoint needs FP32 storage).
size_t state_floats(const lsb_grid *g) { return (size_t)g->Q * (size_t)g->ncell_total; }

void rec_clear(lsb_grid *g) {
  for (float *p : g->rec_ckpt) cudaFree(p);
  g->rec_ckpt.clear();
  g->rec_on = 0;
  g->rec_steps = 0;
  g->adj_cur = -1;
}

// One stored state: the populations, plus phi and u~ (finest level) when the level set moves.
size_t slot_floats(const lsb_grid *g) {
  return state_floats(g) + (g->rec_moving ? (size_t)(1 + g->D) * g->nfine : 0);
}

// Copy the current state into a new checkpoint at the start of a recorded step.
lsb_status rec_checkpoint(lsb_grid *g) {
  const size_t bytes = sizeof(float) * slot_floats(g);
  float *p = nullptr;
  cudaError_t e = cudaMalloc(&p, bytes);
  if (e != cudaSuccess) return fail(g, LSB_ENOMEM, "checkpoint cudaMalloc(%zu): %s", bytes, cudaGetErrorString(e));
  g->rec_ckpt.push_back(p);
  const size_t sf = state_floats(g);
  if (g->Lmax > 1) TRY(snapshot(g, p));
  else CU(cudaMemcpyAsync(p, g->d_buf[g->par[0]], sizeof(float) * sf, cudaMemcpyDeviceToDevice, g->stream));
  if (g->rec_moving) {
    CU(cudaMemcpyAsync(p + sf, g->d_phi, sizeof(float) * g->nfine, cudaMemcpyDeviceToDevice, g->stream));
    CU(cudaMemcpyAsync(p + sf + g->nfine, g->d_ut[0], sizeof(float) * g->D * g->nfine, cudaMemcpyDeviceToDevice,
                       g->stream));
  }
  return LSB_OK;
}

// Scratch of the moving level-set adjoint, carved from one allocation (finest-level
// arrays of nfine floats; "vector" arrays hold D planes).
struct LsaPtrs {
  float *S;                       // S_0 .. S_n_ext: u~ after the interface pass and each sweep
  float *U1;                      // committed u~ of the step
  float *PHI0, *PS, *A1, *A2, *R1, *R2, *SS, *KP;
  float *NV;                      // normals of phi_n (D planes)
  float *L0r, *L1, *L2, *LS0;     // RK3 adjoints and d/dS0
  float *LA, *LK[2], *LOFF, *LV;  // adjoints of the extension (D planes each)
  float *LP[2];                   // adjoint of phi (ping-pong)
  float *LU[2];                   // adjoint of u~ (ping-pong, D planes)
  uint8_t *FR;                    // frozen cells of the reinitialisation
};

size_t lsa_floats_needed(const lsb_grid *g) {
  const size_t NF = g->nfine, D = g->D;
  return NF * (D * (g->n_ext + 1) + D + 8 + D + 4 + 5 * D + 2 + 2 * D) + NF / 4 + 64;
}

LsaPtrs lsa_ptrs(const lsb_grid *g) {
  const size_t NF = g->nfine, D = g->D;
  float *p = g->d_lsa;
  auto take = [&](size_t planes) {
    float *r = p;
    p += planes * NF;
    return r;
  };
  LsaPtrs P;
  P.S = take(D * (g->n_ext + 1));
  P.U1 = take(D);
  P.PHI0 = take(1); P.PS = take(1); P.A1 = take(1); P.A2 = take(1);
  P.R1 = take(1); P.R2 = take(1); P.SS = take(1); P.KP = take(1);
  P.NV = take(D);
  P.L0r = take(1); P.L1 = take(1); P.L2 = take(1); P.LS0 = take(1);
  P.LA = take(D); P.LK[0] = take(D); P.LK[1] = take(D); P.LOFF = take(D); P.LV = take(D);
  P.LP[0] = take(1); P.LP[1] = take(1);
  P.LU[0] = take(D); P.LU[1] = take(D);
  P.FR = reinterpret_cast<uint8_t *>(p);
  return P;
}

// Working buffers of the reverse sweep, allocated on first use.
lsb_status adj_buffers(lsb_grid *g, int seg_len) {
  const size_t sb = sizeof(float) * state_floats(g);
  const int MF = 1 + g->D + g->D * (g->D + 1) / 2;
  if (!g->d_adj[0]) {
    TRY(dalloc(g, &g->d_adj[0], sb));
    TRY(dalloc(g, &g->d_adj[1], sb));
    TRY(dalloc(g, &g->d_fsave, sb));
    TRY(dalloc(g, &g->d_madj, sizeof(float) * (size_t)MF * g->nfine));
    TRY(dalloc(g, &g->d_linkadj, sizeof(float) * 2 * (size_t)g->link_cap));
    TRY(dalloc(g, &g->d_grad, sizeof(double) * NG_ADJ * g->ncase));
    TRY(dalloc(g, &g->d_wobs, sizeof(double) * (4 + 2 * g->D) * g->ncase));
    TRY(dalloc(g, &g->d_gphi, sizeof(float) * (size_t)g->nfine));
    TRY(dalloc(g, &g->d_gn, sizeof(float) * (size_t)g->D * g->nfine));
    TRY(dalloc(g, &g->d_gk, sizeof(float) * (size_t)g->nfine));
    CU(cudaMemsetAsync(g->d_madj, 0, sizeof(float) * (size_t)MF * g->nfine, g->stream));
  }
  const size_t slb = sizeof(float) * slot_floats(g);
  if (seg_len > g->seg_cap || g->seg_slot != slb) {
    if (g->d_seg) cudaFree(g->d_seg);
  if (g->d_seg_tmaps) cudaFree(g->d_seg_tmaps);
    g->d_seg = nullptr;
    g->seg_cap = 0;
    cudaError_t e = cudaMalloc(&g->d_seg, slb * (size_t)seg_len);
    if (e != cudaSuccess) return fail(g, LSB_ENOMEM, "segment store cudaMalloc(%zu): %s", slb * seg_len,
                                      cudaGetErrorString(e));
    g->seg_cap = seg_len;
    g->seg_slot = slb;
    // tensor maps of every slot (both parity entries name the slot), so that the
    // recomputation reads its slots through the TMA-staged collide kernel
    if (g->d_seg_tmaps) cudaFree(g->d_seg_tmaps);
    g->d_seg_tmaps = nullptr;
    if (g->d_tmaps && g->encode_fn) {
      const size_t nld = g->lds.size();
      std::vector<CUtensorMap> maps(2 * nld * (size_t)seg_len);
      bool ok = true;
      for (int j = 0; j < seg_len && ok; ++j)
        for (size_t ld = 0; ld < nld && ok; ++ld) {
          CUtensorMap *m = &maps[(j * nld + ld) * 2];
          ok = encode_pop_map(g, reinterpret_cast<EncodeTiledFn>(g->encode_fn), g->d_seg + slot_floats(g) * j,
                              g->lds[ld], m);
          m[1] = m[0];
        }
      if (ok && cudaMalloc(&g->d_seg_tmaps, sizeof(CUtensorMap) * maps.size()) == cudaSuccess)
        CU(cudaMemcpy(g->d_seg_tmaps, maps.data(), sizeof(CUtensorMap) * maps.size(), cudaMemcpyHostToDevice));
      else
        cudaGetLastError();
    }
  }
  if (g->rec_moving) {
    const size_t need = lsa_floats_needed(g);
    if (g->lsa_floats < need) {
      if (g->d_lsa) cudaFree(g->d_lsa);
      g->d_lsa = nullptr;
      g->lsa_floats = 0;
      cudaError_t e = cudaMalloc(&g->d_lsa, sizeof(float) * need);
      if (e != cudaSuccess) return fail(g, LSB_ENOMEM, "level-set adjoint scratch cudaMalloc: %s", cudaGetErrorString(e));
      g->lsa_floats = need;
    }
    CU(cudaMemsetAsync(g->d_lsa, 0, sizeof(float) * g->lsa_floats, g->stream));
    if (!g->d_phisave) {
      TRY(dalloc(g, &g->d_phisave, sizeof(float) * g->nfine));
      TRY(dalloc(g, &g->d_utsave, sizeof(float) * g->D * g->nfine));
    }
  }
  return LSB_OK;
}

// The lattice Boltzmann part of one reverse (sub-)step of level l (whose cut links
// and moment adjoints exist on the finest level only): lambda at the state F of the
// step's start into lamO from lamN, the adjoint after it.
lsb_status adj_lb(lsb_grid *g, int l, const float *F, float *lamN, float *lamO, GeoAdj G, float *phi = nullptr,
                  float *nvec = nullptr, float *kappa = nullptr) {
  Ctx C = make_ctx(g);
  if (phi) C.phi = phi;  // geometry of phi_n when the level set moves
  if (nvec) C.nvec = nvec;
  if (kappa) C.kappa = kappa;
  BlockShape S = shape(g);
  const int Q = g->Q;
  const bool fine = l == g->Lmax - 1;
  if (fine)
    RUN(KADJ_LINKS, 0, 1, 128, run_adj_links, Q, LN(g, DYN_GRID, 128), C, l, F, lamN, g->d_linkadj, g->d_madj,
        g->d_grad, g->ncase, G);
  const int grid = std::min(g->cs[l].n, 152);
  RUN(KADJ_COLLIDE, 3.0 * Q * sizeof(float) * g->leaf_cells[l], g->cs[l].n, g->nthreads, run_adj_collide, Q,
      LN(g, grid, g->nthreads), C, S, (const int *)g->cs[l].d, g->cs[l].n, F, (const float *)lamN, lamO,
      (const float *)g->d_linkadj, g->d_grad);
  if (fine)
    RUN(KADJ_MACRO, 0, 1, 128, run_adj_macro, Q, LN(g, DYN_GRID, 128), C, l, F, lamO, g->d_madj, g->d_grad,
        g->ncase);
  return LSB_OK;
}

// One reverse step of a single-level grid: lambda_n from lambda_{n+1} = d_adj[cur] at F = f_n.
lsb_status adj_step(lsb_grid *g, const float *F, int cur, GeoAdj G) {
  return adj_lb(g, 0, F, g->d_adj[cur], g->d_adj[1 - cur], G);
}

// One reverse step with a moving level set: replay the level-set passes of step n
// from (f_n, phi_n, u~_n), then the transposes in reverse order (reinitialisation,
// transport, extension, interface velocity), then the lattice Boltzmann part with
// the geometry of phi_n.  l is the finest level; population adjoints lamN -> lamO, the
// level set's LP[cur], LU[cur] -> LP[1 - cur], LU[1 - cur].
lsb_status adj_moving(lsb_grid *g, int l, const float *F, float *phi_n, const float *ut_n, float *lamN, float *lamO,
                      int cur) {
  const LsaPtrs P = lsa_ptrs(g);
  const int Q = g->Q, D = g->D, nt = g->nthreads;
  const long long NF = g->nfine;
  const size_t b1 = sizeof(float) * NF, bD = sizeof(float) * D * NF;
  const Ctx base = make_ctx(g);
  const BlockShape S = shape(g);
  const int nb = std::max(1, std::min(g->band_cap, 152 * 16));
  auto Sk = [&](int k) { return P.S + (size_t)k * D * NF; };
  // ---- replay of the level-set passes of step n
  CU(cudaMemcpyAsync(Sk(0), ut_n, bD, cudaMemcpyDeviceToDevice, g->stream));
  Ctx R = base;
  R.phi = phi_n;
  RUN(KLSA, 0, 1, 128, run_lsa_init, Q, LN(g, DYN_GRID, 128), R, l, F, Sk(0));
  Ctx E = base;
  E.phi = phi_n;
  E.ut0 = Sk(0);
  for (int k = 0; k < g->n_ext; ++k)
    RUN(KLSA, 0, nb, nt, run_ext_iter, D, LN(g, nb, nt), E, S, l, Sk(k), Sk(k + 1), k == 0 ? 2 : 3);
  CU(cudaMemcpyAsync(P.U1, Sk(0), bD, cudaMemcpyDeviceToDevice, g->stream));
  if (g->n_ext > 0) {
    Ctx Cm = base;
    Cm.ut0 = P.U1;
    RUN(KLSA, 0, nb, nt, run_ext_iter, D, LN(g, nb, nt), Cm, S, l, Sk(g->n_ext), (float *)nullptr, 1);
  }
  CU(cudaMemcpyAsync(P.PHI0, phi_n, b1, cudaMemcpyDeviceToDevice, g->stream));
  Ctx A = base;
  A.phi = P.PHI0;
  A.p1 = P.A1;
  A.p2 = P.A2;
  A.ut0 = P.U1;
  for (int st = 1; st <= 3; ++st) RUN(KLSA, 0, nb, nt, run_adv_stage, D, LN(g, nb, nt), A, S, l, st);
  const bool rein = g->reinit_every == 1 && g->n_reinit > 0;
  Ctx Rt = base;
  Rt.phi = P.PS;
  Rt.p1 = P.R1;
  Rt.p2 = P.R2;
  Rt.frozen = P.FR;
  Rt.s0 = P.SS;
  if (rein) {
    CU(cudaMemcpyAsync(P.PS, P.PHI0, b1, cudaMemcpyDeviceToDevice, g->stream));
    RUN(KLSA, 0, nb, nt, run_reinit_prep, Q, LN(g, nb, nt), Rt, S, l);
    Ctx Rs = Rt;
    Rs.phi = P.PHI0;
    for (int st = 1; st <= 3; ++st) RUN(KLSA, 0, nb, nt, run_reinit_stage, D, LN(g, nb, nt), Rs, S, l, st);
  }
  Ctx Gm = base;
  Gm.phi = phi_n;
  Gm.nvec = P.NV;
  Gm.kappa = P.KP;
  RUN(11, 0, 1, 128, run_geometry, D, LN(g, DYN_GRID, 128), Gm, l, 0);
  // ---- transposes
  float *LPin = P.LP[cur], *LPout = P.LP[1 - cur], *LUin = P.LU[cur], *LUout = P.LU[1 - cur];
  const float *lps = LPin;
  if (rein) {
    CU(cudaMemcpyAsync(P.L0r, LPin, b1, cudaMemcpyDeviceToDevice, g->stream));
    CU(cudaMemsetAsync(P.LS0, 0, b1, g->stream));
    RUN(KLSA, 0, nb, nt, run_lsa_mix, D, LN(g, nb, nt), Rt, S, l, 0, 1, LPin, P.L0r, P.L1, P.L2, P.LS0);
    RUN(KLSA, 0, nb, nt, run_lsa_reinit_rt, D, LN(g, nb, nt), Rt, S, l, P.R2, LPin, 2.0f / 3.0f, P.L2, P.L0r, P.LS0);
    RUN(KLSA, 0, nb, nt, run_lsa_mix, D, LN(g, nb, nt), Rt, S, l, 1, 1, LPin, P.L0r, P.L1, P.L2, P.LS0);
    RUN(KLSA, 0, nb, nt, run_lsa_reinit_rt, D, LN(g, nb, nt), Rt, S, l, P.R1, P.L2, 0.25f, P.L1, P.L0r, P.LS0);
    RUN(KLSA, 0, nb, nt, run_lsa_mix, D, LN(g, nb, nt), Rt, S, l, 2, 1, LPin, P.L0r, P.L1, P.L2, P.LS0);
    RUN(KLSA, 0, nb, nt, run_lsa_reinit_rt, D, LN(g, nb, nt), Rt, S, l, P.PS, P.L1, 1.0f, P.L0r, P.L0r, P.LS0);
    RUN(KLSA, 0, nb, nt, run_lsa_mix, D, LN(g, nb, nt), Rt, S, l, 3, 1, LPin, P.L0r, P.L1, P.L2, P.LS0);
    lps = P.L0r;
  }
  Ctx At = base;
  At.phi = phi_n;
  At.p1 = P.A1;
  At.p2 = P.A2;
  At.ut0 = P.U1;
  CU(cudaMemcpyAsync(LPout, lps, b1, cudaMemcpyDeviceToDevice, g->stream));
  CU(cudaMemcpyAsync(P.LA, LUin, bD, cudaMemcpyDeviceToDevice, g->stream));
  RUN(KLSA, 0, nb, nt, run_lsa_mix, D, LN(g, nb, nt), At, S, l, 0, 0, lps, LPout, P.L1, P.L2, P.LS0);
  RUN(KLSA, 0, nb, nt, run_lsa_adv_rt, D, LN(g, nb, nt), At, S, l, P.A2, lps, 2.0f / 3.0f, P.L2, LPout, P.LA);
  RUN(KLSA, 0, nb, nt, run_lsa_mix, D, LN(g, nb, nt), At, S, l, 1, 0, lps, LPout, P.L1, P.L2, P.LS0);
  RUN(KLSA, 0, nb, nt, run_lsa_adv_rt, D, LN(g, nb, nt), At, S, l, P.A1, P.L2, 0.25f, P.L1, LPout, P.LA);
  RUN(KLSA, 0, nb, nt, run_lsa_mix, D, LN(g, nb, nt), At, S, l, 2, 0, lps, LPout, P.L1, P.L2, P.LS0);
  RUN(KLSA, 0, nb, nt, run_lsa_adv_rt, D, LN(g, nb, nt), At, S, l, (const float *)phi_n, P.L1, 1.0f, LPout, LPout,
      P.LA);
  float *Lc = P.LA;
  if (g->n_ext > 0) {
    CU(cudaMemsetAsync(P.LOFF, 0, bD, g->stream));
    for (int k = g->n_ext - 1; k >= 0; --k) {
      float *out = Lc == P.LK[0] ? P.LK[1] : P.LK[0];
      CU(cudaMemcpyAsync(out, Lc, bD, cudaMemcpyDeviceToDevice, g->stream));
      RUN(KLSA, 0, nb, nt, run_lsa_ext_T, D, LN(g, nb, nt), E, S, l, (const float *)Sk(k), (const float *)Sk(0),
          (const float *)Lc, out, P.LOFF, P.LV);
      Lc = out;
    }
    RUN(KLSA, 0, nb, nt, run_lsa_ext_v, D, LN(g, nb, nt), E, S, l, P.LV, LPout);
    RUN(KLSA, 0, 1, 256, run_lsa_axpy, LN(g, 152 * 8, 256), (long long)D * NF, (const float *)P.LOFF, Lc);
  }
  RUN(KLSA, 0, 1, 128, run_lsa_init_T, Q, LN(g, DYN_GRID, 128), R, l, F, Lc, g->d_madj, LPout);
  CU(cudaMemcpyAsync(LUout, Lc, bD, cudaMemcpyDeviceToDevice, g->stream));
  // lattice Boltzmann part with the geometry of phi_n; its phi adjoint goes to LPout
  const GeoAdj G{LPout, g->d_gn, g->d_gk};
  TRY(adj_lb(g, l, F, lamN, lamO, G, phi_n, P.NV, P.KP));
  RUN(KADJ_GEOM, 0, 1, 128, run_adj_geometry, D, LN(g, DYN_GRID, 128), R, l, G);
  CU(cudaMemsetAsync(g->d_gn, 0, bD, g->stream));
  CU(cudaMemsetAsync(g->d_gk, 0, b1, g->stream));
  return LSB_OK;
}

// Multi-level grids: tape buffers for one replayed coarse step (a full-size state
// per call of the level recursion, two for calls of non-finest levels) and the
// zeroed scratch of the ghost rings' coarse shares.
lsb_status amr_buffers(lsb_grid *g) {
  const size_t sb = sizeof(float) * state_floats(g);
  const int ncall = (1 << g->Lmax) - 1;
  if (g->rec_moving && g->tape_ls.size() != (size_t)ncall) {  // finest calls only; others stay null
    for (float *p : g->tape_ls) cudaFree(p);
    g->tape_ls.assign(ncall, nullptr);
    bool ok = true;
    std::function<void(int, int)> walk = [&](int l, int c) {  // c: preorder index of a call of level l
      if (l == g->Lmax - 1) {
        ok = ok && cudaMalloc(&g->tape_ls[c], sizeof(float) * (1 + g->D) * g->nfine) == cudaSuccess;
        return;
      }
      const int sub = (1 << (g->Lmax - l - 1)) - 1;  // calls in a child's subtree
      walk(l + 1, c + 1);
      walk(l + 1, c + 1 + sub);
    };
    walk(0, 0);
    if (!ok) return fail(g, LSB_ENOMEM, "adjoint level-set tape cudaMalloc");
  }
  if ((int)g->tape_old.size() == ncall) return LSB_OK;
  for (float *p : g->tape_old) cudaFree(p);
  for (float *p : g->tape_new) cudaFree(p);
  g->tape_old.assign(ncall, nullptr);
  g->tape_new.assign(ncall, nullptr);
  // preorder: call c sits at level lev[c]
  std::vector<int> lev;
  std::function<void(int)> walk = [&](int l) {
    lev.push_back(l);
    if (l + 1 < g->Lmax) {
      walk(l + 1);
      walk(l + 1);
    }
  };
  walk(0);
  for (int c = 0; c < ncall; ++c) {
    cudaError_t e = cudaMalloc(&g->tape_old[c], sb);
    if (e == cudaSuccess && lev[c] + 1 < g->Lmax) e = cudaMalloc(&g->tape_new[c], sb);
    if (e != cudaSuccess) return fail(g, LSB_ENOMEM, "adjoint tape cudaMalloc(%zu): %s", sb, cudaGetErrorString(e));
  }
  if (!g->d_adjx) TRY(dalloc(g, &g->d_adjx, sb));
  CU(cudaMemsetAsync(g->d_adjx, 0, sb, g->stream));
  return LSB_OK;
}

// Reverse of advance(g, l) for the call with preorder index `call` of the replayed
// step: the second fine sub-step, the ghost transfer at t + 1/2, the first fine
// sub-step, the ghost transfer at t, the level's own sub-step (links, collision and
// streaming, moment adjoints on the finest level), the ghost rings' share of the
// level's state at t, and the restriction, whose adjoint goes to the finer level.
lsb_status adj_amr(lsb_grid *g, int l, int call, GeoAdj G) {
  const int Q = g->Q, Lm = g->Lmax;
  const bool last = l == Lm - 1;
  const Ctx C = make_ctx(g);
  const BlockShape S = shape(g);
  const float *Fold = g->tape_old[call];
  float *lamN = g->d_adj[g->apar[l]], *lamO = g->d_adj[1 - g->apar[l]];
  const int tb = 128;
  if (!last) {
    const int sub = (1 << (Lm - l - 1)) - 1;  // calls in a child's subtree
    const int c1 = call + 1, c2 = call + 1 + sub;
    const CellList &gc = g->ghost_cells[l + 1];
    const int gg = std::max(1, std::min((gc.n + tb - 1) / tb, DYN_GRID));
    TRY(adj_amr(g, l + 1, c2, G));
    // the finer level's adjoint after the sub-step is the input its transpose just read
    RUN(KADJ_GHOST, 0, gc.n, tb, run_adj_ghost, Q, LN(g, gg, tb), C, (const int2 *)gc.d, gc.n, 0.5f, Fold,
        (const float *)g->tape_new[call], (const float *)g->d_adj[1 - g->apar[l + 1]], g->d_adjx, lamN, g->d_grad,
        g->ncase);
    TRY(adj_amr(g, l + 1, c1, G));
    RUN(KADJ_GHOST, 0, gc.n, tb, run_adj_ghost, Q, LN(g, gg, tb), C, (const int2 *)gc.d, gc.n, 0.0f, Fold,
        (const float *)nullptr, (const float *)g->d_adj[1 - g->apar[l + 1]], g->d_adjx, lamN, g->d_grad, g->ncase);
  }
  if (last && g->rec_moving) {  // finest sub-step with the level set transported
    float *t = g->tape_ls[call];
    TRY(adj_moving(g, l, Fold, t, t + g->nfine, lamN, lamO, g->lspar));
    g->lspar ^= 1;
  } else {
    TRY(adj_lb(g, l, Fold, lamN, lamO, G));
  }
  if (!last) {
    const CellList &gc = g->ghost_cells[l + 1];
    const int gg = std::max(1, std::min((gc.n + tb - 1) / tb, DYN_GRID));
    RUN(KADJ_GAPPLY, 0, gc.n, tb, run_adj_ghost_apply, Q, LN(g, gg, tb), C, (const int2 *)gc.d, gc.n, g->d_adjx,
        lamO);
  }
  g->apar[l] ^= 1;
  if (!last) {
    const CellList &rc = g->rl_cells[l];
    const int rg = std::max(1, std::min((rc.n + tb - 1) / tb, DYN_GRID));
    RUN(KADJ_RESTRICT, 0, rc.n, tb, run_adj_restrict, Q, LN(g, rg, tb), C, (const int2 *)rc.d, rc.n,
        (const float *)g->tape_old[call + 1], lamO, g->d_adj[g->apar[l + 1]], g->d_grad, g->ncase);
  }
  return LSB_OK;
}

// Reverse sweep over a multi-level recording (frozen level set): segments are
// recomputed from their checkpoints with every coarse step's start state stored
// (but the last's, whose start is the working state when the recomputation ends);
// each step is then replayed once more with the tape on and transposed.  The
// adjoint of the final observables is already in d_adj[0] (every level).
lsb_status backward_amr(lsb_grid *g, GeoAdj G) {
  const long long T = g->rec_steps;
  const int every = g->rec_every;
  const size_t sl = slot_floats(g), sf = state_floats(g), NF = g->nfine;
  TRY(amr_buffers(g));
  for (int l = 0; l < MAXL; ++l) g->apar[l] = 0;
  g->lspar = 0;
  // a stored state: every level's populations, and with a moving level set phi and u~ after
  // them; a loaded one is reclassified (interface geometry and lists of its phi)
  auto save = [&](float *dst) -> lsb_status {
    TRY(snapshot(g, dst));
    if (g->rec_moving) {
      CU(cudaMemcpyAsync(dst + sf, g->d_phi, sizeof(float) * NF, cudaMemcpyDeviceToDevice, g->stream));
      CU(cudaMemcpyAsync(dst + sf + NF, g->d_ut[0], sizeof(float) * g->D * NF, cudaMemcpyDeviceToDevice, g->stream));
    }
    return LSB_OK;
  };
  auto load = [&](const float *src) -> lsb_status {
    TRY(restore(g, src));
    if (g->rec_moving) {
      CU(cudaMemcpyAsync(g->d_phi, src + sf, sizeof(float) * NF, cudaMemcpyDeviceToDevice, g->stream));
      CU(cudaMemcpyAsync(g->d_ut[0], src + sf + NF, sizeof(float) * g->D * NF, cudaMemcpyDeviceToDevice, g->stream));
      TRY(ls_mirror(g));
      TRY(classify(g, g->Lmax - 1, 0));
    }
    return LSB_OK;
  };
  const long long nseg = (T + every - 1) / every;
  for (long long sgi = nseg - 1; sgi >= 0; --sgi) {
    const long long start = sgi * every;
    const int len = (int)std::min<long long>(every, T - start);
    TRY(load(g->rec_ckpt[sgi]));
    for (int j = 0; j + 1 < len; ++j) {
      TRY(save(g->d_seg + sl * j));
      TRY(advance(g, 0));
    }
    // the working state is the start of the segment's last step: replayed first, as it is
    for (int j = len - 1; j >= 0; --j) {
      if (j + 1 < len) TRY(load(g->d_seg + sl * j));
      g->tape_on = 1;
      g->tape_call = 0;
      const lsb_status st = advance(g, 0);
      g->tape_on = 0;
      TRY(st);
      TRY(adj_amr(g, 0, 0, G));
    }
  }
  return LSB_OK;
}

}  // namespace

// ====================================================================== C ABI
extern "C" {

lsb_status lsb_create_grid(int n_cases, const lsb_grid_desc *descs, const lsb_params *params,
                           const float *const *phi0, void *stream, lsb_grid **out) {
  lsb_grid *g = nullptr;
  if (!out) return fail(nullptr, LSB_EINVAL, "out is NULL");
  *out = nullptr;
  if (n_cases < 1 || !descs || !params || !phi0) return fail(nullptr, LSB_EINVAL, "need n_cases >= 1 and arrays");
  const lsb_grid_desc &d0 = descs[0];
  if (d0.lattice != LSB_D2Q9 && d0.lattice != LSB_D3Q19 && d0.lattice != LSB_D3Q27)
    return fail(nullptr, LSB_EINVAL, "unknown lattice");
  if (d0.storage != LSB_FP32 && d0.storage != LSB_FP16S) return fail(nullptr, LSB_EINVAL, "unknown storage");
  if (d0.lattice == LSB_D3Q27 && d0.storage != LSB_FP32) return fail(nullptr, LSB_EINVAL, "D3Q27 needs FP32 storage");
  const int D = d0.lattice == LSB_D2Q9 ? 2 : 3;
  int bs[3] = {d0.block[0], d0.block[1], D == 3 ? d0.block[2] : 1};
  for (int a = 0; a < D; ++a)
    if (bs[a] < 2 || (bs[a] & (bs[a] - 1))) return fail(nullptr, LSB_EINVAL, "block edges must be powers of two >= 2");
  const int nthreads = bs[0] * bs[1] * bs[2];
  if (nthreads % 32 || nthreads > 512) return fail(nullptr, LSB_EINVAL, "block must hold 32..512 cells, a multiple of 32");
  for (int c = 0; c < n_cases; ++c) {
    const lsb_grid_desc &d = descs[c];
    if (d.lattice != d0.lattice || d.storage != d0.storage) return fail(nullptr, LSB_EINVAL, "cases must share lattice and storage");
    for (int a = 0; a < 3; ++a)
      if (d.block[a] != d0.block[a] && (a < D)) return fail(nullptr, LSB_EINVAL, "cases must share the block shape");
    if (d.n_levels < 1 || d.n_levels > MAXL) return fail(nullptr, LSB_EINVAL, "n_levels must be 1..%d", MAXL);
    for (int k = 0; k < 2; ++k) {
      if (d.collision[k] != LSB_BGK && d.collision[k] != LSB_CUMULANT)
        return fail(nullptr, LSB_EINVAL, "collision must be LSB_BGK or LSB_CUMULANT");
      if (d.collision[k] == LSB_CUMULANT && d.lattice != LSB_D3Q27)
        return fail(nullptr, LSB_EINVAL, "the cumulant collision needs D3Q27");
    }
    for (int a = 0; a < D; ++a) {
      if (d.base[a] < 1) return fail(nullptr, LSB_EINVAL, "base must be positive");
      if (d.bc[a] != LSB_PERIODIC && d.bc[a] != LSB_WALL && d.bc[a] != LSB_SLIP)
        return fail(nullptr, LSB_EINVAL, "bad bc");
    }
    std::string why;
    if (check_params(params[c], d, why)) return fail(nullptr, LSB_EINVAL, "case %d: %s", c, why.c_str());
    if (!phi0[c]) return fail(nullptr, LSB_EINVAL, "phi0[%d] is NULL", c);
    const lsb_params &p = params[c], &p0 = params[0];
    if (p.n_ext != p0.n_ext || p.reinit_every != p0.reinit_every || p.n_reinit != p0.n_reinit ||
        p.regrid_every != p0.regrid_every)
      return fail(nullptr, LSB_EINVAL, "cases must share the level-set iteration counts and regrid period");
  }
  if (d0.storage == LSB_FP16S && !(d0.fp16_scale > 0)) return fail(nullptr, LSB_EINVAL, "fp16_scale must be > 0");

  g = new lsb_grid();
  g->ncase = n_cases;
  g->Q = D == 2 ? 9 : (d0.lattice == LSB_D3Q27 ? 27 : 19);
  g->D = D;
  g->storage = d0.storage;
  g->fp16_scale = d0.storage == LSB_FP16S ? (float)d0.fp16_scale : 1.0f;
  for (int a = 0; a < 3; ++a) g->bs[a] = bs[a];
  g->nthreads = nthreads;
  g->stream = (cudaStream_t)stream;
  g->n_ext = params[0].n_ext;
  g->reinit_every = params[0].reinit_every;
  g->n_reinit = params[0].n_reinit;
  g->regrid_every = params[0].regrid_every;
  // level descriptors
  long long cell_off = 0, fine_off = 0;
  int block_off = 0;
  for (int c = 0; c < n_cases; ++c) {
    CaseHost ch;
    ch.d = descs[c];
    ch.p = params[c];
    ch.L = descs[c].n_levels;
    ch.ld0 = (int)g->lds.size();
    g->Lmax = std::max(g->Lmax, ch.L);
    for (int l = 0; l < ch.L; ++l) {
      LevelDev L;
      memset(&L, 0, sizeof L);
      L.case_id = c;
      L.level = l;
      L.n_levels = ch.L;
      L.finest = l == ch.L - 1;
      L.scale = 1 << (ch.L - 1 - l);
      L.ncell = 1;
      for (int a = 0; a < 3; ++a) {
        L.n[a] = a < D ? descs[c].base[a] << l : 1;
        L.p[a] = ((L.n[a] + bs[a] - 1) / bs[a]) * bs[a];
        L.nb[a] = L.p[a] / bs[a];
        L.per[a] = a < D ? (descs[c].bc[a] == LSB_PERIODIC) : 1;
        L.slip[a] = a < D && descs[c].bc[a] == LSB_SLIP;
        L.ncell *= L.p[a];
      }
      L.nblock = L.nb[0] * L.nb[1] * L.nb[2];
      L.cell_off = cell_off;
      L.block_off = block_off;
      L.fine_off = L.finest ? fine_off : -1;
      L.parent_ld = l > 0 ? ch.ld0 + l - 1 : -1;
      L.child_ld = l < ch.L - 1 ? ch.ld0 + l + 1 : -1;
      L.fine_ld = ch.ld0 + ch.L - 1;
      fill_physics(g, L, ch);
      cell_off += L.ncell;
      block_off += L.nblock;
      if (L.finest) fine_off += L.ncell;
      g->lds.push_back(L);
    }
    g->cases.push_back(ch);
  }
  for (const LevelDev &L : g->lds)
    if ((double)L.ncell * (g->Q + 1) >= 4294967295.0) {
      lsb_destroy(g);
      return fail(nullptr, LSB_EINVAL, "a level holds %lld cells; Q x cells must stay below 2^32", L.ncell);
    }
  g->ncell_total = cell_off;
  g->nblock_total = block_off;
  g->nfine = fine_off;
  const long long nf = g->nfine;
  const int Q = g->Q;
  const size_t fsz = g->storage == LSB_FP32 ? 4 : 2;
  const int MF = 1 + D + D * (D + 1) / 2;
  g->list_cap = std::min<long long>(nf, std::max<long long>(1 << 16, nf / 4));
  g->link_cap = std::min<long long>((long long)Q * nf, std::max<long long>(1 << 18, 2 * nf));
  g->band_cap = 0;
  for (const LevelDev &L : g->lds)
    if (L.finest) g->band_cap += L.nblock;
  lsb_status s = LSB_OK;
#define ALLOC(ptr, bytes)                              \
  do {                                             \
    s = dalloc(g, &(ptr), (size_t)(bytes));        \
    if (s) { g_create_error = g->err; lsb_destroy(g); return s; } \
  } while (0)
  ALLOC(g->d_lds, sizeof(LevelDev) * g->lds.size());
  ALLOC(g->d_blk_ld, sizeof(int) * g->nblock_total);
  ALLOC(g->d_blk_info, sizeof(int4) * g->nblock_total);
  ALLOC(g->d_bstat, g->nblock_total);
  ALLOC(g->d_bstat_old, g->nblock_total);
  ALLOC(g->d_bflag, g->nblock_total);
  ALLOC(g->d_tag, g->ncell_total);
  ALLOC(g->d_buf[0], fsz * Q * g->ncell_total);
  ALLOC(g->d_buf[1], fsz * Q * g->ncell_total);
  ALLOC(g->d_phi, 4 * nf);
  ALLOC(g->d_p1, 4 * nf);
  ALLOC(g->d_p2, 4 * nf);
  ALLOC(g->d_s0, 4 * nf);
  ALLOC(g->d_frozen, nf);
  for (int k = 0; k < 3; ++k) ALLOC(g->d_ut[k], 4 * D * nf);
  ALLOC(g->d_plan_v, 4 * D * nf);
  ALLOC(g->d_plan_f, nf);
  ALLOC(g->d_cmask, 4 * nf);
  ALLOC(g->d_cbase, 4 * nf);
  ALLOC(g->d_macro, 4 * (size_t)MF * nf);
  ALLOC(g->d_nvec, 4 * D * nf);
  ALLOC(g->d_kappa, 4 * nf);
  ALLOC(g->d_linkbuf, 8 * g->link_cap);
  {
    // the link list lives from one classification to the next step's bounce-back, so
    // every finest global level keeps its own region (the link buffer is shared)
    long long nl = 0;
    for (int l = 0; l < MAXL; ++l) {
      g->link_list_off[l] = nl * g->link_cap;
      bool fin = false;
      for (int c = 0; c < n_cases; ++c) fin = fin || (g->cases[c].L - 1 == l);
      if (fin) ++nl;
    }
    ALLOC(g->d_linkcell, 8 * g->link_cap * nl);
    ALLOC(g->d_linkdir, g->link_cap * nl);
  }
  ALLOC(g->d_counters, sizeof(int) * MAXL * NCOUNT);
  ALLOC(g->d_err, sizeof(int));
  ALLOC(g->d_work, sizeof(int) * 2 * MAXL);
  s = pin_host(g);
  if (s) { g_create_error = g->err; lsb_destroy(g); return s; }
  {
    int lo = 0, hi = 0;
    if (cudaDeviceGetStreamPriorityRange(&lo, &hi) == cudaSuccess) g->prio_hi = hi;
    else cudaGetLastError();
  }
  ALLOC(g->d_bar, 2 * sizeof(unsigned));
  ALLOC(g->d_iface, sizeof(int2) * MAXL * g->list_cap);
  ALLOC(g->d_flip, sizeof(int2) * MAXL * g->list_cap);
  ALLOC(g->d_band, sizeof(int) * MAXL * (size_t)std::max(1, g->band_cap));
  ALLOC(g->d_check, sizeof(int) * MAXL * (size_t)std::max(1, g->band_cap));
  ALLOC(g->d_band_info, sizeof(int4) * MAXL * (size_t)std::max(1, g->band_cap));
  ALLOC(g->d_obs, sizeof(double) * n_cases * 16);
  ALLOC(g->d_sens, sizeof(float) * g->nblock_total);
#undef ALLOC
  // block -> level descriptor
  std::vector<int> bl(g->nblock_total);
  std::vector<int4> binfo(g->nblock_total);
  for (size_t ld = 0; ld < g->lds.size(); ++ld)
    for (int b = 0; b < g->lds[ld].nblock; ++b) {
      bl[g->lds[ld].block_off + b] = (int)ld;
      int bc[3];
      block_coords(g->lds[ld], b, bc);
      binfo[g->lds[ld].block_off + b] = make_int4((int)ld, bc[0], bc[1], bc[2]);
    }
  auto cuerr = [&](cudaError_t e, const char *what) -> bool {
    if (e == cudaSuccess) return false;
    g_create_error = std::string(what) + ": " + cudaGetErrorString(e);
    return true;
  };
  if (cuerr(cudaMemcpy(g->d_lds, g->lds.data(), sizeof(LevelDev) * g->lds.size(), cudaMemcpyHostToDevice), "lds") ||
      cuerr(cudaMemcpy(g->d_blk_ld, bl.data(), sizeof(int) * bl.size(), cudaMemcpyHostToDevice), "blk_ld") ||
      cuerr(cudaMemcpy(g->d_blk_info, binfo.data(), sizeof(int4) * binfo.size(), cudaMemcpyHostToDevice), "blk_info") ||
      cuerr(cudaMemset(g->d_tag, 0, g->ncell_total), "tag") ||
      cuerr(cudaMemset(g->d_bflag, 0, g->nblock_total), "bflag") ||
      cuerr(cudaMemset(g->d_err, 0, sizeof(int)), "err") ||
      cuerr(cudaMemset(g->d_work, 0, sizeof(int) * 2 * MAXL), "work") ||
      cuerr(cudaMemset(g->d_bar, 0, 2 * sizeof(unsigned)), "barrier") ||
      cuerr(cudaMemset(g->d_counters, 0, sizeof(int) * MAXL * NCOUNT), "counters") ||
      cuerr(cudaMemset(g->d_cmask, 0, 4 * nf), "cmask") ||
      cuerr(cudaMemset(g->d_nvec, 0, 4 * D * nf), "nvec") ||
      cuerr(cudaMemset(g->d_kappa, 0, 4 * nf), "kappa") ||
      cuerr(cudaMemset(g->d_macro, 0, 4 * (size_t)MF * nf), "macro") ||
      cuerr(cudaMemset(g->d_buf[0], 0, fsz * Q * g->ncell_total), "buf0") ||
      cuerr(cudaMemset(g->d_buf[1], 0, fsz * Q * g->ncell_total), "buf1")) {
    lsb_destroy(g);
    return LSB_ECUDA;
  }
  for (int k = 0; k < 3; ++k)
    if (cuerr(cudaMemset(g->d_ut[k], 0, 4 * D * nf), "ut")) { lsb_destroy(g); return LSB_ECUDA; }
  // phi: dense caller array -> padded finest array
  for (int c = 0; c < n_cases; ++c) {
    const LevelDev &F = g->lds[g->cases[c].ld0 + g->cases[c].L - 1];
    if (cuerr(cudaMemset(g->d_phi + F.fine_off, 0, 4 * F.ncell), "phi")) { lsb_destroy(g); return LSB_ECUDA; }
    cudaMemcpy3DParms pr;
    memset(&pr, 0, sizeof pr);
    pr.srcPtr = make_cudaPitchedPtr((void *)phi0[c], sizeof(float) * F.n[0], F.n[0], F.n[1]);
    pr.dstPtr = make_cudaPitchedPtr(g->d_phi + F.fine_off, sizeof(float) * F.p[0], F.p[0], F.p[1]);
    pr.extent = make_cudaExtent(sizeof(float) * F.n[0], F.n[1], F.n[2]);
    pr.kind = cudaMemcpyDeviceToDevice;
    if (cuerr(cudaMemcpy3D(&pr), "phi0 copy")) { lsb_destroy(g); return LSB_ECUDA; }
  }
  s = build_tensor_maps(g);
  if (s == LSB_OK) s = ls_mirror(g);
  if (s == LSB_OK) s = regrid(g, true);
  if (s) { g_create_error = g->err; lsb_destroy(g); return s; }
  *out = g;
  return LSB_OK;
}

lsb_status lsb_set_params(lsb_grid *g, int case_idx, const lsb_params *params) {
  if (!g || !params) return LSB_EINVAL;
  if (case_idx < -1 || case_idx >= g->ncase) return fail(g, LSB_EINVAL, "case_idx out of range");
  for (int c = 0; c < g->ncase; ++c) {
    if (case_idx != -1 && c != case_idx) continue;
    std::string why;
    if (check_params(*params, g->cases[c].d, why)) return fail(g, LSB_EINVAL, "%s", why.c_str());
  }
  if (params->n_ext != g->n_ext || params->reinit_every != g->reinit_every || params->n_reinit != g->n_reinit)
    if (g->ncase > 1 && case_idx != -1) return fail(g, LSB_EINVAL, "level-set iteration counts are shared by all cases");
  if (g->rec_on) rec_clear(g);  // a recording covers one parameter set
  // captured graphs hold the launch sequence, which these decide on the host
  bool relaunch = params->n_ext != g->n_ext || params->reinit_every != g->reinit_every ||
                  params->n_reinit != g->n_reinit || params->regrid_every != g->regrid_every;
  for (int c = 0; c < g->ncase; ++c) {
    if (case_idx != -1 && c != case_idx) continue;
    relaunch = relaunch || params->ls_active != g->cases[c].p.ls_active;
    g->cases[c].p = *params;
    for (int l = 0; l < g->cases[c].L; ++l) fill_physics(g, g->lds[g->cases[c].ld0 + l], g->cases[c]);
  }
  g->n_ext = params->n_ext;
  g->reinit_every = params->reinit_every;
  g->n_reinit = params->n_reinit;
  g->regrid_every = params->regrid_every;
  if (relaunch) drop_graphs(g);
  // stream-ordered before the next step; a copy from pageable memory returns once the
  // source is staged, so the host descriptors may change again right away
  CU(cudaMemcpyAsync(g->d_lds, g->lds.data(), sizeof(LevelDev) * g->lds.size(), cudaMemcpyHostToDevice, g->stream));
  return LSB_OK;
}

lsb_status lsb_step(lsb_grid *g, int n) {
  if (!g || n < 0) return LSB_EINVAL;
  if (g->ls_dirty && g->driver == 0) TRY(ls_mirror(g));
  if (g->rec_on) {  // recorded steps run eagerly, checkpointing every rec_every steps
    for (int k = 0; k < n; ++k) {
      if (g->rec_steps % g->rec_every == 0 && (size_t)(g->rec_steps / g->rec_every) == g->rec_ckpt.size())
        TRY(rec_checkpoint(g));
      TRY(advance(g, 0));
      if (g->rec_moving)
        TRY(launched(g, run_lsa_flipflag(LN(g, 1, 32), g->d_counters, g->Lmax - 1, g->d_recflip)));
      g->updates_done += updates_per_step(g);
      g->coarse_steps++;
      g->rec_steps++;
      g->adj_cur = -1;
    }
    return LSB_OK;
  }
  int k = 0;
  while (k < n) {
    const bool regrid_on = g->regrid_every > 0 && g->Lmax > 1;
    const bool regrid_soon =
        regrid_on && ((g->coarse_steps + 1) % g->regrid_every == 0 || (g->coarse_steps + 2) % g->regrid_every == 0);
    if (n - k >= 2 && !regrid_soon && graphs_usable(g)) {
      TRY(replay_steps(g, 2));
      k += 2;
      continue;
    }
    if (graphs_usable(g)) {  // one step (a regrid, if due, follows it as after an eager step)
      TRY(replay_steps(g, 1));
    } else {
      TRY(advance(g, 0));
      g->updates_done += updates_per_step(g);
      g->coarse_steps++;
    }
    ++k;
    if (regrid_on && g->coarse_steps % g->regrid_every == 0) TRY(regrid(g, false));
  }
  return LSB_OK;
}

lsb_status lsb_use_graphs(lsb_grid *g, int enable) {
  if (!g || (enable != 0 && enable != 1)) return LSB_EINVAL;
  if (enable && !g->stream) return fail(g, LSB_EINVAL, "CUDA graphs need a non-default stream");
  g->use_graphs = enable;
  if (!enable) drop_graphs(g);
  return LSB_OK;
}

lsb_status lsb_set_objective(lsb_grid *g, double eps) {
  if (!g || !(eps >= 0.0) || !std::isfinite(eps)) return LSB_EINVAL;
  if (g->rec_on) rec_clear(g);  // a recording covers one objective
  g->obj_eps = (float)eps;
  return LSB_OK;
}

lsb_status lsb_set_wait_limit(lsb_grid *g, long long spins) {
  if (!g || spins < 0) return LSB_EINVAL;
  if (spins != g->wait_limit) drop_graphs(g);  // the limit is a captured kernel argument
  g->wait_limit = spins;
  return LSB_OK;
}

lsb_status lsb_set_driver(lsb_grid *g, int mode) {
  if (!g || (mode != 0 && mode != 1)) return LSB_EINVAL;
  if (mode == 1) {
    int dev = 0, coop = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    if (!coop) return fail(g, LSB_EINVAL, "the device does not support cooperative launches");
  }
  if (mode != g->driver) drop_graphs(g);  // captured launch sequences change
  g->driver = mode;
  return LSB_OK;
}

lsb_status lsb_refine(lsb_grid *g) {
  if (!g) return LSB_EINVAL;
  if (g->rec_on) rec_clear(g);
  return regrid(g, false);
}

lsb_status lsb_sync(lsb_grid *g) {
  if (!g) return LSB_EINVAL;
  TRY(pin_host(g));
  // the error word comes back with the stream's work: one wait for both
  CU(cudaMemcpyAsync(g->h_err, g->d_err, sizeof(int), cudaMemcpyDeviceToHost, g->stream));
  CU(cudaStreamSynchronize(g->stream));
  const int e = *g->h_err;
  g->latched |= e;
  if (g->latched & (ERR_LINK_OVF | ERR_LIST_OVF | ERR_BAND_OVF))
    return fail(g, LSB_ENOMEM, "device work list overflow (flags %d)", g->latched);
  if (g->latched & ERR_TIMEOUT) return fail(g, LSB_ETIMEOUT, "a bounded device-side wait gave up");
  if (g->latched & ERR_NONFINITE) return fail(g, LSB_EUNSTABLE, "non-finite density or velocity");
  return LSB_OK;
}

size_t lsb_field_bytes(const lsb_grid *g, int case_idx, int field, int level) {
  if (!g || case_idx < 0 || case_idx >= g->ncase) return 0;
  const CaseHost &ch = g->cases[case_idx];
  if (level < 0 || level >= ch.L) return 0;
  const LevelDev &L = g->lds[ch.ld0 + level];
  const size_t n = (size_t)L.n[0] * L.n[1] * L.n[2];
  const bool fine_only = field == LSB_FIELD_PHI || field == LSB_FIELD_CUTMASK || field == LSB_FIELD_KAPPA ||
                         field == LSB_FIELD_UEXT;
  if (fine_only && !L.finest) return 0;
  switch (field) {
    case LSB_FIELD_RHO: case LSB_FIELD_PHI: case LSB_FIELD_KAPPA: return 4 * n;
    case LSB_FIELD_U: case LSB_FIELD_UEXT: return 4 * n * g->D;
    case LSB_FIELD_PHASE: case LSB_FIELD_TAG: return n;
    case LSB_FIELD_F: case LSB_FIELD_ADJ_F: return 4 * n * g->Q;
    case LSB_FIELD_ADJ_UEXT: return L.finest ? 4 * n * g->D : 0;
    case LSB_FIELD_BLOCKS: return (size_t)L.nblock;
    case LSB_FIELD_CUTMASK: return 4 * n;
    default: return 0;
  }
}

lsb_status lsb_get_fields(lsb_grid *g, int case_idx, int field, int level, void *dst, size_t dst_bytes,
                          int dst_on_host) {
  if (!g || !dst) return LSB_EINVAL;
  const size_t need = lsb_field_bytes(g, case_idx, field, level);
  if (need == 0) return fail(g, LSB_EINVAL, "invalid case/field/level");
  if (dst_bytes < need) return fail(g, LSB_EINVAL, "dst too small: %zu < %zu", dst_bytes, need);
  const CaseHost &ch = g->cases[case_idx];
  const int ld = ch.ld0 + level;
  const LevelDev &L = g->lds[ld];
  const size_t n = (size_t)L.n[0] * L.n[1] * L.n[2];
  const cudaMemcpyKind kind = dst_on_host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  if (field == LSB_FIELD_BLOCKS) {
    if (dst_on_host) memcpy(dst, g->status[ld].data(), L.nblock);
    else CU(cudaMemcpy(dst, g->status[ld].data(), L.nblock, cudaMemcpyHostToDevice));
    return lsb_sync(g);
  }
  if (field == LSB_FIELD_RHO || field == LSB_FIELD_U || field == LSB_FIELD_F) {
    float *tmp = nullptr;
    CU(cudaMalloc(&tmp, need));
    Ctx C = make_ctx(g);
    const int fcode = field == LSB_FIELD_RHO ? 0 : (field == LSB_FIELD_U ? 1 : 4);
    lsb_status s = LSB_OK;
    s = launched(g, run_export(g->Q, g->storage, LN(g, 1024, 256), C, ld, fcode, tmp));
    if (s == LSB_OK) {
      cudaError_t e = cudaMemcpyAsync(dst, tmp, need, kind, g->stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
      if (e != cudaSuccess) s = fail(g, LSB_ECUDA, "export copy: %s", cudaGetErrorString(e));
    }
    cudaFree(tmp);
    if (s) return s;
    return lsb_sync(g);
  }
  // plain per-cell arrays: strided 3-D copies from the padded layout
  const void *src = nullptr;
  size_t esz = 4;
  int planes = 1;
  long long plane_stride = 0;
  switch (field) {
    case LSB_FIELD_PHI: src = g->d_phi + L.fine_off; break;
    case LSB_FIELD_KAPPA: src = g->d_kappa + L.fine_off; break;
    case LSB_FIELD_CUTMASK: src = g->d_cmask + L.fine_off; break;
    case LSB_FIELD_UEXT: src = g->d_ut[0] + L.fine_off; planes = g->D; plane_stride = g->nfine; break;
    case LSB_FIELD_ADJ_UEXT:
      if (g->adj_cur < 0 || !g->rec_moving)
        return fail(g, LSB_ESTATE, "no u~ adjoint: lsb_backward over a moving level set first");
      src = lsa_ptrs(g).LU[g->adj_cur] + L.fine_off;
      planes = g->D;
      plane_stride = g->nfine;
      break;
    case LSB_FIELD_ADJ_F:
      if (g->adj_cur < 0) return fail(g, LSB_ESTATE, "no adjoint field: call lsb_backward first");
      src = g->d_adj[g->apar[L.level]] + L.cell_off * g->Q;
      planes = g->Q;
      plane_stride = L.ncell;
      break;
    case LSB_FIELD_PHASE: case LSB_FIELD_TAG: src = g->d_tag + L.cell_off; esz = 1; break;
    default: return fail(g, LSB_EINVAL, "field");
  }
  CU(cudaStreamSynchronize(g->stream));
  for (int pl = 0; pl < planes; ++pl) {
    cudaMemcpy3DParms pr;
    memset(&pr, 0, sizeof pr);
    const char *sp = (const char *)src + esz * plane_stride * pl;
    pr.srcPtr = make_cudaPitchedPtr((void *)sp, esz * L.p[0], L.p[0], L.p[1]);
    pr.dstPtr = make_cudaPitchedPtr((char *)dst + esz * n * pl, esz * L.n[0], L.n[0], L.n[1]);
    pr.extent = make_cudaExtent(esz * L.n[0], L.n[1], L.n[2]);
    pr.kind = kind;
    CU(cudaMemcpy3D(&pr));
  }
  if (field == LSB_FIELD_PHASE) {
    if (dst_on_host) {
      uint8_t *p = (uint8_t *)dst;
      for (size_t i = 0; i < n; ++i) p[i] &= TAG_GAS;
    } else {
      std::vector<uint8_t> h(n);
      CU(cudaMemcpy(h.data(), dst, n, cudaMemcpyDeviceToHost));
      for (size_t i = 0; i < n; ++i) h[i] &= TAG_GAS;
      CU(cudaMemcpy(dst, h.data(), n, cudaMemcpyHostToDevice));
    }
  }
  return lsb_sync(g);
}

// The observables of every case into d_obs (zeroed by the caller): the TMA-staged pass
// when the population maps are the plain ones, else per-thread loads.
lsb_status observables_pass(lsb_grid *g, const Ctx &C, const BlockShape &S, int stride) {
  const bool tma = g->obs_tma_grid > 0 && g->d_tmaps && !g->no_tma && !g->tma_a;
  const CUtensorMap *tm = tma ? (const CUtensorMap *)g->d_tmaps : nullptr;
  const CUtensorMap *tt = tma && g->tma_tags ? tm + 2 * g->lds.size() : nullptr;
  // the resident CTAs of the kernel that runs
  const int og = std::min(g->leaf.n, tma ? g->obs_tma_grid : 152 * LSB_OBS_MINB);
  RUN(6, 0, g->leaf.n, g->nthreads, run_observables, g->Q, g->storage, LN(g, og, g->nthreads), C, S,
      (const int *)g->leaf.d, g->leaf.n, g->d_obs, stride, g->obj_eps, tm, tt);
  return LSB_OK;
}

lsb_status lsb_observables(lsb_grid *g, double *out_host, size_t n_doubles) {
  if (!g || !out_host) return LSB_EINVAL;
  const int stride = 4 + 2 * g->D;
  if (n_doubles < (size_t)stride * g->ncase) return fail(g, LSB_EINVAL, "need %d doubles", stride * g->ncase);
  CU(cudaMemsetAsync(g->d_obs, 0, sizeof(double) * stride * g->ncase, g->stream));
  Ctx C = make_ctx(g);
  BlockShape S = shape(g);
  TRY(observables_pass(g, C, S, stride));
  TRY(pin_host(g));
  CU(cudaMemcpyAsync(g->h_obs, g->d_obs, sizeof(double) * stride * g->ncase, cudaMemcpyDeviceToHost, g->stream));
  lsb_status s = lsb_sync(g);
  for (int c = 0; c < g->ncase; ++c) {
    double *o = out_host + (size_t)stride * c;
    const double *v = g->h_obs + (size_t)stride * c;
    o[0] = v[0];
    o[1] = v[1];
    o[2] = v[2];
    o[3] = v[3];
    for (int a = 0; a < g->D; ++a) {
      o[4 + a] = v[2] > 0 ? v[4 + a] / v[2] : NAN;
      o[4 + g->D + a] = v[2] > 0 ? v[4 + g->D + a] / v[2] : NAN;
    }
  }
  return s;
}

lsb_status lsb_autotune(int n_cases, const lsb_grid_desc *descs, const lsb_params *params,
                        const float *const *phi0, void *stream, const int *candidates, int n_cand, int steps,
                        int *best, double *ms_per_step) {
  if (n_cases < 1 || !descs || !params || !phi0 || !best || steps < 1)
    return fail(nullptr, LSB_EINVAL, "autotune: need cases, phi0, best and steps >= 1");
  if (candidates && n_cand < 1) return fail(nullptr, LSB_EINVAL, "autotune: n_cand must be >= 1");
  const bool d2 = descs[0].lattice == LSB_D2Q9;
  // default shapes: one warp per x row (or two), thin in the other axes
  static const int def2[][3] = {{32, 8, 1}, {32, 16, 1}, {64, 8, 1}, {16, 16, 1}, {64, 4, 1}, {128, 4, 1}};
  static const int def3[][3] = {{32, 4, 4}, {32, 8, 2}, {16, 8, 4}, {64, 4, 2}, {32, 2, 8}, {16, 4, 8}};
  const int *cand = candidates ? candidates : (d2 ? &def2[0][0] : &def3[0][0]);
  const int nc = candidates ? n_cand : 6;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    return fail(nullptr, LSB_ECUDA, "autotune: event creation failed");
  double best_ms = INFINITY;
  std::vector<lsb_grid_desc> dd(descs, descs + n_cases);
  std::string last_err;
  for (int k = 0; k < nc; ++k) {
    for (int c = 0; c < n_cases; ++c)
      for (int a = 0; a < 3; ++a) dd[c].block[a] = cand[3 * k + a];
    double ms = NAN;
    lsb_grid *g = nullptr;
    if (lsb_create_grid(n_cases, dd.data(), params, phi0, stream, &g) == LSB_OK) {
      // two untimed steps, then `steps` steps bracketed by events on the handle's stream
      lsb_status s = lsb_step(g, 2);
      if (s == LSB_OK && cudaEventRecord(e0, st) == cudaSuccess && (s = lsb_step(g, steps)) == LSB_OK &&
          cudaEventRecord(e1, st) == cudaSuccess && (s = lsb_sync(g)) == LSB_OK) {
        float t = 0.f;
        if (cudaEventElapsedTime(&t, e0, e1) == cudaSuccess) ms = t / steps;
      }
      if (s != LSB_OK) last_err = g->err;
      lsb_destroy(g);
    } else {
      last_err = g_create_error;
    }
    if (ms_per_step) ms_per_step[k] = ms;
    if (ms == ms && ms < best_ms) {
      best_ms = ms;
      for (int a = 0; a < 3; ++a) best[a] = cand[3 * k + a];
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (!(best_ms < INFINITY)) return fail(nullptr, LSB_EINVAL, "autotune: no candidate ran (%s)", last_err.c_str());
  return LSB_OK;
}

lsb_status lsb_cell_updates(const lsb_grid *g, double *per_coarse_step, double *total_done) {
  if (!g) return LSB_EINVAL;
  if (per_coarse_step) *per_coarse_step = updates_per_step(g);
  if (total_done) *total_done = g->updates_done;
  return LSB_OK;
}

lsb_status lsb_work_counts(lsb_grid *g, int level, long long *out, int n) {
  if (!g || !out || n < 0 || level < 0 || level >= MAXL) return LSB_EINVAL;
  long long v[LSB_NWORK] = {0};
  v[0] = (long long)g->leaf_cells[level];
  v[5] = g->ghost_cells[level].n;
  v[6] = g->rl_cells[level].n;
  if (has_finest(g, level)) {
    int h[NCOUNT] = {0};
    CU(cudaMemcpyAsync(h, g->d_counters + level * NCOUNT, sizeof(int) * NCOUNT, cudaMemcpyDeviceToHost, g->stream));
    CU(cudaStreamSynchronize(g->stream));
    v[1] = (long long)std::min(h[3], g->band_cap) * g->nthreads;
    v[2] = std::min<long long>(h[1], g->list_cap);
    v[3] = std::min<long long>(h[0], g->link_cap);
    v[4] = std::min<long long>(h[2], g->list_cap);
  }
  for (int k = 0; k < n && k < LSB_NWORK; ++k) out[k] = v[k];
  return LSB_OK;
}

lsb_status lsb_profile(lsb_grid *g, int mode) {
  if (!g || mode < 0 || mode > 2) return LSB_EINVAL;
  CU(cudaStreamSynchronize(g->stream));
  for (ProfRec &r : g->prof) {
    g->ev_pool.push_back(r.a);
    g->ev_pool.push_back(r.b);
  }
  g->prof.clear();
  g->prof_mode = mode;
  return LSB_OK;
}

lsb_status lsb_profile_read(lsb_grid *g, double *ms, double *bytes, uint64_t *launches, int n) {
  if (!g || n < 0) return LSB_EINVAL;
  CU(cudaStreamSynchronize(g->stream));
  for (int k = 0; k < n; ++k) {
    if (ms) ms[k] = 0;
    if (bytes) bytes[k] = 0;
    if (launches) launches[k] = 0;
  }
  for (ProfRec &r : g->prof) {
    float t = 0.f;
    CU(cudaEventElapsedTime(&t, r.a, r.b));
    if (r.kid < n) {
      if (ms) ms[r.kid] += t;
      if (bytes) bytes[r.kid] += r.bytes;
      if (launches) launches[r.kid] += 1;
    }
    g->ev_pool.push_back(r.a);
    g->ev_pool.push_back(r.b);
  }
  g->prof.clear();
  return LSB_OK;
}

const char *lsb_kernel_name(int k) { return (k >= 0 && k < NKERN) ? KNAMES[k] : nullptr; }

int lsb_kernel_count(void) { return NKERN; }

lsb_status lsb_record(lsb_grid *g, int checkpoint_every) {
  if (!g || checkpoint_every < 1) return LSB_EINVAL;
  if (g->storage != LSB_FP32) return fail(g, LSB_ESTATE, "the adjoint needs FP32 population storage");
  if (g->Q == 27) return fail(g, LSB_ESTATE, "the adjoint covers D2Q9 and D3Q19 with BGK collision");
  int live = 0;
  for (const CaseHost &c : g->cases) live += c.p.ls_active ? 1 : 0;
  if (live != 0 && live != g->ncase)
    return fail(g, LSB_ESTATE, "the adjoint needs the level set live in every case or frozen in every case");
  if (g->Lmax > 1) {
    for (const CaseHost &c : g->cases)
      if (c.L != g->Lmax) return fail(g, LSB_ESTATE, "a multi-level recording needs the same levels in every case");
  }
  if (live && (g->reinit_every > 1 || g->n_reinit > 1))
    return fail(g, LSB_ESTATE, "the moving-interface adjoint needs reinit_every <= 1 and n_reinit <= 1");
  CU(cudaStreamSynchronize(g->stream));
  rec_clear(g);
  if (!g->d_recflip) TRY(dalloc(g, &g->d_recflip, sizeof(int)));
  CU(cudaMemset(g->d_recflip, 0, sizeof(int)));
  g->rec_on = 1;
  g->rec_moving = live ? 1 : 0;
  g->rec_every = checkpoint_every;
  return LSB_OK;
}

lsb_status lsb_backward(lsb_grid *g, const double *dJ_dobs, double *dJ_dparams, float *dJ_dphi0) {
  if (!g || !dJ_dobs) return LSB_EINVAL;
  if (!g->rec_on) return fail(g, LSB_ESTATE, "no recording: call lsb_record before the steps to differentiate");
  const int Q = g->Q, D = g->D, stride = 4 + 2 * D;
  const long long T = g->rec_steps;
  const int every = g->rec_every;
  const bool mv = g->rec_moving != 0;
  if (mv) {
    int flip = 0;
    CU(cudaStreamSynchronize(g->stream));
    CU(cudaMemcpy(&flip, g->d_recflip, sizeof(int), cudaMemcpyDeviceToHost));
    if (flip) return fail(g, LSB_ESTATE, "a cell changed phase during the recorded window");
  }
  TRY(adj_buffers(g, (int)std::min<long long>(every, std::max<long long>(T, 1))));
  const size_t sf = state_floats(g), sb = sizeof(float) * sf, sl = slot_floats(g);
  const size_t NF = g->nfine;
  const int MF = 1 + D + D * (D + 1) / 2;
  CU(cudaMemsetAsync(g->d_adj[0], 0, sb, g->stream));
  CU(cudaMemsetAsync(g->d_adj[1], 0, sb, g->stream));
  CU(cudaMemsetAsync(g->d_madj, 0, sizeof(float) * (size_t)MF * g->nfine, g->stream));
  CU(cudaMemsetAsync(g->d_grad, 0, sizeof(double) * NG_ADJ * g->ncase, g->stream));
  GeoAdj G{nullptr, nullptr, nullptr};
  if (dJ_dphi0) {
    G = GeoAdj{g->d_gphi, g->d_gn, g->d_gk};
    CU(cudaMemsetAsync(g->d_gphi, 0, sizeof(float) * (size_t)g->nfine, g->stream));
    CU(cudaMemsetAsync(g->d_gn, 0, sizeof(float) * (size_t)D * g->nfine, g->stream));
    CU(cudaMemsetAsync(g->d_gk, 0, sizeof(float) * (size_t)g->nfine, g->stream));
  }
  CU(cudaMemcpyAsync(g->d_wobs, dJ_dobs, sizeof(double) * stride * g->ncase, cudaMemcpyHostToDevice, g->stream));
  // the final state; restored when the sweep is done
  const int par0 = g->par[0];
  const bool amr = g->Lmax > 1;
  int par_all[MAXL];
  long long fs_all[MAXL];
  for (int l = 0; l < MAXL; ++l) {
    par_all[l] = g->par[l];
    fs_all[l] = g->fine_steps[l];
  }
  void *const bufs[2] = {g->d_buf[0], g->d_buf[1]};
  const long long fs0 = g->fine_steps[0], cs0 = g->coarse_steps;
  const double ud0 = g->updates_done;
  if (amr) TRY(snapshot(g, g->d_fsave));
  else CU(cudaMemcpyAsync(g->d_fsave, g->d_buf[par0], sb, cudaMemcpyDeviceToDevice, g->stream));
  if (mv) {
    CU(cudaMemsetAsync(g->d_gn, 0, sizeof(float) * D * NF, g->stream));
    CU(cudaMemsetAsync(g->d_gk, 0, sizeof(float) * NF, g->stream));
    CU(cudaMemcpyAsync(g->d_phisave, g->d_phi, sizeof(float) * NF, cudaMemcpyDeviceToDevice, g->stream));
    CU(cudaMemcpyAsync(g->d_utsave, g->d_ut[0], sizeof(float) * D * NF, cudaMemcpyDeviceToDevice, g->stream));
  }
  Ctx C = make_ctx(g);
  BlockShape S = shape(g);
  CU(cudaMemsetAsync(g->d_obs, 0, sizeof(double) * stride * g->ncase, g->stream));
  TRY(observables_pass(g, C, S, stride));
  // the objective's direct dependence on phi (smoothed indicator): into the level set's
  // adjoint at the end of the window (moving), or into dJ/dphi (frozen)
  float *lphi = g->obj_eps > 0.f ? (mv ? lsa_ptrs(g).LP[0] : (dJ_dphi0 ? g->d_gphi : nullptr)) : nullptr;
  RUN(KADJ_SEED, 0, g->leaf.n, g->nthreads, run_adj_seed, Q, LN(g, std::min(g->leaf.n, 152 * 8), g->nthreads), C,
      S, (const int *)g->leaf.d, g->leaf.n, (const float *)g->d_fsave, g->d_adj[0], g->d_wobs, g->d_obs, stride,
      g->obj_eps, lphi);
  int cur = 0;
  lsb_status st = LSB_OK;
  const long long nseg = amr ? 0 : (T + every - 1) / every;
  if (amr) st = backward_amr(g, G);
  for (long long sgi = nseg - 1; sgi >= 0 && st == LSB_OK; --sgi) {
    const long long start = sgi * every;
    const int len = (int)std::min<long long>(every, T - start);
    // recompute the segment from its checkpoint: step j reads slot j and pushes into
    // slot j + 1 (the last step's result is not needed and goes to a grid buffer)
    float *ck = g->rec_ckpt[sgi];
    cudaError_t e = cudaMemcpyAsync(g->d_seg, ck, sb, cudaMemcpyDeviceToDevice, g->stream);
    if (e == cudaSuccess && mv) {
      e = cudaMemcpyAsync(g->d_phi, ck + sf, sizeof(float) * NF, cudaMemcpyDeviceToDevice, g->stream);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(g->d_ut[0], ck + sf + NF, sizeof(float) * D * NF, cudaMemcpyDeviceToDevice, g->stream);
    }
    if (e != cudaSuccess) { st = fail(g, LSB_ECUDA, "checkpoint restore: %s", cudaGetErrorString(e)); break; }
    if (mv && (st = ls_mirror(g)) != LSB_OK) break;
    // the interface geometry (n, kappa) the first step uses is that of the restored phi
    if (mv && (st = classify(g, 0, 0)) != LSB_OK) break;
    // the grid's tensor maps describe its own buffers: the slots have maps of their own,
    // else the plain collide kernel runs
    if (!g->d_seg_tmaps) g->no_tma = 1;
    for (int j = 0; j < len && st == LSB_OK; ++j) {
      float *slot = g->d_seg + sl * j;
      if (g->d_seg_tmaps) g->tma_a = g->d_seg_tmaps + (size_t)j * 2 * g->lds.size();
      if (mv) {
        e = cudaMemcpyAsync(slot + sf, g->d_phi, sizeof(float) * NF, cudaMemcpyDeviceToDevice, g->stream);
        if (e == cudaSuccess)
          e = cudaMemcpyAsync(slot + sf + NF, g->d_ut[0], sizeof(float) * D * NF, cudaMemcpyDeviceToDevice, g->stream);
        if (e != cudaSuccess) { st = fail(g, LSB_ECUDA, "segment store: %s", cudaGetErrorString(e)); break; }
      }
      g->d_buf[g->par[0]] = slot;
      g->d_buf[1 - g->par[0]] = j + 1 < len ? (void *)(g->d_seg + sl * (j + 1)) : bufs[0];
      st = advance(g, 0);
    }
    g->no_tma = 0;
    g->tma_a = nullptr;
    g->d_buf[0] = bufs[0];
    g->d_buf[1] = bufs[1];
    for (int j = len - 1; j >= 0 && st == LSB_OK; --j) {
      float *slot = g->d_seg + sl * j;
      st = mv ? adj_moving(g, 0, slot, slot + sf, slot + sf + NF, g->d_adj[cur], g->d_adj[1 - cur], cur)
              : adj_step(g, slot, cur, G);
      cur ^= 1;
    }
  }
  g->par[0] = par0;
  g->fine_steps[0] = fs0;
  g->coarse_steps = cs0;
  g->updates_done = ud0;
  if (amr) {
    for (int l = 0; l < MAXL; ++l) {
      g->par[l] = par_all[l];
      g->fine_steps[l] = fs_all[l];
    }
    TRY(restore(g, g->d_fsave));
  } else {
    CU(cudaMemcpyAsync(g->d_buf[par0], g->d_fsave, sb, cudaMemcpyDeviceToDevice, g->stream));
  }
  if (mv) {
    CU(cudaMemcpyAsync(g->d_phi, g->d_phisave, sizeof(float) * NF, cudaMemcpyDeviceToDevice, g->stream));
    CU(cudaMemcpyAsync(g->d_ut[0], g->d_utsave, sizeof(float) * D * NF, cudaMemcpyDeviceToDevice, g->stream));
    TRY(ls_mirror(g));
    if (st == LSB_OK) st = classify(g, g->Lmax - 1, 0);  // geometry and lists of the restored phi
  }
  if (st != LSB_OK) return st;
  if (dJ_dphi0) {
    const float *src = g->d_gphi;
    if (mv) {
      src = lsa_ptrs(g).LP[amr ? g->lspar : cur];  // the adjoint of phi_0 through every pass
    } else {
      // normal and curvature adjoints through the least-squares fit, then the dense boxes
      Ctx C2 = make_ctx(g);
      RUN(KADJ_GEOM, 0, 1, 128, run_adj_geometry, D, LN(g, DYN_GRID, 128), C2, g->Lmax - 1, G);
    }
    size_t off = 0;
    for (int c = 0; c < g->ncase; ++c) {
      const LevelDev &L = g->lds[g->cases[c].ld0 + g->cases[c].L - 1];
      cudaMemcpy3DParms pr;
      memset(&pr, 0, sizeof pr);
      pr.srcPtr = make_cudaPitchedPtr((void *)(src + L.fine_off), 4 * (size_t)L.p[0], L.p[0], L.p[1]);
      pr.dstPtr = make_cudaPitchedPtr((void *)(dJ_dphi0 + off), 4 * (size_t)L.n[0], L.n[0], L.n[1]);
      pr.extent = make_cudaExtent(4 * (size_t)L.n[0], L.n[1], L.n[2]);
      pr.kind = cudaMemcpyDeviceToDevice;
      CU(cudaMemcpy3DAsync(&pr, g->stream));
      off += (size_t)L.n[0] * L.n[1] * L.n[2];
    }
  }
  std::vector<double> h((size_t)NG_ADJ * g->ncase);
  CU(cudaMemcpyAsync(h.data(), g->d_grad, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, g->stream));
  TRY(lsb_sync(g));
  g->adj_cur = amr ? g->lspar : cur;  // with a moving level set on several levels: LU[lspar]
  if (!amr) g->apar[0] = cur;
  if (dJ_dparams) {
    for (int c = 0; c < g->ncase; ++c) {
      const lsb_params &p = g->cases[c].p;
      const double *gr = h.data() + (size_t)NG_ADJ * c;
      double *o = dJ_dparams + (size_t)LSB_NPARAM_ADJ * c;
      o[0] = gr[0];
      for (int ph = 0; ph < 2; ++ph) {
        double dacc = 0.0;
        for (int a = 0; a < D; ++a) dacc += gr[7 + 3 * ph + a] * (-p.body_force[a] / (p.rho[ph] * p.rho[ph]));
        o[1 + ph] = gr[1 + ph] + gr[3 + ph] * p.nu[ph] + dacc;
        o[3 + ph] = gr[3 + ph] * p.rho[ph] + gr[5 + ph];
      }
    }
  }
  return LSB_OK;
}

lsb_status lsb_get_fields_noalloc(lsb_grid *g, int case_idx, int field, int level, void *dst, size_t dst_bytes,
                                  int dst_on_host) {
  if (!g || !dst) return LSB_EINVAL;
  if (field != LSB_FIELD_RHO && field != LSB_FIELD_U && field != LSB_FIELD_F)
    return fail(g, LSB_EINVAL, "lsb_get_fields_noalloc exports LSB_FIELD_RHO, LSB_FIELD_U and LSB_FIELD_F only");
  const size_t need = lsb_field_bytes(g, case_idx, field, level);
  if (need == 0) return fail(g, LSB_EINVAL, "invalid case/field/level");
  if (dst_bytes < need) return fail(g, LSB_EINVAL, "dst too small: %zu < %zu", dst_bytes, need);
  if (need > kNoAllocFloats * sizeof(float))
    return fail(g, LSB_EINVAL, "field needs %zu bytes, more than the %zu-byte fixed staging array of "
                "lsb_get_fields_noalloc; use lsb_get_fields", need, kNoAllocFloats * sizeof(float));
  const int ld = g->cases[case_idx].ld0 + level;
  const int fcode = field == LSB_FIELD_RHO ? 0 : (field == LSB_FIELD_U ? 1 : 4);
  float *staged = nullptr;
  Ctx C = make_ctx(g);
  TRY(launched(g, run_export_noalloc(g->Q, g->storage, LN(g, 1024, 256), C, ld, fcode, &staged)));
  CU(cudaMemcpyAsync(dst, staged, need, dst_on_host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, g->stream));
  CU(cudaStreamSynchronize(g->stream));
  return lsb_sync(g);
}

uint64_t lsb_kernel_launches(const lsb_grid *g) { return g ? g->launches : 0; }

const char *lsb_last_error(const lsb_grid *g) { return g ? g->err.c_str() : g_create_error.c_str(); }

void lsb_destroy(lsb_grid *g) {
  if (!g) return;
  if (g->stream) cudaStreamSynchronize(g->stream);
  else cudaDeviceSynchronize();
  drop_graphs(g);
  for (int l = 0; l < MAXL; ++l) {
    if (g->side2[l]) {
      cudaStreamSynchronize(g->side2[l]);
      cudaStreamDestroy(g->side2[l]);
      cudaEventDestroy(g->ev_free[l]);
      cudaEventDestroy(g->ev_fill[l]);
      if (g->ev_ring0[l]) cudaEventDestroy(g->ev_ring0[l]);
      if (g->ev_ring0_done[l]) cudaEventDestroy(g->ev_ring0_done[l]);
    }
    if (g->side[l]) {
      cudaStreamSynchronize(g->side[l]);
      cudaStreamDestroy(g->side[l]);
      cudaEventDestroy(g->ev_fork[l]);
      cudaEventDestroy(g->ev_join[l]);
    }
  }
  for (void *p : g->allocs) cudaFree(p);
  if (g->d_lsa) cudaFree(g->d_lsa);
  if (g->d_seg) cudaFree(g->d_seg);
  for (float *p : g->rec_ckpt) cudaFree(p);
  for (float *p : g->tape_old) cudaFree(p);
  for (float *p : g->tape_new) cudaFree(p);
  for (float *p : g->tape_ls) cudaFree(p);
  for (ProfRec &r : g->prof) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  for (cudaEvent_t e : g->ev_pool) cudaEventDestroy(e);
  if (g->h_err) cudaFreeHost(g->h_err);
  delete g;
}

// Velocity-set tables compiled into the library, for host-side checks:
// c (Q x 3 ints), w (Q floats), opp (Q ints).  Returns Q, or 0 for an unknown lattice.
int lsb_lattice_table(int lattice, int *c, float *w, int *opp) {
  if (lattice == LSB_D2Q9) {
    for (int i = 0; i < 9; ++i) {
      if (c) { c[3 * i] = Lat<9>::cx(i); c[3 * i + 1] = Lat<9>::cy(i); c[3 * i + 2] = 0; }
      if (w) w[i] = Lat<9>::w(i);
      if (opp) opp[i] = Lat<9>::opp(i);
    }
    return 9;
  }
  if (lattice == LSB_D3Q19) {
    for (int i = 0; i < 19; ++i) {
      if (c) { c[3 * i] = Lat<19>::cx(i); c[3 * i + 1] = Lat<19>::cy(i); c[3 * i + 2] = Lat<19>::cz(i); }
      if (w) w[i] = Lat<19>::w(i);
      if (opp) opp[i] = Lat<19>::opp(i);
    }
    return 19;
  }
  if (lattice == LSB_D3Q27) {
    for (int i = 0; i < 27; ++i) {
      if (c) { c[3 * i] = Lat<27>::cx(i); c[3 * i + 1] = Lat<27>::cy(i); c[3 * i + 2] = Lat<27>::cz(i); }
      if (w) w[i] = Lat<27>::w(i);
      if (opp) opp[i] = Lat<27>::opp(i);
    }
    return 27;
  }
  return 0;
}

}  // extern "C"

// ------------------------------------------------------------------ regrid
namespace {

// Compact ghost-ring and restriction-layer cells of every level into cell lists.
lsb_status collect_cells(lsb_grid *g) {
  BlockShape S = shape(g);
  if (!g->d_count) TRY(dalloc(g, &g->d_count, sizeof(int)));
  for (int l = 0; l < g->Lmax; ++l) {
    for (int kind = 0; kind < 2; ++kind) {
      WorkList &bl = kind == 0 ? g->ghost[l] : g->rst[l];
      CellList &cl = kind == 0 ? g->ghost_cells[l] : g->rl_cells[l];
      const int bits = kind == 0 ? TAG_GHOST : TAG_RLAYER;
      cl.n = 0;
      if (bl.n == 0) continue;
      const int need = bl.n * g->nthreads;
      if (need > cl.cap) {
        TRY(dalloc(g, &cl.d, sizeof(int2) * (size_t)need));
        cl.cap = need;
      }
      CU(cudaMemsetAsync(g->d_count, 0, sizeof(int), g->stream));
      Ctx C = make_ctx(g);
      RUN(20, 0, bl.n, g->nthreads, run_collect, LN(g, bl.n, g->nthreads), C, S, (const int *)bl.d, bl.n, bits, cl.d,
          g->d_count, cl.cap);
      int n = 0;
      CU(cudaMemcpyAsync(&n, g->d_count, sizeof(int), cudaMemcpyDeviceToHost, g->stream));
      CU(cudaStreamSynchronize(g->stream));
      cl.n = std::min(n, cl.cap);
      // the atomics append in arbitrary order: sort so that neighbouring threads work on
      // neighbouring cells.  Restriction cells: by (level, cell).  Ghost cells: by (level,
      // coarse parent, position in the parent), so that the up to 2^D fine cells
      // interpolated from the same coarse cells sit in adjacent lanes.
      if (cl.n > 1) {
        std::vector<int2> h(cl.n);
        CU(cudaMemcpy(h.data(), cl.d, sizeof(int2) * cl.n, cudaMemcpyDeviceToHost));
        if (kind == 0) {
          auto key = [g](const int2 &a) {
            const LevelDev &L = g->lds[a.x];
            const unsigned long long c = (unsigned)a.y, p0 = L.p[0], p1 = L.p[1];
            const unsigned long long x = c % p0, y = (c / p0) % p1, z = c / (p0 * p1);
            const unsigned long long par = (x >> 1) + (p0 >> 1) * ((y >> 1) + (p1 >> 1) * (z >> 1));
            return ((unsigned long long)a.x << 56) | (par << 3) | ((z & 1) << 2) | ((y & 1) << 1) | (x & 1);
          };
          std::sort(h.begin(), h.end(), [&](const int2 &a, const int2 &b) { return key(a) < key(b); });
        } else {
          std::sort(h.begin(), h.end(),
                    [](const int2 &a, const int2 &b) { return a.x != b.x ? a.x < b.x : a.y < b.y; });
        }
        CU(cudaMemcpy(cl.d, h.data(), sizeof(int2) * cl.n, cudaMemcpyHostToDevice));
      }
    }
  }
  return LSB_OK;
}

lsb_status regrid(lsb_grid *g, bool initial) {
  BlockShape S = shape(g);
  const int nt = g->nthreads;
  // sensor over every block of every non-finest level
  g->sens.h.clear();
  for (const CaseHost &ch : g->cases)
    for (int l = 0; l < ch.L - 1; ++l) {
      const LevelDev &L = g->lds[ch.ld0 + l];
      for (int b = 0; b < L.nblock; ++b) g->sens.h.push_back(L.block_off + b);
    }
  std::vector<float> sv(g->sens.h.size());
  if (!g->sens.h.empty()) {
    TRY(upload_list(g, g->sens));
    Ctx C = make_ctx(g);
    // mode per case: launch once per mode present (cases with the other mode are overwritten below)
    for (int mode = 0; mode < 2; ++mode) {
      bool any = false;
      for (const CaseHost &ch : g->cases) any |= (ch.p.sensor == mode);
      if (!any) continue;
      RUN(18, 0, g->sens.n, 256, run_sensor, LN(g, g->sens.n, 256), C, S, (const int *)g->sens.d, g->sens.n, mode, g->d_sens);
      std::vector<float> tmp(g->sens.h.size());
      CU(cudaMemcpyAsync(tmp.data(), g->d_sens, sizeof(float) * tmp.size(), cudaMemcpyDeviceToHost, g->stream));
      CU(cudaStreamSynchronize(g->stream));
      size_t k = 0;
      for (const CaseHost &ch : g->cases)
        for (int l = 0; l < ch.L - 1; ++l) {
          const LevelDev &L = g->lds[ch.ld0 + l];
          for (int b = 0; b < L.nblock; ++b, ++k)
            if (ch.p.sensor == mode) sv[k] = tmp[k];
        }
    }
  }
  // wanted refinement and grading per case
  std::vector<std::vector<int8_t>> newst(g->lds.size());
  size_t k = 0;
  for (const CaseHost &ch : g->cases) {
    std::vector<std::vector<char>> want(ch.L);
    for (int l = 0; l < ch.L - 1; ++l) {
      const LevelDev &L = g->lds[ch.ld0 + l];
      want[l].assign(L.nblock, 0);
      const double dref = ch.p.refine_dist[l];
      for (int b = 0; b < L.nblock; ++b, ++k)
        want[l][b] = ch.p.sensor == LSB_SENSOR_SIGNED ? (sv[k] >= -dref) : (sv[k] <= dref);
    }
    std::vector<std::vector<int8_t>> st;
    grade_case(g, ch, want, st);
    for (int l = 0; l < ch.L; ++l) newst[ch.ld0 + l] = st[l];
  }
  if (initial) {
    g->status = newst;
    TRY(upload_status(g, g->status));
    TRY(build_lists(g));
    TRY(level_tags(g));
    Ctx C = make_ctx(g);
    RUN(19, 0, g->all_active.n, nt, run_init, g->Q, g->storage, LN(g, g->all_active.n, nt), C, S,
        (const int *)g->all_active.d, g->all_active.n);
  } else {
    std::vector<std::vector<int8_t>> old = g->status;
    bool changed = false;
    for (size_t ld = 0; ld < old.size(); ++ld) changed |= (old[ld] != newst[ld]);
    if (!changed) return LSB_OK;
    // coarsening, finest to coarsest: parents of deactivated blocks take the children's mean
    for (int l = g->Lmax - 2; l >= 0; --l) {
      WorkList wl;
      for (const CaseHost &ch : g->cases) {
        if (l >= ch.L - 1) continue;
        const int ld = ch.ld0 + l;
        for (int b = 0; b < g->lds[ld].nblock; ++b)
          if (old[ld][b] == BLK_REFINED && newst[ld][b] != BLK_REFINED) wl.h.push_back(g->lds[ld].block_off + b);
      }
      if (wl.h.empty()) continue;
      TRY(upload_list(g, wl));
      Ctx C = make_ctx(g);
      RUN(2, 0, wl.n, nt, run_restrict, g->Q, g->storage, LN(g, wl.n, nt), C, S, (const int *)wl.d, wl.n, 1);
      CU(cudaStreamSynchronize(g->stream));
      cudaFree(wl.d);
      g->allocs.erase(std::remove(g->allocs.begin(), g->allocs.end(), (void *)wl.d), g->allocs.end());
    }
    // refinement, coarsest to finest: new fine blocks from the coarse data
    std::vector<std::vector<int8_t>> merged = newst;
    for (size_t ld = 0; ld < merged.size(); ++ld)
      for (size_t b = 0; b < merged[ld].size(); ++b)
        if (old[ld][b] == BLK_LEAF || newst[ld][b] == BLK_LEAF) merged[ld][b] = BLK_LEAF;
    TRY(upload_status(g, merged));
    g->status = merged;
    TRY(build_lists(g));
    TRY(level_tags(g));
    for (int l = 0; l < g->Lmax - 1; ++l) {
      WorkList wl;
      for (const CaseHost &ch : g->cases) {
        if (l >= ch.L - 1) continue;
        const LevelDev &Lc = g->lds[ch.ld0 + l];
        const LevelDev &Lf = g->lds[ch.ld0 + l + 1];
        for (int b = 0; b < Lf.nblock; ++b) {
          int pb = parent_block(Lc, Lf, b);
          if (newst[ch.ld0 + l][pb] == BLK_REFINED && old[ch.ld0 + l][pb] != BLK_REFINED)
            wl.h.push_back(Lf.block_off + b);
        }
      }
      if (wl.h.empty()) continue;
      TRY(upload_list(g, wl));
      Ctx C = make_ctx(g);
      RUN(4, 0, wl.n, nt, run_prolong, g->Q, g->storage, LN(g, wl.n, nt), C, S, (const int *)wl.d, wl.n);
      CU(cudaStreamSynchronize(g->stream));
      cudaFree(wl.d);
      g->allocs.erase(std::remove(g->allocs.begin(), g->allocs.end(), (void *)wl.d), g->allocs.end());
    }
    g->status = newst;
    TRY(upload_status(g, g->status));
    TRY(build_lists(g));
    TRY(level_tags(g));
  }
  TRY(collect_cells(g));
  drop_graphs(g);
  CU(cudaMemsetAsync(g->d_bflag, 0, g->nblock_total, g->stream));
  for (int l = 0; l < g->Lmax; ++l) TRY(classify(g, l, 1));
  return LSB_OK;
}

}  // namespace
