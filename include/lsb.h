/*
 * lsb.h - C ABI of the GB300 coupled level-set lattice Boltzmann library.
 *
 * The library advances two immiscible fluid phases, each with its own
 * lattice Boltzmann solver (Sec. 2.1: BGK collision, Eq. feq, Eq. omega,
 * forcing), coupled at a sharp interface given by a level set phi (Sec. 2.2;
 * phi < 0 liquid, phi >= 0 gas) through interpolated bounce-back with the
 * velocity and stress-jump conditions (Sec. 2.3, Eq. bb, bb_cc, Sdecomp),
 * refill of cells that change phase (Sec. 2.4), on a block-structured
 * adaptive Cartesian grid with Dupuis-Chopard level coupling (Sec. 2.1 last
 * paragraph, Sec. 2.5, 2.6).
 *
 * Conventions for every entry point:
 *  - Units are lattice units of the case's FINEST level (dx = dt = 1 there).
 *  - Dense arrays are row-major with x fastest: index x + nx*(y + ny*z).
 *  - Pointers marked "device" must be CUDA device memory of the current
 *    device; pointers marked "host" are ordinary host memory.  The library
 *    never takes ownership of caller buffers.
 *  - All device work is enqueued on the stream given at creation; calls that
 *    return data synchronise that stream.
 *  - Every call validates its arguments before enqueuing work and returns
 *    LSB_EINVAL without side effects on bad input.  Errors raised on the
 *    device (non-finite state, list overflow) are latched and returned by
 *    the next synchronising call (lsb_get_fields, lsb_observables,
 *    lsb_sync).  lsb_last_error() gives a human-readable message.
 *  - A handle is not thread safe: use one handle per host thread/stream.
 */
#ifndef LSB_H
#define LSB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lsb_grid lsb_grid;

typedef enum {
  LSB_OK = 0,
  LSB_EINVAL = 1,    /* invalid argument */
  LSB_ENOMEM = 2,    /* device allocation failed or a work list overflowed */
  LSB_ECUDA = 3,     /* CUDA runtime error */
  LSB_EUNSTABLE = 4, /* non-finite density or velocity detected */
  LSB_ETIMEOUT = 5,  /* a bounded device-side wait gave up */
  LSB_ESTATE = 6     /* call not valid in the handle's current state */
} lsb_status;

enum { LSB_D2Q9 = 0, LSB_D3Q19 = 1, LSB_D3Q27 = 2 }; /* velocity sets, Sec. 2.1 / Fig. 1 */
/* collision operator of a phase: BGK with forcing (Eq. 1), or the cumulant model
 * (D3Q27 only; the paper's gas operator in 3D, Sec. 3.2): second cumulants relaxed
 * with the phase's shear rate (deviatoric part) and rate 1 (trace), every higher
 * cumulant relaxed to zero with rate 1 */
enum { LSB_BGK = 0, LSB_CUMULANT = 1 };
/* per-axis boundary kind: periodic, no-slip wall (half-way bounce-back, Eq. bb
 * with q = 1/2, plus the moving-wall term) or slip wall (specular reflection: a
 * population leaving through the wall returns with its normal component negated,
 * moved on tangentially; the lateral walls of the paper's 3D benchmark, Sec. 3.2).
 * Where a link crosses a slip and a no-slip wall the no-slip bounce-back applies;
 * a reflected link into the other phase takes plain bounce-back. */
enum { LSB_PERIODIC = 0, LSB_WALL = 1, LSB_SLIP = 2 };
enum { LSB_FP32 = 0, LSB_FP16S = 1 };           /* population storage */
enum { LSB_SENSOR_BAND = 0, LSB_SENSOR_SIGNED = 1 }; /* refinement sensor, Sec. 2.6, 3.2.2 */

/* Fields for lsb_get_fields (dense arrays of one level of one case). */
enum {
  LSB_FIELD_RHO = 0,   /* normalised density rho_hat (float, 1 per cell)           */
  LSB_FIELD_U = 1,     /* velocity, D floats per cell, component-major (D x cells) */
  LSB_FIELD_PHI = 2,   /* level set (float, finest level only)                     */
  LSB_FIELD_PHASE = 3, /* uint8 per cell: 0 liquid, 1 gas                          */
  LSB_FIELD_F = 4,     /* populations f_i (float, Q x cells, Fig. 1 order)         */
  LSB_FIELD_TAG = 5,   /* uint8 per cell: bit0 phase, bit1 interface cell,
                          bit2 flipped at the last step, bit3 previous phase,
                          bit4 covered cell streamed from by a leaf, bit5 ghost   */
  LSB_FIELD_BLOCKS = 6,/* int8 per block: 0 inactive, 1 leaf, 2 refined           */
  LSB_FIELD_CUTMASK = 7,/* uint32 per cell: bit k set when the incoming direction
                          k's source lies in the other phase (finest level)       */
  LSB_FIELD_KAPPA = 8, /* curvature at interface cells (float, finest level)      */
  LSB_FIELD_UEXT = 9,  /* extension velocity u~ (D x cells, finest level)         */
  LSB_FIELD_ADJ_F = 10,/* after lsb_backward: dJ/df at the start of the recorded
                          window (float, Q x cells, Fig. 1 order)                 */
  LSB_FIELD_ADJ_UEXT = 11 /* after lsb_backward over a moving level set: dJ/du~ at
                          the start of the window (D x cells, finest level)      */
};

/* Geometry and discretisation of one case, fixed for the handle's life. */
typedef struct {
  int lattice;          /* LSB_D2Q9, LSB_D3Q19 or LSB_D3Q27 (FP32 storage only);
                           all cases share it                                       */
  int base[3];          /* base-level cells per axis (base[2] ignored in 2D)         */
  int n_levels;         /* total levels including the base (1 = uniform), <= 4       */
  int block[3];         /* block edge in cells, powers of two, same on every level;
                           their product is a multiple of 32 and at most 512        */
  int bc[3];            /* per axis: LSB_PERIODIC, LSB_WALL or LSB_SLIP (walls on cell faces) */
  double wall_u[6][3];  /* velocity of faces x-, x+, y-, y+, z-, z+                  */
  int storage;          /* LSB_FP32 or LSB_FP16S; all cases of a handle share it     */
  double fp16_scale;    /* LSB_FP16S: populations stored as (f - w) * scale, a power
                           of two that keeps them out of the half subnormal range   */
  int collision[2];     /* operator of [0] liquid, [1] gas: LSB_BGK or LSB_CUMULANT
                           (D3Q27 only); zero-initialised = BGK in both            */
} lsb_grid_desc;

/* Physics and method parameters of one case (lattice units of the finest level). */
typedef struct {
  double rho[2];        /* physical densities: [0] liquid (phi < 0), [1] gas        */
  double nu[2];         /* kinematic viscosities on the finest level (Eq. omega)    */
  double body_force[3]; /* force density, acts as acceleration body_force/rho_k     */
  double gravity[3];    /* acceleration acting on both phases                       */
  double sigma;         /* surface tension (Eq. Sdecomp)                            */
  double x_ref[3];      /* hydrostatic reference point for the initial density:
                           rho_hat = 1 - gravity.(x - x_ref)/c_s^2, plus in the gas
                           p_gas0 / (rho[1] c_s^2)                                   */
  double p_gas0;        /* initial gas gauge pressure (e.g. its Laplace pressure)    */
  int n_ext;            /* extension sweeps per step (Eq. hyperbolicExtension)      */
  double dtau_ext;      /* extension pseudo time step                               */
  int reinit_every;     /* reinitialise every this many finest steps (0 = never)    */
  int n_reinit;         /* TVD-RK3 pseudo steps per reinitialisation                */
  double dtau_reinit;   /* reinitialisation pseudo time step                        */
  double refine_dist[4];/* sensor distance per level l < n_levels-1 (finest cells)  */
  int sensor;           /* LSB_SENSOR_BAND or LSB_SENSOR_SIGNED                      */
  int regrid_every;     /* regrid every this many coarse steps (0 = never)          */
  int ls_active;        /* 0 freezes the level set (no transport, no refill)        */
} lsb_params;

/*
 * Create a handle holding n_cases independent cases (an ensemble; n_cases = 1
 * for a single simulation).  descs/params: arrays of n_cases host structs.
 * phi0: array of n_cases DEVICE pointers, each the case's initial level set
 * on its finest level (float, dense, x fastest, base * 2^(n_levels-1) cells
 * per axis).  stream: a cudaStream_t (NULL = legacy default stream).
 * The initial grid is refined from phi0 by the sensor (Sec. 2.6), the
 * populations set to rest equilibrium with the hydrostatic density of
 * params.gravity / x_ref.  On success *out receives the handle; the caller
 * frees it with lsb_destroy.  Errors: LSB_EINVAL (bad descriptor or
 * parameters, e.g. nu <= 0, odd block edge, mismatched lattices),
 * LSB_ENOMEM, LSB_ECUDA.
 */
lsb_status lsb_create_grid(int n_cases, const lsb_grid_desc *descs, const lsb_params *params,
                           const float *const *phi0, void *stream, lsb_grid **out);

/* Replace the physics parameters of one case (case_idx) or all (-1); takes
 * effect at the next step.  Grid-shaping fields (refine_dist, sensor) apply
 * at the next regrid.  Errors: LSB_EINVAL. */
lsb_status lsb_set_params(lsb_grid *g, int case_idx, const lsb_params *params);

/* Advance every case by n coarse steps (each is 2^(n_levels-1) finest steps
 * of that case), Sec. 2 method.  Asynchronous on the handle's stream. */
lsb_status lsb_step(lsb_grid *g, int n);

/* Replay steps from CUDA graphs (enable = 1) instead of launching each kernel.
 * Graphs hold two coarse steps, or one for an odd remainder (so lsb_step(g, 1)
 * replays too), one graph per level-0 buffer parity at the start; they are
 * re-captured after every regrid and after an lsb_set_params call that
 * changes the launch sequence (level-set iteration counts, regrid interval,
 * level set on or off).  Two-step replays are not used across a regrid; steps
 * while kernel timing is on and handles whose reinitialisation period is
 * above 1 run eagerly.  Needs the handle to use a non-default stream
 * (LSB_EINVAL otherwise).  Results are identical to eager stepping. */
lsb_status lsb_use_graphs(lsb_grid *g, int enable);

/*
 * Launch structure of the level-set update (Sec. 2.2 passes: extension sweeps,
 * TVD-RK3 transport, reinitialisation).  mode 0 (default): one launch per pass
 * (up to 16 per finest step).  mode 1: one persistent cooperative launch per
 * finest step that runs every pass over the band work list of all cases, with
 * a device-wide barrier between passes; the barrier's wait has an iteration
 * limit, and on expiry the kernel ends and the next synchronising call returns
 * LSB_ETIMEOUT.  Both modes give identical results.  Errors: LSB_EINVAL (bad
 * mode, or no cooperative launch on this device).
 */
lsb_status lsb_set_driver(lsb_grid *g, int mode);

/*
 * Iteration limit of the library's bounded device-side waits (the grid barrier
 * of lsb_set_driver mode 1; the paper has no counterpart).  A waiting CTA
 * sleeps ~64 ns per iteration and, after `spins` iterations, records the
 * timeout, leaves the kernel, and the next synchronising call returns
 * LSB_ETIMEOUT (a latched error: the handle stays in error; the CUDA context
 * stays usable).  Default 2^22 (~0.3 s).  0 makes every wait that would have to
 * wait give up at once, which exercises the timeout path without a stalled
 * GPU.  Errors: LSB_EINVAL (negative spins).
 */
lsb_status lsb_set_wait_limit(lsb_grid *g, long long spins);

/* Run the refinement sensor and regrid every case now (Sec. 2.6). */
lsb_status lsb_refine(lsb_grid *g);

/*
 * Copy one field of one level of one case into dst (dense over that level's
 * box; see the LSB_FIELD_* list for element type and count).  dst_bytes must
 * be at least the field size (lsb_field_bytes); dst_on_host selects a host
 * or device destination.  Synchronises the stream.  Errors: LSB_EINVAL,
 * LSB_ECUDA, or a latched device error.
 */
lsb_status lsb_get_fields(lsb_grid *g, int case_idx, int field, int level, void *dst,
                          size_t dst_bytes, int dst_on_host);

/*
 * Allocation-free variant of lsb_get_fields for LSB_FIELD_RHO, LSB_FIELD_U and
 * LSB_FIELD_F (the paper has no counterpart: this is a service of the library).
 * lsb_get_fields stages these fields in a temporary cudaMalloc buffer; this
 * entry point stages them in a fixed 16 MiB array that the library reserves
 * on every GPU it is loaded on, held until the process exits.  It is meant
 * for callers that cannot allocate device memory at the point of the call:
 * code whose device memory is entirely owned by another allocator (such as a
 * framework's caching allocator), real-time loops that cannot afford an
 * allocation's latency or its implicit synchronisation, or callbacks in
 * which allocation is not permitted.  It calls no cudaMalloc or cudaFree.
 * The first call on a device resolves the array's device address (with that
 * device current); make that first call before any stream capture.
 * Fields larger than 16 MiB are rejected with LSB_EINVAL.  Every call shares
 * the one array: calls whose work overlaps on the GPU (two handles on
 * different streams, or two host threads) race and must be serialised by the
 * caller.  Each call writes the whole staged range before copying it out, so
 * nothing carries over from an earlier call.  Arguments and result as for
 * lsb_get_fields; synchronises the handle's stream.
 */
lsb_status lsb_get_fields_noalloc(lsb_grid *g, int case_idx, int field, int level, void *dst,
                                  size_t dst_bytes, int dst_on_host);

/*
 * Gas indicator of the volume, centroid and velocity observables (Sec. 3.2 gives them
 * as integrals over the gas region).  eps = 0 (default): the sharp indicator [phi >= 0]
 * (the leaf's phase).  eps > 0: the smoothed indicator H_eps(phi) = 1/2 (1 + t +
 * sin(pi t)/pi), t = phi/eps on |phi| <= eps (0 below, 1 above), of phi at the leaf's
 * first finest child, eps in finest cells (1.5 is the usual width).  The masses stay
 * phase sums.  With the sharp indicator these observables are piecewise constant in
 * phi, so their adjoint gradients with respect to sigma, the densities, viscosities or
 * the initial interface vanish between cell flips; the smoothed one makes them
 * differentiable: lsb_observables and lsb_backward use it, and dJ/dphi0 then also
 * carries the indicator's own dependence on phi.  Ends a recording (lsb_record).
 * Errors: LSB_EINVAL (negative or non-finite eps).
 */
lsb_status lsb_set_objective(lsb_grid *g, double eps);

/* Bytes lsb_get_fields writes for (case, field, level); 0 for invalid input. */
size_t lsb_field_bytes(const lsb_grid *g, int case_idx, int field, int level);

/*
 * Observables of every case in float64 (Sec. 3.2: bubble centroid and
 * velocity as Heaviside-weighted integrals), written to a host array of
 * n_cases * (4 + 2*D) doubles per case: mass liquid, mass gas, gas volume,
 * number of leaf cells updated per coarse step, centroid[D], velocity[D];
 * lengths in finest cells.  Synchronises.  LSB_EUNSTABLE if a density or
 * velocity is not finite.
 */
lsb_status lsb_observables(lsb_grid *g, double *out_host, size_t n_doubles);

/*
 * Block-shape autotuner (the paper has no counterpart; the block edge is a
 * free parameter of the block-structured grid, Sec. 2.5).  For each candidate
 * shape (candidates: host array of n_cand x 3 ints, block edges x, y, z; NULL
 * = six built-in shapes for the lattice of descs[0], n_cand ignored) it
 * creates the handle with that block shape for every case, runs 2 untimed
 * coarse steps, times `steps` coarse steps with CUDA events on `stream`
 * (a cudaStream_t, NULL = legacy default) and destroys the handle.
 * best: host, 3 ints, receives the fastest shape; ms_per_step: host array of
 * n_cand doubles (6 with NULL candidates) or NULL, receives each candidate's
 * milliseconds per coarse step (NaN for a shape that was rejected or failed).
 * Other arguments as for lsb_create_grid.  Block shape changes the refined
 * region (the sensor marks whole blocks), so the candidates are compared by
 * wall time per coarse step of the same problem.  Synchronises.  Errors:
 * LSB_EINVAL (bad arguments, or no candidate ran; lsb_last_error(NULL) says
 * why).
 */
lsb_status lsb_autotune(int n_cases, const lsb_grid_desc *descs, const lsb_params *params,
                        const float *const *phi0, void *stream, const int *candidates, int n_cand, int steps,
                        int *best, double *ms_per_step);

/* Cell updates (the MLUPS numerator): per_coarse_step = sum over levels of
 * leaf cells x 2^level for the current grid (all cases); total_done = the same
 * summed over every coarse step taken so far (regrids change the per-step
 * count).  Either pointer may be NULL.  Needs no synchronisation. */
lsb_status lsb_cell_updates(const lsb_grid *g, double *per_coarse_step, double *total_done);

/*
 * Sizes of the work lists of global level `level` (summed over the cases whose
 * level it is) as they stand after the last step, for diagnostics and the
 * throughput accounting (the paper has no counterpart): out[0] leaf cells,
 * out[1] band cells (band blocks x block cells), out[2] interface cells,
 * out[3] cut links, out[4] cells flipped at the last finest step (1..4: the
 * finest level of a case only, else 0), out[5] ghost-ring cells filled from
 * the coarser level, out[6] covered cells restricted from the finer level.
 * Host array of n <= LSB_NWORK values.  Synchronises.  Errors: LSB_EINVAL.
 */
enum { LSB_NWORK = 7 };
lsb_status lsb_work_counts(lsb_grid *g, int level, long long *out, int n);

/* Velocity-set tables compiled into the library (Sec. 2.1, Fig. 1): c receives
 * Q x 3 ints, w Q floats, opp Q ints (opposite directions); any may be NULL.
 * Returns Q, or 0 for an unknown lattice.  Needs no GPU. */
int lsb_lattice_table(int lattice, int *c, float *w, int *opp);

/*
 * Adjoint (the paper has no counterpart; the differentiated map is its
 * step, Sec. 2).  lsb_backward computes, for J = sum over cases of
 * dJ_dobs . observables (the lsb_observables vector after the last recorded
 * step), the exact derivatives of the discrete step map by a hand-written
 * reverse sweep, on windows where the discrete decisions of the method stay
 * fixed:
 *  - frozen level set (ls_active = 0 in every case): the phases, cut links,
 *    q, n and kappa are constants; transposes of the collision with forcing,
 *    the streaming with wall bounce-back and the interface bounce-back of
 *    Eq. bb with Eq. bb_cc and Eq. Sdecomp; on block-refined grids (Sec. 2.1,
 *    last paragraph; Sec. 2.6) also of the level recursion: the restriction
 *    to the covered cells leaves stream from (children mean, f^neq scaled by
 *    2 tau_c / tau_f), the fine ghost ring's values at t and t + 1/2 (coarse
 *    interpolation, f^neq scaled by tau_f / (2 tau_c), fine collision) and
 *    every level's sub-steps, with the block layout fixed (recorded steps do
 *    not regrid) and every case on the same number of levels;
 *  - moving level set (ls_active = 1 in every case, reinit_every <= 1,
 *    n_reinit <= 1): the state is (f, phi, u~) and the sweep also transposes
 *    the interface velocity, the extension sweeps (Eq.
 *    hyperbolicExtension), the TVD-RK3 upwind-5 transport and the HJ-WENO5
 *    reinitialisation (Sec. 2.2), with phases, cut links, band, frozen cells,
 *    upwind sides and Godunov branches as in the forward steps.  No cell may
 *    change phase inside the window (refill is not differentiated):
 *    lsb_backward returns LSB_ESTATE if one did.  On block-refined grids the
 *    level set lives on the finest level and advances in each of its
 *    sub-steps; the coarser levels keep the phases of the last regrid.
 *
 * lsb_record(g, checkpoint_every): start a recording at the current state.
 * The following lsb_step calls run eagerly (no CUDA graphs) and copy the
 * state (populations; with a moving level set also phi and u~) into a device
 * checkpoint at the start of every checkpoint_every-th step (allocated as
 * needed).  A new lsb_record, lsb_set_params or lsb_refine ends the
 * recording and frees the checkpoints.  Recorded steps never regrid.
 * Errors: LSB_EINVAL (checkpoint_every < 1), LSB_ESTATE (FP16 storage, D3Q27,
 * cases mixing live and frozen level sets, a moving level set with
 * reinit_every > 1 or n_reinit > 1, or cases with different numbers of levels
 * on a multi-level grid).
 *
 * lsb_backward(g, dJ_dobs, dJ_dparams, dJ_dphi0): reverse sweep over every
 * step recorded so far.  Segment by segment, from the last, it restores the
 * checkpoint, recomputes the segment's steps keeping their states (device
 * memory for checkpoint_every states), and runs the adjoint steps backwards
 * (with a moving level set each adjoint step first replays that step's
 * level-set passes; on a multi-level grid each adjoint step first replays
 * its coarse step, keeping every level's populations per call of the level
 * recursion: 2^L - 1 further states plus 2^(L-1) - 1 for the coarse
 * sub-steps' results, and with a moving level set phi and u~ at the start of
 * each finest sub-step; allocated on the first multi-level lsb_backward).
 * dJ_dobs: host, n_cases x (4 + 2 D) doubles, weights of the observables
 * in lsb_observables order (centroid, volume and leaf count are constants of
 * the map).  dJ_dparams: host, n_cases x LSB_NPARAM_ADJ doubles, or NULL;
 * per case dJ/dsigma, dJ/drho[0], dJ/drho[1], dJ/dnu[0], dJ/dnu[1] at the
 * recorded start state.  dJ_dphi0: device, or NULL; receives for each case
 * in order the dense finest-level array (x fastest) of dJ/dphi at the start
 * of the window: frozen level set: through the link fractions q (radiation
 * theorem, Sec. 2.3) and the interface cells' normal and curvature from the
 * least-squares fit (Sec. 2.2); moving level set: through every pass of
 * every step.  Valid for perturbations of phi that change no sign.
 * Afterwards the state is that of the last recorded step again, the
 * recording stays open (lsb_backward may be called again, e.g. with other
 * weights, and lsb_step extends the recording), LSB_FIELD_ADJ_F returns dJ/df
 * (per level; zero outside the leaves) and, with a moving level set,
 * LSB_FIELD_ADJ_UEXT dJ/du~ at the start of the window.  FP32 adjoint fields, FP64 parameter sums.  Synchronises.  Errors:
 * LSB_EINVAL, LSB_ESTATE (no recording, or a phase change in the window),
 * LSB_ENOMEM, LSB_ECUDA.
 */
enum { LSB_NPARAM_ADJ = 5 };
lsb_status lsb_record(lsb_grid *g, int checkpoint_every);
lsb_status lsb_backward(lsb_grid *g, const double *dJ_dobs, double *dJ_dparams, float *dJ_dphi0);

/* Kernel timing for diagnostics and the bench roofline: mode 0 off, 1 times
 * every collide-and-stream launch (one class per level: k_collide_stream,
 * k_collide_stream_l1, _l2, _l3), 2 times every launch.  Timed launches are
 * bracketed by CUDA events on the handle's stream (a few microseconds each).
 * Calling it discards earlier records.  Synchronises. */
lsb_status lsb_profile(lsb_grid *g, int mode);

/* Per kernel class k < n (see lsb_kernel_name): device milliseconds, launches
 * and algorithmic bytes (collide-and-stream: 2*Q*sizeof(storage) per leaf cell
 * update) summed over the records since the last lsb_profile or
 * lsb_profile_read; consumes them.  Any output pointer may be NULL.  Synchronises. */
lsb_status lsb_profile_read(lsb_grid *g, double *ms, double *bytes, uint64_t *launches, int n);

/* Name of kernel class k, or NULL; lsb_kernel_count() classes exist. */
const char *lsb_kernel_name(int k);
int lsb_kernel_count(void);

/* Wait for the handle's stream and return any latched device error. */
lsb_status lsb_sync(lsb_grid *g);

/* Number of kernels launched by the handle so far (all entry points). */
uint64_t lsb_kernel_launches(const lsb_grid *g);

/* Last error message of the handle, or of a failed lsb_create_grid when g is NULL. */
const char *lsb_last_error(const lsb_grid *g);

/* Free every device buffer of the handle.  NULL is ignored. */
void lsb_destroy(lsb_grid *g);

#ifdef __cplusplus
}
#endif

#endif /* LSB_H */
