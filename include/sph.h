/*
 * sph.h -- C ABI of libsph.so, the GB300 (sm_103a) hot path of the weakly
 * compressible SPH method of the DualSPHysics paper (arXiv 2104.00537).
 *
 * One "engine" holds one or more independent SPH cases resident in device
 * memory and advances them together, one Symplectic step at a time (Sect. 5.1:
 * neighbour list NL -> particle interaction PI -> system update SU, Fig. 7).
 * A single case is an engine with one case (sph_create); a batch is an
 * engine created with many (sph_batch_create); a serving pool is an engine
 * whose cases are admitted and released while it runs (sph_pool_*).
 *
 * Conventions for every call:
 *  - Return SPH_OK (0) on success or a negative SPH_ERR_* code; the message
 *    of the last error of the calling thread is in sph_last_error().
 *  - Host pointers are caller-owned and only read (inputs) or written
 *    (outputs) during the call; the library keeps no reference to them.
 *  - Device memory is allocated at creation / admission only, through the
 *    caller's allocator callback when one is given, else cudaMalloc, and is
 *    released by the matching destroy call.
 *  - All device work runs on the CUDA stream given at creation; calls that
 *    return host data synchronise that stream.  One engine must not be used
 *    from two threads at once; different engines are independent.
 *  - Arrays of particles are in the caller's (generator) order on input and
 *    on output; the device order (sorted by cell) is internal.
 */
#ifndef SPH_H
#define SPH_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SPH_OK 0
#define SPH_ERR_ARG (-1)      /* invalid argument or parameter            */
#define SPH_ERR_OOM (-2)      /* allocation failed / capacity exhausted   */
#define SPH_ERR_CUDA (-3)     /* a CUDA runtime call failed               */
#define SPH_ERR_UNSTABLE (-4) /* NaN/Inf in the state or dt < dt_min      */
#define SPH_ERR_DOMAIN (-5)   /* more particles left the domain than allowed */
/* (-6) is not used: no kernel of the library waits on a flag or a peer, so
 * there is no bounded device wait that could give up */
#define SPH_ERR_BUSY (-7)     /* pool: no free slot or not enough memory  */
#define SPH_ERR_STATE (-8)    /* call not valid in the engine's state     */

typedef struct { double x, y, z; } sph_d3;

/* Constants of one case.  Paper references: h, the Wendland C2 kernel with
 * support 2h (Eq 11); rho0, cs0, gamma of the Tait equation of state (Eq 28);
 * alpha of the artificial viscosity (Eq 21); delta of the density diffusion
 * term (Eq 17-18); cfl = C_CFL of Eq 35; eta2 = eta^2 of Eq 21 and 35. */
typedef struct {
  double dp;        /* initial particle spacing; particle mass m = rho0 dp^3 */
  double h, rho0, cs0, gamma, alpha, delta, cfl, eta2;
  sph_d3 gravity;   /* body force f of Eq 13 (m/s^2)                        */
  sph_d3 domain_min, domain_max; /* particles outside are frozen ("out")    */
  double dt_fixed;  /* > 0: fixed time step instead of Eq 35                */
  double dt_min;    /* a step with dt < dt_min fails with SPH_ERR_UNSTABLE  */
  int32_t cell_mode;          /* 0: cells of 2h (Sect. 5.1); 1: of h (Sect. 5.3); 2: of 2h/3 */
  int32_t ddt_mode;           /* 0: no density diffusion; 1: Eq 17 with Eq 18;
                               * 2: Eq 17 with Eq 19-20 (dynamic density)  */
  int32_t clamp_boundary_rho; /* 1: boundary density kept >= rho0           */
  int32_t max_out;            /* out-of-domain quota; < 0: unlimited        */
  int32_t integrator;         /* 0: Symplectic, Eq 33-34 (two PI per step);
                               * 1: Verlet, Eq 30-31 (one PI per step).  All
                               * cases of one engine use the same scheme;
                               * pools run the Symplectic scheme only.     */
  int32_t verlet_steps;       /* N_S of Eq 31: a step whose count of completed
                               * steps is a multiple of N_S (the first step
                               * included) is an Eq 31 step; 0 means 40    */
  int32_t visc_mode;          /* 0: artificial viscosity (Eq 21-22, alpha);
                               * 1: laminar viscosity (Eq 23, nu0) + SPS
                               * turbulence (Eq 24-27, C_S = 0.12, C_l =
                               * 0.0066, Delta = dp); needs one more
                               * neighbour pass per interaction             */
  int32_t boundary_mode;      /* 0: dynamic boundary condition, Eq 36;
                               * 1: modified DBC, Eq 38-39 (needs ghost
                               * offsets, sph_particles.ghost)             */
  double nu0;                 /* kinematic viscosity of Eq 23 (m^2/s)       */
  int32_t mdbc_slip;          /* mDBC boundary velocity: 0 the imposed one
                               * (Eq 37); 1 no-slip, v_B = 2 v_wall - v_G;
                               * 2 free slip: the tangential part of v_G
                               * with the normal part of 2 v_wall - v_G
                               * (normal along the ghost offset)            */
  int32_t pad2_;
} sph_case_params;

/* Imposed translation of a group of boundary particles (Eq 37):
 * displacement D(t) = amplitude (sin(omega t + phase) - sin(phase)) along
 * axis, velocity D'(t) axis. */
typedef struct {
  sph_d3 axis;
  double amplitude, omega, phase;
} sph_motion;

/* Initial particles of one case (the sets P = F u B of Sect. 2.1). */
typedef struct {
  int64_t n;                    /* number of particles                         */
  const double *pos;            /* [3n] x,y,z (m)                              */
  const float *vel;             /* [3n] or NULL for zero                       */
  const float *rho;             /* [n] density (kg/m^3)                        */
  const uint8_t *type;          /* [n] 0 fluid (F), 1 boundary (B)             */
  const int32_t *motion_group;  /* [n] index into motions, -1 fixed; or NULL   */
  const sph_motion *motions;    /* [n_motions] (at most 8 per case)            */
  int32_t n_motions;
  const float *ghost;           /* [3n] mDBC ghost offset r_G - r_B of each
                                 * boundary particle (the mirror image across
                                 * the wall surface, Sect. 2.6.2); required
                                 * when boundary_mode = 1, else ignored     */
} sph_particles;

/* Counters and diagnostics of one case (FP64 reductions on the device). */
typedef struct {
  double t;              /* simulated time                                  */
  double last_dt;        /* last Eq 35 time step                            */
  int64_t step;          /* completed time steps                            */
  int64_t interactions;  /* evaluated ordered pairs (a,b), all PI evaluations */
  int64_t interactions_fb; /* ... of which a in F, b in B                    */
  int64_t interactions_bf; /* ... of which a in B (b in F, Eq 36)             */
  double mass;           /* sum of particle masses (Eq 14)                  */
  double kinetic_energy; /* sum over F of m |v|^2 / 2                       */
  double momentum[3];    /* sum over F of m v                               */
  double front;          /* max x over in-domain fluid particles            */
  int64_t n_out;         /* particles frozen outside the domain             */
  int32_t flags;         /* bit 0 NaN/Inf, bit 1 dt < dt_min, bit 2 quota   */
  int32_t n_fluid;
  int64_t n;
} sph_stats;

typedef struct sph_engine_t *sph_engine;

/* Device allocator callback (e.g. the PyTorch caching allocator); must
 * return memory usable on `stream`, aligned to at least 256 bytes. */
typedef void *(*sph_alloc_fn)(size_t bytes, void *stream, void *ctx);
typedef void (*sph_free_fn)(void *ptr, size_t bytes, void *stream, void *ctx);

/* Engine-wide launch options (the autotuner's knobs). */
typedef struct {
  int32_t pi_block;   /* threads per block of the list walk of the default
                       * physics: 0 (default: 128), 128, 256, 512 or 1024;
                       * the other interaction kernels use 128 */
  int32_t pi_variant; /* interaction pair loop: -1 the engine default (5 where
                       * a list is supported, else 0); 0 compacted hit
                       * masks; 1 test
                       * and evaluate inline; 2 hit masks queued per lane
                       * across rows (same sums as 0, bit for bit); 3, 4
                       * and 5 a neighbour list: candidates within 2h + skin
                       * of state n in chunk records, walked by both
                       * evaluations of a Symplectic step, no re-sort for
                       * the half step; 3 writes the list during the first
                       * evaluation, 4 builds it alone, once per step; 5
                       * builds it with a larger skin and keeps it (and the
                       * particle order and cells) across steps until a
                       * particle could leave the skin, decided on the
                       * device per case (a case of a batch or pool takes
                       * the steps it takes alone, bit for bit, however
                       * the steps are split into calls).  5 also serves
                       * the Verlet scheme; 3 and 4 with Verlet, and any
                       * list beyond 2^25 particles, fall back to 0; 6 the
                       * cell walk with warp-shared candidate tiles: the
                       * lanes of a warp in one row of cells stage the
                       * union of their candidates 32 at a time in shared
                       * memory and each tests every staged candidate
                       * (default physics; the extended terms take 0)    */
  int32_t use_graph;  /* 1: replay each step from a captured CUDA graph        */
  int32_t timing;     /* 1: time every PI launch and every step with CUDA
                       * events (sph_get_timing, sph_get_step_times); the
                       * steps then run without the captured step graph   */
  float list_skin;    /* pi_variant 5: skin added for the steps the list is
                       * kept, as a fraction of 2h, in [0, 0.25]; < 0: the
                       * default (0.04)                                    */
  int32_t check_list; /* 1: after every list evaluation, count the pairs of
                       * every target by brute force and compare (tests;
                       * sph_list_info reports the result)                */
  int32_t pi_lanes;   /* threads that share one target in the list walk
                       * (pi_variant 3-5): 0 (default: 1), 1, 2, 4 or 8;
                       * thread k of a target takes the candidates at bit
                       * positions k, k + lanes, ... of each chunk record and
                       * the partial sums are added at the end, so the sums'
                       * order (not the pair set) depends on it           */
  int32_t pair_once;  /* 1: the list walk (pi_variant 3-5) of an engine with
                       * the default physics (Eq 18 or no diffusion,
                       * Eq 21 viscosity, DBC) evaluates each pair once:
                       * the target of lower index takes the pair and adds
                       * the partner's share (Eq 22's antisymmetric
                       * momentum term, its continuity term) by atomic
                       * vector additions, so the sums are not the same
                       * bit for bit from run to run, alone, in a batch or
                       * in a pool; other engines (and a pool once it has
                       * admitted a case with other physics) evaluate as
                       * with 0.  0 (default): every target sums its own
                       * pairs, deterministically                         */
  int32_t wide_records; /* 1: neighbour-list records with a 32-bit first
                       * index and no row code (the walk takes a record's
                       * row from its first candidate's cell) at any size;
                       * 0: only where the engine needs them, beyond 2^25
                       * particles.  The default physics only (Eq 18 or no
                       * diffusion, Eq 21 viscosity, DBC); the pair set and
                       * the order of the sums are those of the narrow
                       * records, so results are the same bit for bit    */
} sph_options;

/* Last error message of the calling thread ("" if none). */
const char *sph_last_error(void);

/* ---- single case -------------------------------------------------------
 * sph_create: copy one case to the device (Sect. 5.1: data are copied once
 * and stay resident) and build its cell grid.  stream: cudaStream_t or NULL
 * for the default stream.  alloc/free: optional allocator, ctx passed back. */
int sph_create(const sph_case_params *params, const sph_particles *parts,
               void *stream, sph_alloc_fn alloc, sph_free_fn free_fn,
               void *alloc_ctx, sph_engine *out);

/* sph_step: advance every case of the engine by nsteps steps of its scheme:
 * Symplectic (Eq 33-34): PI (state n) -> dt (Eq 35) -> predictor -> PI
 * (state n+1/2) -> corrector; Verlet (Eq 30-31): PI -> dt -> update.  The
 * neighbour list behind each PI is rebuilt as pi_variant says (0-2: a cell
 * walk per PI; 3, 4: one list per step; 5: a case's list kept until one of
 * its particles could leave the skin; a call continues the previous call's
 * lists unless cases were admitted or released, a snapshot was taken or a
 * parity helper re-sorted the state, which rebuild them).  Work is queued
 * on the engine's stream; the call returns after synchronising and checking
 * the failure flags (a list overflow or skin violation is an error, never a
 * dropped pair). */
int sph_step(sph_engine e, int64_t nsteps);

/* sph_get_state: copy case `icase` (0 for a single case) to host arrays in
 * the caller's original particle order.  Any output pointer may be NULL.
 * pos [3n] double, vel [3n] float, rho [n] float, press [n] float (Eq 28). */
int sph_get_state(sph_engine e, int32_t icase, double *pos, float *vel,
                  float *rho, float *press, double *t, int64_t *step,
                  double *last_dt);

/* sph_get_stats: counters and FP64 diagnostics of case icase. */
int sph_get_stats(sph_engine e, int32_t icase, sph_stats *out);

/* sph_set_options / sph_get_timing: launch options; with timing on, the
 * accumulated device time of the interaction kernel (ms, CUDA events on the
 * engine's stream), its number of launches, the device time of whole
 * sph_step calls, and the number of kernels launched by sph_step since the
 * last reset (reset = 1 clears all after reading). */
int sph_set_options(sph_engine e, const sph_options *opt);
int sph_get_timing(sph_engine e, double *pi_ms, int64_t *pi_launches,
                   double *step_ms, int64_t *kernel_launches, int32_t reset);

/* sph_get_step_times: with timing on, the device time of each step timed
 * since the last reset of sph_get_timing, in ms (CUDA events on the engine's
 * stream: from the start of a step's first interaction evaluation to the
 * start of the next step's; for the last step of an sph_step call, to the
 * end of that call).  Copies min(*n, cap) values to the caller-owned host
 * array ms (NULL or cap = 0: none); *n (may be NULL) receives the number of
 * steps stored, at most 1,048,576 between resets.  SPH_ERR_ARG for a null
 * engine or cap < 0.  Used for the p50/p99 step time of a run. */
int sph_get_step_times(sph_engine e, float *ms, int64_t cap, int64_t *n);

/* sph_list_info: neighbour-list builds since the engine was created (the
 * rebuilds of pi_variant 5, or one per step for 3 and 4), and with
 * check_list on the pairs found by brute force and the number of targets
 * whose list yielded a different count (0: every pair inside 2h was in the
 * list).  Any output pointer may be NULL. */
int sph_list_info(sph_engine e, int64_t *builds, int64_t *check_pairs,
                  int64_t *check_bad);

/* ---- checkpoint ----------------------------------------------------------
 * sph_get_raw: bit-exact snapshot of case icase (device storage format:
 * integer cell + float offset, float velocity/density, time, step, dt; for
 * the Verlet scheme also v^{n-1} and rho^{n-1} of Eq 30).  With buf == NULL
 * only *bytes is set.  sph_create_from_raw rebuilds a single-case engine
 * that continues bit-identically (a Verlet engine needs a Verlet snapshot). */
int sph_get_raw(sph_engine e, int32_t icase, void *buf, size_t *bytes);
int sph_create_from_raw(const sph_case_params *params, const sph_particles *parts,
                        const void *buf, size_t bytes, void *stream,
                        sph_alloc_fn alloc, sph_free_fn free_fn, void *alloc_ctx,
                        sph_engine *out);

/* ---- parity / diagnostic entry points -----------------------------------
 * sph_eval_forces: rebuild the neighbour list and evaluate the particle
 * interaction once on the current state of case icase, without advancing
 * it.  Outputs in original order: acc [3n] (dv/dt of Eq 22 + f, zero for
 * B), drho [n] (Eq 15 with D_a, Eq 36 for B), mumax [n] (inner max of Eq 35);
 * *dt = the Eq 35 step from this evaluation.  Any output may be NULL. */
int sph_eval_forces(sph_engine e, int32_t icase, float *acc, float *drho,
                    float *mumax, double *dt, int64_t *pairs);

/* sph_eval_step: one interaction evaluation of the next step of the engine's
 * scheme, through the very launches sph_step makes (Sect. 5.1, Fig. 7; Eq 15-18,
 * 21-22, 35-36), without advancing the engine.  stage 0: the step's first
 * evaluation, on state n; stage 1: its second, on the half-step state of
 * Eq 33-34 (dt of Eq 35 from stage 0, then the predictor).  With a neighbour
 * list (pi_variant 3-5) both walk the list's chunk records, and with the list
 * kept across steps (5) state n and state n+1/2 are those kept in the order
 * and cells of the list's build (cell offsets up to half the skin outside
 * [0, cs)).  The part of the next step before its first evaluation runs for
 * real -- a pending rebuild of the kept list, or the sort of a per-step list
 * or cell walk -- and everything else the next step reads is restored, so
 * sph_step afterwards takes the steps it would have taken (bit for bit with
 * each target's own sums; with pair_once the evaluations take the pair-once
 * walk, whose atomic sums vary in their last bits from run to run).
 * Outputs, caller-owned host buffers in the caller's particle order, any may
 * be NULL: pos [3n] (FP64, from the evaluated cell + offset), vel [3n], rho [n]
 * the evaluated state; acc [3n] dv/dt of Eq 22 + f (zero for B), drho [n]
 * (Eq 15 with D_a; Eq 36 for B), mumax [n] the inner max of Eq 35 (zero for
 * B); *dt the Eq 35 step of the step's first evaluation; *pairs the ordered
 * pairs of this evaluation (Eq 4 support).  Particles frozen outside the
 * domain report zero results.  SPH_ERR_ARG for a stage other than 0 or 1,
 * or stage 1 on a cell walk (pi_variant 0-2) or the Verlet scheme (one
 * evaluation per step); SPH_ERR_UNSTABLE (NaN/Inf, or the half step left the
 * skin) and SPH_ERR_STATE (list overflow) as sph_step reports them. */
int sph_eval_step(sph_engine e, int32_t icase, int32_t stage, double *pos, float *vel,
                  float *rho, float *acc, float *drho, float *mumax, double *dt,
                  int64_t *pairs);


/* sph_eval_sps: tau / rho of Eq 25 (the SPS stress of Eq 24-25 with the
 * velocity gradient of the SPH estimate over b in P) for every particle of
 * case icase, on its current state and without advancing it.  tau6 [6n]
 * caller-owned host buffer, original particle order, per particle xx, yy,
 * zz, xy, xz, yz; zero for boundary particles, frozen particles and cases
 * with visc_mode 0.  SPH_ERR_STATE if no case of the engine uses
 * visc_mode 1. */
int sph_eval_sps(sph_engine e, int32_t icase, float *tau6);

/* sph_eval_boundary: the values that the modified dynamic boundary condition
 * (Sect. 2.6.2) gives the boundary particles of case icase on its current
 * state, without advancing it: rho [n] (Eq 38) and vel [3n] (Eq 39 with the
 * case's mdbc_slip), original particle order; fluid and frozen particles
 * report their state values.  Host buffers, caller-owned, either may be
 * NULL.  SPH_ERR_STATE if no case of the engine uses boundary_mode 1. */
int sph_eval_boundary(sph_engine e, int32_t icase, float *vel, float *rho);
/* sph_get_order: rebuild the neighbour list and return, for case icase, the
 * original ids in device (cell-sorted) order and their cell ids (-1 out). */
int sph_get_order(sph_engine e, int32_t icase, int64_t *ids, int64_t *cells,
                  int64_t *n_inside);

/* sph_pair_stats: per particle (original order) the number of neighbours b
 * with 0 < |r_ab|^2 < (2h)^2 and the sum mod 2^64 of SplitMix64-finalised
 * neighbour ids (an order-independent fingerprint of the pair set). */
int sph_pair_stats(sph_engine e, int32_t icase, int64_t *count, uint64_t *hash);

/* ---- batches -------------------------------------------------------------
 * sph_batch_create: ncases independent cases in one engine: their particles
 * are concatenated and their cell grids laid out at segment offsets of one
 * table, so each stage is one launch over all cases; each case keeps its
 * own dt and t.  Step with sph_step, read with the icase argument. */
int sph_batch_create(const sph_case_params *params, const sph_particles *parts,
                     int32_t ncases, void *stream, sph_alloc_fn alloc,
                     sph_free_fn free_fn, void *alloc_ctx, sph_engine *out);

/* ---- serving pool ----------------------------------------------------------
 * sph_pool_create: an engine with room for max_particles particles, max_cells
 * grid cells and max_cases cases, allocated once.  sph_pool_admit copies a
 * new case in (SPH_ERR_BUSY if it does not fit) and returns its slot; the
 * case runs until its simulated time reaches t_end.  sph_pool_step advances
 * all admitted cases and reports the slots that reached t_end;
 * sph_pool_release frees a slot (its particles leave at the next step). */
int sph_pool_create(int64_t max_particles, int64_t max_cells, int32_t max_cases,
                    void *stream, sph_alloc_fn alloc, sph_free_fn free_fn,
                    void *alloc_ctx, sph_engine *out);
int sph_pool_admit(sph_engine e, const sph_case_params *params,
                   const sph_particles *parts, double t_end, int32_t *slot);
int sph_pool_step(sph_engine e, int64_t nsteps, int32_t *finished,
                  int32_t *n_finished);
int sph_pool_release(sph_engine e, int32_t slot);
int sph_pool_usage(sph_engine e, int64_t *particles_used, int64_t *cells_used,
                   int32_t *cases_used);

/* sph_destroy: release all device memory of the engine. */
void sph_destroy(sph_engine e);

/* ---- roofline denominators ------------------------------------------------
 * sph_probe_peaks: not an operation of the paper.  Measures the FP32 and FP64
 * fused multiply-add throughput of the current device (TFLOP/s, 2 FLOP per
 * FMA): independent FMA chains in every thread of 8 blocks of 256 threads per
 * SM, best of 3 launches timed with CUDA events on `stream` (cudaStream_t,
 * NULL = default) after one untimed launch; about 50 ms in all.  These are the
 * denominators of the interaction kernel's roofline, whose pair loop is bound
 * by FP32 arithmetic.  *sm_count receives the device's SM count.  Any output
 * may be NULL (a NULL TFLOP/s output skips that measurement).  Allocates and
 * frees 16 bytes of device memory; synchronises the stream.  SPH_ERR_CUDA if
 * there is no device or a launch fails. */
int sph_probe_peaks(double *fp32_tflops, double *fp64_tflops, int32_t *sm_count, void *stream);

/* ---- allocation-free cell-key sort ------------------------------------------
 * The paper has no counterpart of this call; it exists for callers that may
 * not let a library allocate device memory (a host program that owns the
 * whole device-memory budget, or a loop that cannot accept the device
 * synchronisation that cudaMalloc/cudaFree may cause).
 *
 * sph_sort_cell_keys_static: stable sort of n 32-bit keys -- the sort the
 * neighbour list uses.  It orders by the low 8 ceil(nbits/8) bits of each key
 * (one pass per 8-bit digit), so every key must be below 2^nbits for the
 * order to be by value; bits from 8 ceil(nbits/8) up are ignored.  keys_in [n]
 * (read), keys_out [n] and perm_out [n] (written; perm_out[i] = index in
 * keys_in of the i-th smallest key, ties in input order) are caller-owned
 * DEVICE pointers that must not overlap (SPH_ERR_ARG otherwise: the passes
 * write one output while other blocks still read the input); work is queued
 * on `stream` (cudaStream_t, NULL = default stream) and the call returns
 * without synchronising.
 * It calls no cudaMalloc/cudaFree: its scratch is one fixed array of
 * 4,457,472 bytes (exactly what n = SPH_SORT_STATIC_MAX_KEYS needs) in the
 * library's device data, present on every GPU that loads the
 * library until the process exits.  n above SPH_SORT_STATIC_MAX_KEYS is
 * rejected with SPH_ERR_ARG.  The first call on a device looks up that
 * array's device address (with that device current); make that first call
 * before any stream capture.  All calls on a device share the one array: two
 * calls whose work overlaps on the GPU (different streams, or different host
 * threads) race and corrupt each other's results; serialise them.  No scratch
 * content carries over between calls. */
#define SPH_SORT_STATIC_MAX_KEYS 524288
int sph_sort_cell_keys_static(const uint32_t *keys_in, uint32_t *keys_out,
                              uint32_t *perm_out, int64_t n, int32_t nbits,
                              void *stream);

#ifdef __cplusplus
}
#endif
#endif
