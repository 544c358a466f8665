/*
 * fmm2d.h -- C ABI of the GB300 (sm_103a) 2D vortex-particle fast multipole
 * library.
 *
 * The library evaluates the velocity induced by N Gaussian-regularised
 * vortex particles at the particles themselves, following Cruz & Barba,
 * "Characterization of the errors of the Fast Multipole Method approximation
 * in particle simulations" (2008):
 *
 *   u_sigma(x_i) = sum_{j != i} Gamma_j K_sigma(x_i - x_j)          (Eq. 7, Eq. 9)
 *   K_sigma(x)   = (-y, x) (1 - exp(-r^2 / 2 sigma^2)) / (2 pi r^2)  (Eq. 6)
 *
 * approximated by the FMM of Sec. 3: a uniform quadtree of depth L (Sec. 3.3),
 * p-term multipole and local expansions of the singular kernel in complex
 * form (Eqs. 16-22), and the regularised kernel summed directly over each
 * leaf's local list -- the leaf and its up to 8 neighbours (Eq. 10,
 * Sec. 3.3.1).
 *
 * Conventions shared by every call
 * --------------------------------
 * - All pointers named *_dev are device pointers; *_host are host pointers.
 *   The caller owns every buffer it passes; the library never frees them.
 * - Positions are interleaved pairs (x0, y0, x1, y1, ...); velocities are
 *   written the same way (u_x, u_y), in the input order of the particles.
 * - The element type follows the plan's precision: double for FMM2D_FP64,
 *   float for FMM2D_FP32 and FMM2D_FP32_TC.
 * - Calls taking a cudaStream_t enqueue work on that stream and return
 *   without synchronising unless stated otherwise.
 * - Nothing crosses the ABI as an exception; every call returns a status.
 *   Errors the device detects while running (a point outside the root box, a
 *   non-finite input) are recorded in the plan and reported by
 *   fmm2d_plan_check() once the stream has reached that point.
 * - A plan is not thread-safe: calls on one plan must not overlap in time,
 *   on the host or on the device.
 */
#ifndef FMM2D_H
#define FMM2D_H

#include <stdint.h>

#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    FMM2D_OK = 0,
    FMM2D_INVALID_ARG = 1,    /* p, L, n, sigma or root box out of range; null pointer */
    FMM2D_OUT_OF_DOMAIN = 2,  /* a particle lies outside the closed root box */
    FMM2D_NONFINITE = 3,      /* a position or circulation is NaN or infinite */
    FMM2D_CUDA_ERROR = 4,     /* a CUDA runtime call failed */
    FMM2D_TIMEOUT = 5,        /* a bounded device-side wait gave up */
    FMM2D_OUT_OF_MEMORY = 6,  /* workspace allocation failed */
    FMM2D_UNSUPPORTED = 7     /* valid request this build does not serve */
} fmm2d_status;

typedef enum {
    FMM2D_FP64 = 0,    /* every step in double precision */
    FMM2D_FP32 = 1,    /* float storage and arithmetic; box-size-scaled expansions */
    FMM2D_FP32_TC = 2  /* as FP32, with M2L as a 3xTF32 tensor-core contraction */
} fmm2d_precision;

typedef struct {
    int p;            /* expansion terms, m = 0 .. p-1 (Eq. 21); 1 <= p <= 32 */
    int L;            /* quadtree depth: leaves are the 4^L boxes of level L; 0 <= L <= 12 */
    double sigma;     /* Gaussian core size of Eq. 3 / Eq. 6; > 0 */
    int precision;    /* fmm2d_precision */
    double x0, y0, W; /* root box [x0, x0 + W] x [y0, y0 + W]; W > 0 */
    int64_t max_n;    /* largest particle count any call on this plan passes */
    double cutoff;    /* the distance a of Sec. 4.1 (Eq. 29): a pair closer than a keeps
                         the regularised kernel of Eq. 6 even when its leaves are not
                         neighbours (the far field's singular contribution is corrected
                         by K_sigma - K' of Eq. 27).  0 = the plain 3x3 rule; at L >= 2
                         at most 2 W / 2^L (one ring of leaves beyond the 3x3 block). */
} fmm2d_params;

typedef struct fmm2d_plan fmm2d_plan;

/* Human-readable name of a status code (static storage, never NULL). */
const char* fmm2d_status_string(fmm2d_status s);

/* Detail of the last error raised on the calling host thread (static or
 * thread-local storage, never NULL; empty when there is none). */
const char* fmm2d_last_error(void);

/* Create a plan: validates the parameters, allocates the device workspace
 * for up to max_n particles on the current device, and builds the
 * translation tables (M2M of Sec. 3.3.2, M2L of Eq. 22, L2L of Sec. 3.3.3)
 * in double precision on the device.  FP32 plans with a cutoff (L >= 2,
 * max_n < 2^30) also hold the near field's ring strips: 64 bytes per
 * particle and 16 per leaf.  Synchronous.  On failure *out is set to NULL and
 * nothing is leaked. */
fmm2d_status fmm2d_plan_create(fmm2d_plan** out, const fmm2d_params* prm);

/* Release the plan and its workspace.  Synchronises the device first.
 * NULL is accepted. */
void fmm2d_plan_destroy(fmm2d_plan* plan);

/* FMM velocity at every particle (Eq. 7 with Eq. 9, by the method of Sec. 3):
 *   xy_dev    n interleaved positions, element type per precision
 *   gamma_dev n circulations
 *   uv_dev    n interleaved velocities (output; must not alias the inputs)
 * 0 <= n <= max_n.  Steps, all on `stream`: Morton keys, stable radix sort
 * and leaf ranges; P2M; M2M for levels L-1..2; M2L at levels 2..L over the
 * interaction lists; L2L for levels 3..L; L2P plus the near-field sum over
 * each leaf's local list.  The sequence is recorded once into a CUDA graph
 * per (buffers, n) and replayed on later calls with the same arguments.
 * Device-detected input errors: see fmm2d_plan_check(). */
fmm2d_status fmm2d_velocity(fmm2d_plan* plan, int64_t n, const void* xy_dev,
                            const void* gamma_dev, void* uv_dev, cudaStream_t stream);

/* Same computation from host buffers: copies the inputs to the device, runs
 * fmm2d_velocity on `stream`, copies the velocities back and synchronises
 * `stream`.  Page-locked host buffers make the copies asynchronous with
 * respect to other streams.  Returns the device-detected status as well. */
fmm2d_status fmm2d_velocity_host(fmm2d_plan* plan, int64_t n, const void* xy_host,
                                 const void* gamma_host, void* uv_host, cudaStream_t stream);

/* count independent particle sets of n particles each, from host buffers,
 * pipelined: set k + 1's inputs are copied to the device (on a copy stream
 * of the plan) while set k is evaluated on `stream`, and set k's velocities
 * are copied back (on a second copy stream) while set k + 1 is evaluated.
 * Each set is evaluated exactly as fmm2d_velocity_host evaluates it, so
 * every set's velocities are the same bit for bit.
 *   xy_host[k], gamma_host[k], uv_host[k]   the host buffers of set k, as in
 *              fmm2d_velocity_host (page-locked, or the copies cannot overlap)
 * Allocates on first use two more staging sets of max_n particles, two
 * streams and eight events, kept until the plan is destroyed, and (without
 * phase timing) records one evaluation graph per staging set for each new n,
 * reading that set's inputs and writing its output set directly.  Returns after
 * the last set's velocities are in host memory, with the device-detected
 * status of all sets (fmm2d_plan_check).  Errors: FMM2D_INVALID_ARG for
 * count < 0, n outside [0, max_n] or a null buffer. */
fmm2d_status fmm2d_velocity_host_many(fmm2d_plan* plan, int count, int64_t n,
                                      const void* const* xy_host,
                                      const void* const* gamma_host, void* const* uv_host,
                                      cudaStream_t stream);

/* One explicit step of the convection part of the vortex method, Eq. 5
 * (dx_i/dt = u(x_i) with u from the FMM of this plan), in place:
 *   order 1  forward Euler, x' = x + dt u(x)                 (one evaluation)
 *   order 2  Heun, x* = x + dt u(x), x' = x + dt (u(x) + u(x*)) / 2   (two)
 *   xy_dev     n interleaved positions in the plan's element type (device,
 *              read and overwritten with the new positions)
 *   gamma_dev  n circulations (device; the viscous part of Eq. 5, which would
 *              change them, is not part of this library)
 * The positions must stay inside the root box: an intermediate position
 * outside it is reported by fmm2d_plan_check, the final ones only by the
 * next evaluation.  Uses the plan's staging buffers (calls on one plan must
 * not overlap).  Asynchronous on `stream`. */
fmm2d_status fmm2d_convect(fmm2d_plan* plan, int64_t n, void* xy_dev, const void* gamma_dev,
                           double dt, int order, cudaStream_t stream);

/* Velocities at m evaluation points that carry no circulation, induced by n
 * particles (the velocity field of Eq. 7 at arbitrary points z; the
 * single-source experiment of Sec. 5.2 evaluates it on a lattice of such
 * points).  The points enter the evaluation as particles of zero
 * circulation: they induce nothing, take part in the tree, the near field
 * and L2P like particles, and a point that coincides with a particle gets
 * K_sigma(0) = 0 from it.
 *   xy_dev, gamma_dev  n particles as in fmm2d_velocity (device)
 *   txy_dev            m interleaved points (x, y) in the plan's element type,
 *                      inside the root box (device)
 *   tuv_dev            2 m velocities (u, v) at the points (device, output)
 * Needs n + m <= max_n; uses the plan's staging buffers (allocated on the
 * first host or target call), so calls on one plan must not overlap.
 * Asynchronous on `stream`; input errors are reported by fmm2d_plan_check. */
fmm2d_status fmm2d_velocity_targets(fmm2d_plan* plan, int64_t n, const void* xy_dev,
                                    const void* gamma_dev, int64_t m, const void* txy_dev,
                                    void* tuv_dev, cudaStream_t stream);

/* Wait for `stream` and report (and clear) any input error the device
 * recorded during earlier calls on this plan. */
fmm2d_status fmm2d_plan_check(fmm2d_plan* plan, cudaStream_t stream);

/* Quadtree of the last fmm2d_velocity call, for bit-exact checks
 * (Sec. 3.3, Fig. 6).  Device outputs, each may be NULL to skip it:
 *   keys_dev        n Morton keys in sorted order (leaf x index in the even
 *                   bits, y index in the odd bits)
 *   perm_dev        n input indices in sorted order (stable: equal keys keep
 *                   input order)
 *   leaf_start_dev  4^L + 1 offsets: leaf k holds sorted positions
 *                   [leaf_start[k], leaf_start[k+1])
 * Enqueued on `stream` after the call it describes. */
fmm2d_status fmm2d_tree_debug(fmm2d_plan* plan, uint32_t* keys_dev, uint32_t* perm_dev,
                              uint32_t* leaf_start_dev, cudaStream_t stream);

/* Reference velocities in double precision at s sampled particles, by direct
 * summation over all n particles (the accuracy yardstick of Sec. 5):
 *   kernel 0  regularised kernel of Eq. 6 for every pair (Eq. 7 with Eq. 9)
 *   kernel 1  the FMM's own limit: Eq. 6 for pairs in each other's 3x3 leaf
 *             neighbourhood at the plan's L and root box and for pairs closer
 *             than the plan's cutoff, the singular kernel of Eq. 27 for the
 *             rest (Eq. 10, Sec. 4.1)
 *   xy_dev, gamma_dev  inputs in the plan's element type
 *   target_idx_dev     s particle indices in [0, n)
 *   uv_ref_dev         2 s doubles (output)
 * Out-of-range indices are skipped and recorded as FMM2D_INVALID_ARG for
 * fmm2d_plan_check(). */
fmm2d_status fmm2d_direct_sampled(fmm2d_plan* plan, int kernel, int64_t n, const void* xy_dev,
                                  const void* gamma_dev, int64_t s, const int64_t* target_idx_dev,
                                  double* uv_ref_dev, cudaStream_t stream);

/* Error statistics of an FMM result against sampled references, in double
 * precision (the normalisation of Sec. 5.1: errors are divided by the
 * maximum reference speed):
 *   uv_dev         n velocities from fmm2d_velocity (plan element type)
 *   target_idx_dev s particle indices; uv_ref_dev the 2 s reference values
 *   stats_dev      4 doubles (output): max_i |du_i|, max_i |u_ref,i|,
 *                  sum_i |du_i|^2, sum_i |u_ref,i|^2  (|.| the 2-norm)
 *   leaf_err_dev   optional (may be NULL): 4^L doubles, the largest |du_i|
 *                  among sampled particles of each leaf (0 where none);
 *                  needs the tree of the last fmm2d_velocity call on the
 *                  same positions.
 * stats_dev and leaf_err_dev are overwritten, not accumulated. */
fmm2d_status fmm2d_error_stats(fmm2d_plan* plan, int64_t n, const void* xy_dev, const void* uv_dev,
                               int64_t s, const int64_t* target_idx_dev, const double* uv_ref_dev,
                               double* stats_dev, double* leaf_err_dev, cudaStream_t stream);

/* Per-phase device timing of fmm2d_velocity (tracing).  The phases of one
 * evaluation, in order: 0 tree build (keys, radix sort, leaf ranges), 1 P2M,
 * 2 M2M, 3 M2L, 4 L2L, 5 L2P plus near field. */
#define FMM2D_NUM_PHASES 6

/* ring > 0: every later fmm2d_velocity call records CUDA events at its phase
 * boundaries (event-record nodes inside the CUDA graph) into the next of
 * `ring` slots, so the last `ring` calls can be read back.  ring = 0 turns
 * timing off.  While timing is on the FP32 forms run their phases one after
 * another (untimed, the far-field phases run beside the near field), so each
 * phase time is the duration of its own kernels.  Synchronises the device;
 * 0 <= ring <= 4096. */
fmm2d_status fmm2d_plan_set_timing(fmm2d_plan* plan, int ring);

/* Phase durations in milliseconds of the call made `age` calls ago (0 = the
 * latest), FMM2D_NUM_PHASES doubles written to ms_host.  Waits for that
 * call's events.  FMM2D_INVALID_ARG when timing is off or the call has left
 * the ring.  In the FP32 forms at L >= 2 the far field (P2M, M2M, M2L, L2L)
 * runs beside the near field: the last phase then spans from the end of the
 * tree to the end of the far part's L2P, and the far-field phases are
 * measured on their own branch. */
fmm2d_status fmm2d_plan_phase_ms(fmm2d_plan* plan, int age, double* ms_host);

/* ------------------------------------------------------------------------
 * Batched evaluation: many independent problems of uneven size, expansion
 * order and depth, like the parameter sweeps of Sec. 5, in one packed
 * evaluation.  FP32 form (float inputs and arithmetic, M2L on CUDA cores).
 * Instance i owns particles [offset_i, offset_i + n_i) of the packed arrays,
 * offset_i = n_0 + ... + n_{i-1}; its velocities are exactly those of a
 * single-instance FMM2D_FP32 plan with the same parameters.
 * ------------------------------------------------------------------------ */
typedef struct {
    int64_t n;        /* particles of this instance (>= 0) */
    int p;            /* expansion terms, 1..32 */
    int L;            /* quadtree depth, 0..12 */
    double sigma;     /* core size, > 0 */
    double x0, y0, W; /* root box, W > 0 */
    double cutoff;    /* the distance a of Sec. 4.1 as in fmm2d_params (0: the plain
                         3x3 rule; at L >= 2 at most 2 W / 2^L) */
} fmm2d_instance;

typedef struct fmm2d_batch_plan fmm2d_batch_plan;

/* Detail of the last batch-call error on the calling host thread. */
const char* fmm2d_batch_last_error(void);

/* Create a batch plan for `count` instances (copied): validates them, packs
 * them (sum of n and sum of 4^L below 2^32), allocates the workspace on the
 * current device and builds the translation tables.  Synchronous. */
fmm2d_status fmm2d_batch_plan_create(fmm2d_batch_plan** out, int count,
                                     const fmm2d_instance* instances);
/* The same with a precision: FMM2D_FP32 (as fmm2d_batch_plan_create: float
 * storage and arithmetic, M2L on the CUDA cores) or FMM2D_FP32_TC (M2L as the
 * 3xTF32 tensor-core contraction of every instance with L >= 2, one launch
 * per class of equal p rounded up to 4).  Every other step is the same in
 * both, and a batched instance gives bit for bit what a single plan of the
 * same precision gives. */
fmm2d_status fmm2d_batch_plan_create_ex(fmm2d_batch_plan** out, int count,
                                        const fmm2d_instance* instances, int precision);
void fmm2d_batch_plan_destroy(fmm2d_batch_plan* plan);

/* Velocities of every instance (packed xy: 2 sum(n) floats, gamma: sum(n),
 * uv: 2 sum(n) floats, device).  The whole batch -- tree build, the upward
 * and downward sweeps of every instance, and the near field as one
 * persistent launch -- is recorded once per (buffers) into a CUDA graph and
 * replayed.  Asynchronous on `stream`; input errors via fmm2d_batch_check. */
fmm2d_status fmm2d_batch_velocity(fmm2d_batch_plan* plan, const float* xy_dev,
                                  const float* gamma_dev, float* uv_dev, cudaStream_t stream);

/* Wait for `stream`; report and clear device-recorded input errors. */
fmm2d_status fmm2d_batch_check(fmm2d_batch_plan* plan, cudaStream_t stream);

/* Autotuner: times candidate launch shapes of the two heaviest steps on the
 * given batch (persistent near-field CTAs per SM in {2..6}; for FP32_TC
 * batches the tensor-core M2L's operator stages in flight, 2, 3, 4 or as many
 * as shared memory holds, and its tile policy, the fewest tiles per level or
 * the widest rows; for FP32 batches the CUDA-core M2L block size in
 * {64, 128, 256}), keeps the fastest and leaves uv_dev holding the
 * velocities.  Synchronous; later fmm2d_batch_velocity calls use the
 * choices. */
fmm2d_status fmm2d_batch_autotune(fmm2d_batch_plan* plan, const float* xy_dev,
                                  const float* gamma_dev, float* uv_dev, cudaStream_t stream);

/* FP64 direct sums at s sampled particles (global packed indices), each
 * over its own instance only; kernel 0/1 as in fmm2d_direct_sampled. */
fmm2d_status fmm2d_batch_direct_sampled(fmm2d_batch_plan* plan, int kernel, const float* xy_dev,
                                        const float* gamma_dev, int64_t s,
                                        const int64_t* target_idx_dev, double* uv_ref_dev,
                                        cudaStream_t stream);

/* Error statistics per instance (4 doubles each, as in fmm2d_error_stats)
 * and, when leaf_err_dev is not NULL, the max |du| of sampled particles per
 * leaf in the global leaf order (instance i's leaves follow instance i-1's,
 * 4^L_i of them, in Morton order). */
fmm2d_status fmm2d_batch_error_stats(fmm2d_batch_plan* plan, const float* xy_dev,
                                     const float* uv_dev, int64_t s,
                                     const int64_t* target_idx_dev, const double* uv_ref_dev,
                                     double* stats_dev, double* leaf_err_dev, cudaStream_t stream);

/* Sizes and chosen launch shapes (each output may be NULL): total particles,
 * total leaves, kernel launches per fmm2d_batch_velocity call (after the
 * first), persistent near-field CTAs per SM, M2L block size. */
fmm2d_status fmm2d_batch_info(const fmm2d_batch_plan* plan, int64_t* n_total,
                              int64_t* leaves_total, int* kernels_per_call, int* p2p_ctas_per_sm,
                              int* m2l_threads);

/* Tracing: one evaluation of the batch, its steps launched one after another
 * on the plan's stream with CUDA events between them (not the recorded
 * graph), then the durations in ms (5 doubles): tree build, P2M and M2M, M2L,
 * L2L, near field with L2P.  Synchronous; uv_dev receives the velocities. */
fmm2d_status fmm2d_batch_profile(fmm2d_batch_plan* plan, const float* xy_dev,
                                 const float* gamma_dev, float* uv_dev, double* ms_host,
                                 cudaStream_t stream);

/* FP32_TC batches: tensor-core M2L classes (one per p rounded up to 4),
 * their tiles in all, the operator stages in flight (of the first class)
 * and the tile policy the autotuner chose (0: fewest tiles per level, 1:
 * widest rows).  Each output may be NULL; zeros for FP32 batches. */
fmm2d_status fmm2d_batch_info_tc(const fmm2d_batch_plan* plan, int* classes, int* tiles,
                                 int* b_stages, int* tile_policy);

/* Quadtree of the last batch evaluation in the global leaf order (keys are
 * leaf_base_i + Morton key): as fmm2d_tree_debug, leaf_start has
 * sum(4^L) + 1 entries. */
fmm2d_status fmm2d_batch_tree_debug(fmm2d_batch_plan* plan, uint32_t* keys_dev, uint32_t* perm_dev,
                                    uint32_t* leaf_start_dev, cudaStream_t stream);

/* Quadtree build that allocates nothing.  The paper has no counterpart: this
 * entry point exists for callers that cannot allocate device memory -- for
 * example a host framework whose memory manager owns the whole device budget
 * and forbids allocations behind its back, or a latency-critical loop in
 * which cudaMalloc / cudaFree, which can synchronise the whole device, are
 * not acceptable.  It computes exactly what fmm2d_velocity's first step
 * computes (Morton keys, stable radix sort, leaf ranges; the outputs match
 * fmm2d_tree_debug bit for bit) without a plan:
 *   precision          FMM2D_FP64 (double inputs) or FMM2D_FP32 / FMM2D_FP32_TC (float)
 *   xy_dev, gamma_dev  n interleaved positions and n circulations (device)
 *   L, x0, y0, W       leaf level (0..12) and the root box
 *   keys_dev, perm_dev n sorted keys and n input indices (device, caller-owned)
 *   leaf_start_dev     4^L + 1 leaf offsets (device, caller-owned)
 *   flags_dev          optional device int: overwritten with the input-error
 *                      flags (bit 1 << FMM2D_OUT_OF_DOMAIN, 1 << FMM2D_NONFINITE)
 * Limit: n <= 262144 (2^18); larger n returns FMM2D_INVALID_ARG before any
 * work is enqueued.  Its scratch (key/value ping-pong buffers, digit counts,
 * a status word; about 4.3 MB) is one fixed device array inside the
 * library, held by every GPU that loads the library until the process exits.
 * The call makes no cudaMalloc, cudaFree or other allocating call.
 * The first call on a device looks up that array's device address (once per
 * device, with the device current; again only if that device's context was
 * destroyed and created anew, e.g. by cudaDeviceReset); make that first call
 * before any stream capture.  All calls share the one array and it keeps the last call's
 * contents (the status word is cleared at the start of each call): calls
 * whose work overlaps on the GPU -- on different streams, or from different
 * host threads -- race on it and must be serialised by the caller. */
fmm2d_status fmm2d_tree_build_noalloc(int precision, int64_t n, const void* xy_dev,
                                      const void* gamma_dev, int L, double x0, double y0,
                                      double W, uint32_t* keys_dev, uint32_t* perm_dev,
                                      uint32_t* leaf_start_dev, int* flags_dev,
                                      cudaStream_t stream);

/* ------------------------------------------------------------------------
 * Learned (p, L) proposer.
 *
 * Sec. 5 measures how the FMM error moves with the expansion order p and the
 * tree depth l, and Sec. 4.1 (Eqs. 26-29) shows that a leaf too small
 * against the core size sigma puts a floor under it that no p removes.  The
 * proposer learns that error surface from the library's own measurements --
 * FMM velocities against the FP64 direct sum at sampled particles -- and
 * picks the cheapest (p, L) whose predicted maximum error meets a
 * tolerance, falling back to a conservative fixed setting when no candidate
 * qualifies.  The paper tunes (p, l) by hand; the network is not in it.
 *
 * Network: FMM2D_MLP_INPUTS -> 128 -> 128 -> 128 -> FMM2D_MLP_OUTPUTS,
 * SiLU between layers, weights stored in BF16 (rounded to nearest even from
 * FP32 master copies), biases, activations and every accumulation in FP32.
 * Inputs are standardised and outputs de-standardised with constants the
 * caller sets.  Outputs: (log10 of the median over sampled leaves of the
 * per-leaf max error, log10 of the max error), both relative to max |u|.
 *
 * Master parameter layout (FMM2D_MLP_PARAMS floats): for layers l = 0..3,
 * W_l as [out][in] row-major, then b_l [out].
 *
 * Features (fmm2d_features), for a particle set and a candidate (p, L):
 *   0 p                       6 max / mean particles per leaf
 *   1 L                       7 sum_b |S_b| / sum_i |Gamma_i|
 *   2 sigma / h, h = W/sqrt(n) 8 std_b(S_b) / A
 *   3 log2 n                  9 max_b |S_b| / A
 *   4 log2 mean per leaf     10 sum Gamma / sum |Gamma|
 *   5 std / mean per leaf    11 log10(leaf width / sigma)
 * where S_b is the circulation sum of leaf b at depth L and
 * A = sum |Gamma| / 4^L.  Circulations enter only as ratios: the relative
 * error does not change when every Gamma is scaled.
 * ------------------------------------------------------------------------ */
#define FMM2D_MLP_INPUTS 12
#define FMM2D_MLP_OUTPUTS 2
#define FMM2D_MLP_PARAMS 34946

typedef struct fmm2d_mlp fmm2d_mlp;

/* Detail of the last proposer-call error on the calling host thread. */
const char* fmm2d_mlp_last_error(void);

/* Create a network for batches of up to max_rows rows (1 .. 2^20) on the
 * current device; weights uniform in +-1/sqrt(fan_in) from a splitmix64
 * stream seeded with `seed`, biases zero, identity normalisation, Adam
 * moments zero.  Synchronous. */
fmm2d_status fmm2d_mlp_create(fmm2d_mlp** out, int max_rows, uint64_t seed);
void fmm2d_mlp_destroy(fmm2d_mlp* net);

/* Standardisation constants (host arrays of 12, 12, 2, 2 floats; every std
 * > 0): the network sees (x - in_mean) / in_std, and its raw output y is
 * reported as y * out_std + out_mean.  Training targets are standardised
 * the same way.  Synchronous. */
fmm2d_status fmm2d_mlp_set_normalization(fmm2d_mlp* net, const float* in_mean,
                                         const float* in_std, const float* out_mean,
                                         const float* out_std);

/* Read (get_host != NULL) and/or replace (set_host != NULL) the FP32 master
 * parameters, FMM2D_MLP_PARAMS floats in the layout above; replacing also
 * re-rounds the BF16 copies.  Adam moments are kept.  Synchronous. */
fmm2d_status fmm2d_mlp_params(fmm2d_mlp* net, float* get_host, const float* set_host);

/* y_dev[rows][2] = network(x_dev[rows][12]) in de-standardised units (device
 * buffers, rows <= max_rows).  Asynchronous on `stream`. */
fmm2d_status fmm2d_mlp_forward(fmm2d_mlp* net, int rows, const float* x_dev, float* y_dev,
                               cudaStream_t stream);

/* Gradient of the mean squared error between the standardised output and
 * the standardised targets t_dev[rows][2], mean over rows x outputs, with
 * respect to the master parameters (computed through the BF16 weights):
 * grad_dev receives FMM2D_MLP_PARAMS floats, loss_dev (optional) the loss.
 * Asynchronous on `stream`. */
fmm2d_status fmm2d_mlp_gradients(fmm2d_mlp* net, int rows, const float* x_dev,
                                 const float* t_dev, float* grad_dev, float* loss_dev,
                                 cudaStream_t stream);

/* One Adam step (Kingma & Ba 2015; beta1 0.9, beta2 0.999, eps 1e-8, bias
 * correction by the step count) on that gradient at learning rate lr > 0;
 * loss_dev (optional) receives the loss before the step.  Asynchronous. */
fmm2d_status fmm2d_mlp_train_step(fmm2d_mlp* net, int rows, const float* x_dev,
                                  const float* t_dev, float lr, float* loss_dev,
                                  cudaStream_t stream);

/* The 12 features above for n >= 1 particles (float xy_dev, gamma_dev on the
 * device) with core size sigma, root box (x0, y0, W), candidate p >= 1 and
 * depth L (0..10); particles outside the box count in the nearest edge
 * leaf.  Allocates stream-ordered scratch (16 * 4^L bytes), synchronises
 * `stream` and writes feat_host[12]. */
fmm2d_status fmm2d_features(int64_t n, const float* xy_dev, const float* gamma_dev,
                            double sigma, double x0, double y0, double W, int p, int L,
                            float* feat_host, cudaStream_t stream);

/* Pick the cheapest candidate whose predicted log10 max error is at most
 * log10(tol) - margin.  features_host holds ncand rows of 12 features whose
 * first two entries are the candidate's integral p (1..32) and L (0..12);
 * cost_host its cost (any unit, smaller is better).  *p_out, *L_out receive
 * the choice, or (fallback_p, fallback_L) when no candidate qualifies or
 * ncand == 0; *choice_out (optional) the chosen row or -1;
 * predicted_host (optional) 2 * ncand predicted outputs.  Synchronous, on
 * the legacy default stream. */
fmm2d_status fmm2d_propose(fmm2d_mlp* net, int ncand, const float* features_host,
                           const double* cost_host, double tol, double margin, int fallback_p,
                           int fallback_L, int* p_out, int* L_out, int* choice_out,
                           float* predicted_host);

/* Number of kernel launches one fmm2d_velocity call makes (the kernel nodes
 * of its recorded CUDA graph); -1 before the first call. */
int fmm2d_plan_kernels_per_call(const fmm2d_plan* plan);

/* A split of one evaluation over several devices (Sec. 3.3: the leaves in
 * Morton order cut into contiguous key ranges, one per device).  The
 * multipole expansion of Eq. 20 is linear in the particles, so each device
 * forms the multipoles of its own particles, the devices add up the partial
 * expansions of the boxes in each other's interaction lists (Eq. 22, Sec.
 * 3.3.1), and each device then evaluates its own particles together with
 * the halo particles of the neighbouring leaves (Eq. 10) from the summed
 * multipoles.  The caller moves the data (peer copies or NCCL).
 *
 * Length, in reals of the plan's element type, of its multipole array:
 * boxes of levels 2..L one level after another, each level four parity
 * planes (ix & 1, iy & 1) of a row-major (2^(level-1))^2 grid of boxes,
 * 2P reals per box (P = 16 when p <= 16, else 32; coefficient k as (re, im)
 * at reals 2k, 2k+1, scaled by the box width: a~_k = a_k / s^k; zero beyond
 * p).  0 when L < 2. */
int64_t fmm2d_plan_multipole_reals(const fmm2d_plan* plan);

/* Tree build, P2M (Eq. 20) and M2M (Sec. 3.3.2) of n particles; the
 * multipoles of every box are written to me_dev (device,
 * fmm2d_plan_multipole_reals reals, caller-owned).  Launched on `stream`
 * directly (no graph); input errors as for fmm2d_velocity. */
fmm2d_status fmm2d_multipoles(fmm2d_plan* plan, int64_t n, const void* xy_dev,
                              const void* gamma_dev, void* me_dev, cudaStream_t stream);

/* The rest of one evaluation from given multipoles: tree build of the n
 * particles, M2L (Eq. 22) and L2L (Sec. 3.3.3) from me_dev (read, not
 * changed), then the near field over the n particles and L2P (Eqs. 10, 12),
 * velocities of all n particles to uv_dev in input order.  In a split,
 * the n particles are the device's own followed by its halo particles
 * (sources only: their velocities lack parts and are to be discarded), and
 * me_dev the summed multipoles.  Launched on `stream` directly (no graph). */
fmm2d_status fmm2d_velocity_from_multipoles(fmm2d_plan* plan, int64_t n, const void* xy_dev,
                                            const void* gamma_dev, const void* me_dev,
                                            void* uv_dev, cudaStream_t stream);

/* Failure detection (no counterpart in the paper): every wait of the
 * tensor-core M2L (FMM2D_FP32_TC) on a pipeline barrier polls at most
 * `polls` times (each poll suspends the waiting thread for about 32 ns);
 * when one runs out the kernel stops, records FMM2D_TIMEOUT (reported by
 * fmm2d_plan_check), waits for the copies and MMAs it already issued with
 * the default limit, frees its tensor memory and returns, leaving the
 * affected local expansions unwritten.  polls = 0 restores the default
 * (2^26 polls, about two seconds: never reached by a healthy run).  A small
 * limit exists to test this path without hanging or faulting the GPU.  The
 * next fmm2d_velocity call records its graph anew. */
fmm2d_status fmm2d_plan_set_spin_limit(fmm2d_plan* plan, uint32_t polls);

/* Where the FP32 near field of a plan with a cutoff (Sec. 4.1) gathers the
 * sources of its ring (the leaves two leaves away) from.  enable != 0 (the
 * default): from per-side strips of those leaves, built each evaluation
 * (the sources within reach of the leaf on that side, about a third of the
 * leaf at a = 1.3 leaf widths), while a strip is at most half a leaf wide
 * (a <= 1.5 leaf widths); 0, or a wider cutoff: from the whole leaves.  Both keep the
 * same sources in the same order, so the velocities agree bit for bit while
 * a leaf's ring sources fit one shared-memory chunk (558 records).  Plans
 * without a cutoff, FP64 plans and L < 2 ignore it.  The next fmm2d_velocity
 * call records its graph anew.  Errors: FMM2D_INVALID_ARG for a null plan. */
fmm2d_status fmm2d_plan_set_ring_strips(fmm2d_plan* plan, int enable);

#ifdef __cplusplus
}
#endif

#endif /* FMM2D_H */
