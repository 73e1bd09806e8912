/*
 * pm.h -- C ABI of the GB300 (sm_103a) library for confidence-aware human
 * prediction: the Bayesian belief update over (rationality beta, goal g), the
 * particle rollout of Algorithm 1 and the per-step occupancy histogram of
 * Lu, Bui, Lyu and Chen, "Fast Confidence-Aware Human Prediction via
 * Hardware-accelerated Bayesian Inference for Safe Robot Navigation".
 *
 * Conventions for every call
 *   - Plain pointers and sizes only. Unless stated otherwise a pointer is a
 *     DEVICE pointer on the context's device, owned by the caller, and must
 *     stay valid until the work queued on `stream` has finished.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream). Calls are stream-ordered and asynchronous unless stated.
 *   - Every call returns a pm_status and never throws. Invalid sizes and
 *     arguments are rejected with PM_EINVAL before anything is queued; the
 *     message of the last failure on the calling thread is pm_last_error().
 *   - There is no CPU fallback: every numeric step runs in this library's
 *     CUDA kernels.
 *   - Floats are IEEE binary32; log-beliefs are natural logarithms.
 *
 * Model (Sec. III-A, running example, and the readings of the open points):
 *   state z = (x, y); controls are K headings theta_k = 2*pi*k/K
 *   (counter-clockwise from +x) at one speed v; one step moves v*dt along the
 *   heading (Eq. 1, forward Euler). The state-control value is
 *     Q(z, theta; g) = -w1*v*dt - w2*|| z + v*dt*(cos theta, sin theta) - g ||
 *   and the policy is the Boltzmann distribution pi(k | z; beta, g)
 *   proportional to exp(beta * Q) (Eq. 2). The joint belief over
 *   (beta, g) is a table of G*B log-probabilities indexed j = g*B + b.
 */
#ifndef PM_H_
#define PM_H_

#include <stddef.h>
#include <stdint.h>

#include "pm_limits.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef enum pm_status {
    PM_OK = 0,
    PM_EINVAL = 1,  /* invalid argument; nothing was queued                 */
    PM_ENOMEM = 2,  /* a device or pinned allocation of the context failed */
    PM_ECUDA = 3,   /* a CUDA runtime call or launch failed                */
    PM_EDEVICE = 5  /* a kernel reported an error in its status word       */
} pm_status;

/* Opaque context: one device, its properties, scratch buffers and tuned
 * launch parameters. Not thread-safe; use one context per host thread. */
typedef struct pm_ctx pm_ctx;

/* Human model. `goals` and `beta` are device pointers ([G][2] and [B]).
 * `heading_off` bit k set disables heading k (Q = -inf, so pi = 0), the
 * control masking of Sec. IV-B. The beta values (device memory, so not
 * checked on the host) may be any finite numbers: beta > 0 is the goal-seeking
 * Boltzmann policy of Eq. 2, beta = 0 the uniform policy over the enabled
 * controls, and beta < 0 a policy whose most probable heading is the one
 * farthest from the goal. The predictions latch a non-finite beta or goal
 * in the context's status word (pm_sync_status then returns PM_EDEVICE).
 *
 * Controls: with n_speeds = 0 (or 1 with speed_mult[0] = 1) the K headings at
 * the one speed v. With n_speeds = S in [1, PM_MAX_SPEEDS], the S*K controls
 * u = s*K + k move v*speed_mult[s]*dt along theta_k, with
 * Q_u = -w1*v*speed_mult[s]*dt - w2*||z + v*speed_mult[s]*dt*e_k - g||, and
 * `speed_off` bit s disables speed s (the stationary masking of Sec. IV-B:
 * the high-speed controls of a human seen standing still). Several speeds
 * need K a multiple of 4 with no heading disabled, S*K <= 256, and
 * multipliers > 0; the observed control of a displacement is its continuous
 * heading at the enabled speed whose multiplier is nearest to its length /
 * (v*dt). Traced heading indices are control indices u.
 *
 * `snap_heading` = 1 reads the heading of an observed displacement as the
 * enabled heading theta_k nearest to it (largest e_k . dz, the lower index on
 * a tie), so the belief update and the log-likelihood evaluate the discrete
 * control's Q; 0 (the default) keeps the continuous heading. The nearest
 * heading is decided in FP32. */
typedef struct pm_model {
    int32_t K;
    float speed; /* v  [m/s]            */
    float dt;    /* Delta t [s]         */
    float w1;    /* Q weight of -v*dt   */
    float w2;    /* Q weight of distance */
    int32_t G;
    int32_t B;
    const float *goals;
    const float *beta;
    uint64_t heading_off;
    int32_t n_speeds;                 /* 0: one speed, multiplier 1      */
    float speed_mult[PM_MAX_SPEEDS];  /* speed s is v * speed_mult[s]    */
    uint32_t speed_off;               /* bit s set: speed s disabled     */
    int32_t snap_heading;             /* 0 or 1, see above               */
} pm_model;

/* Occupancy grid: cell (cx, cy) covers [x0 + cx*res, x0 + (cx+1)*res) x
 * [y0 + cy*res, y0 + (cy+1)*res), 0 <= cx < W, 0 <= cy < H. A state is binned
 * with FP32 operations: cx = floor((x - x0) * inv_res), inv_res = 1.0f/res.
 * W and H are at most 2^22 (PM_EINVAL otherwise), and a state more than 2^22
 * cells from (x0, y0) along either axis counts as outside every grid (this
 * also bounds the windows of the batched form: a centred window is useful
 * only for humans within 2^22 cells of the origin, e.g. 209 km at 5 cm). */
typedef struct pm_grid {
    float x0;
    float y0;
    float res;
    int32_t W;
    int32_t H;
} pm_grid;

/* ---- context ------------------------------------------------------------ */

/* Create a context on CUDA device `device`. Allocates nothing on the device
 * until a call needs scratch. */
pm_status pm_create(pm_ctx **ctx, int device);

/* Release the context and the device and page-locked memory it owns, after
 * waiting for the context's copy stream and the uploads of its host-buffer
 * calls. Work the caller queued on its own streams with this context must
 * have finished (synchronise those streams first). NULL is accepted. */
void pm_destroy(pm_ctx *ctx);

/* Message of the last failed call on the calling thread ("" if none). */
const char *pm_last_error(void);

/* Library version string. */
const char *pm_version(void);

/* Wait for the work queued on `stream` (NULL: the legacy default stream) and
 * report the errors that kernels of this context latched in its device status
 * word since the last call, then clear the word. Kernels latch, and carry on
 * past, inputs they cannot use: a non-finite goal or beta (the results of that
 * human are meaningless), a log-belief that is NaN, +inf or -inf everywhere, an
 * observed state or a trajectory point that is not finite (its steps are
 * skipped). Returns PM_OK, PM_EDEVICE with pm_last_error() naming what was
 * latched, or PM_ECUDA. Synchronous. */
pm_status pm_sync_status(pm_ctx *ctx, void *stream);

/* Launch an instantiated CUDA graph (a cudaGraphExec_t, e.g. a captured
 * serving frame) on `stream` and, when `done` (a cudaEvent_t) is not NULL,
 * record it on the stream after the graph; with `wait` != 0 also wait for
 * that event (for the stream when `done` is NULL) before returning: one
 * native call per frame, so a frame loop pays no framework overhead. The
 * caller owns the graph and the event. PM_EINVAL for a NULL graph, PM_ECUDA
 * if the launch, the record or the wait fails. */
pm_status pm_graph_launch(void *graph_exec, void *stream, void *done, int32_t wait);

/* ---- the hot path -------------------------------------------------------- */

/* Bayesian update of the joint belief (Eq. 3), in log space (Eq. 7), over
 * `n_obs` observed steps.
 *   obs_xy      [n_obs+1][2] observed states z_t (device, FP32).
 *   log_belief  [G*B] in/out (device): a normalised log-belief before the
 *               call; the posterior after all n_obs steps on return.
 * The control of step t is recovered from (z_t, z_{t+1}) by differential
 * flatness: the heading of the displacement; Q is evaluated at that
 * continuous heading and normalised over the K headings. A displacement
 * shorter than 1e-6 m leaves the belief unchanged for that step. n_obs = 0
 * is a no-op. The per-step log-likelihoods are accumulated in double-float
 * (pairs of FP32) on the device and the LogSumExp normalisation is applied
 * once, which equals the sequential form of Eq. 7 exactly in real
 * arithmetic. */
pm_status pm_update_posterior(pm_ctx *ctx, const pm_model *model, const float *obs_xy,
                              int32_t n_obs, float *log_belief, void *stream);

/* The same update out of place: the prior is read from `log_prior` [G*B]
 * (device, normalised, left unchanged) and the posterior is written to
 * `log_belief` [G*B] (device). The two are either the same buffer (then this
 * is pm_update_posterior) or disjoint; a partial overlap is PM_EINVAL. With
 * n_obs = 0 the prior is copied. A caller that keeps its prior, or runs the
 * same update repeatedly, needs no copy of its own. */
pm_status pm_update_posterior_into(pm_ctx *ctx, const pm_model *model, const float *obs_xy,
                                   int32_t n_obs, const float *log_prior, float *log_belief,
                                   void *stream);

/* Algorithm 1 with the bootstrapped belief (Sec. III-B): `n_particles`
 * particles start at (z0x, z0y), each draws (beta, g) once from
 * exp(log_belief), then for t = 1..horizon samples a heading from
 * pi(. | z_t; beta, g) at its own state and takes one Euler step; the
 * states of step t are emplaced onto the grid.
 *   log_belief  [G*B] (device), normalised.
 *   counts      [horizon][H][W] uint32 (device), zeroed by the callee, then
 *               counts[t-1][cy][cx] = particles in cell (cx, cy) after step t.
 *   oob         [horizon] uint32 (device), zeroed by the callee: particles
 *               outside the grid after step t (they stay alive).
 * Invariant: sum(counts[t-1]) + oob[t-1] = n_particles. Occupancy
 * probability = count / n_particles.
 * Random numbers: Philox4x64-10 with key (seed, human_id) and counter
 * (particle, block, purpose, 0); the (beta, g) draw of particle i uses word 0
 * of block 0 of purpose 1; the heading draw of step t uses 32-bit word
 * (t-1)&7 of block (t-1)>>3 of purpose 2 (word w is bits 32*(w&1).. of
 * 64-bit output w>>1); u = (word >> 8) * 2^-24. Sampling takes the smallest
 * index k whose running weight sum C_k exceeds u * (total). */
pm_status pm_predict_occupancy(pm_ctx *ctx, const pm_model *model, const float *log_belief,
                               float z0x, float z0y, int32_t n_particles, int32_t horizon,
                               const pm_grid *grid, uint64_t seed, uint32_t human_id,
                               uint32_t *counts, uint32_t *oob, void *stream);

/* The two halves of pm_predict_occupancy, for a caller that overlaps the
 * zeroing with other work: pm_zero_occupancy zeroes counts [horizon][H][W]
 * and oob [horizon] (it touches no scratch of the context, so it may run on
 * a second stream beside the context's other calls, e.g. the belief update);
 * pm_rollout_occupancy is pm_predict_occupancy without the zeroing: it adds
 * to counts and oob, which must have been zeroed since their last rollout
 * (stream order or an event). Arguments, layout and errors as for
 * pm_predict_occupancy (pm_zero_occupancy checks horizon, grid and the two
 * pointers). Asynchronous. */
pm_status pm_zero_occupancy(pm_ctx *ctx, int32_t horizon, const pm_grid *grid, uint32_t *counts, uint32_t *oob,
                            void *stream);
pm_status pm_rollout_occupancy(pm_ctx *ctx, const pm_model *model, const float *log_belief, float z0x, float z0y,
                               int32_t n_particles, int32_t horizon, const pm_grid *grid, uint64_t seed,
                               uint32_t human_id, uint32_t *counts, uint32_t *oob, void *stream);

/* The same launch as pm_predict_occupancy, also recording the trajectories
 * of particles [0, n_trace):
 *   states      [n_trace][horizon][2] FP32 state after each step, or NULL;
 *               8-byte aligned (each state is stored as one pair), else PM_EINVAL
 *   headings    [n_trace][horizon] uint8 heading index of each step, or NULL
 *   components  [n_trace] int32 drawn component j, or NULL
 * `counts`/`oob` may both be NULL to skip the histogram (then `grid` may be
 * NULL too). n_trace <= n_particles. Used for parity checks and to draw
 * synthetic observed trajectories from the model. */
pm_status pm_predict_occupancy_traced(pm_ctx *ctx, const pm_model *model,
                                      const float *log_belief, float z0x, float z0y,
                                      int32_t n_particles, int32_t horizon, const pm_grid *grid,
                                      uint64_t seed, uint32_t human_id, uint32_t *counts,
                                      uint32_t *oob, int32_t n_trace, float *states,
                                      uint8_t *headings, int32_t *components, void *stream);

/* Convenience form with HOST buffers (what a robot-side caller holds):
 * copies the model tables, observations and prior in, runs
 * pm_update_posterior and pm_predict_occupancy on the context's own device
 * buffers, copies the posterior and the histogram out, and returns when they
 * are on the host. Host pointers: goals [G][2], beta [B], obs_xy
 * [n_obs+1][2], log_prior [G*B], posterior_out [G*B], counts_out
 * [horizon][H][W], oob_out [horizon]. The model's goals/beta fields are
 * ignored. The inputs are read during the call (into page-locked staging of
 * the context, uploaded in one copy), so they may be pageable and are free on
 * return; page-locked output buffers make the copies out asynchronous. The
 * rollout starts at the last observed state. */
pm_status pm_predict_host(pm_ctx *ctx, const pm_model *model, const float *goals,
                          const float *beta, const float *obs_xy, int32_t n_obs,
                          const float *log_prior, int32_t n_particles, int32_t horizon,
                          const pm_grid *grid, uint64_t seed, uint32_t human_id,
                          float *posterior_out, uint32_t *counts_out, uint32_t *oob_out,
                          void *stream);

/* The same prediction without waiting, for a caller that issues one
 * prediction after another: the inputs are copied in and the prediction runs
 * on `stream` in one of two device staging slots of the context (alternating
 * per call), and the posterior and histogram are copied out on a copy stream
 * of the context, so that a call's copy-out overlaps the next call's
 * prediction. The outputs of a call are complete once pm_host_fence has made
 * a stream wait for the pending copies and that stream has been synchronised.
 * The output buffers must stay valid, and must not be reused by the caller,
 * until then; the inputs are read during the call and are free on return.
 * A call may wait on the host for the upload of the call before the previous
 * one (its staging is reused). Output buffers as pm_predict_host
 * (page-locked: pageable ones make the copies synchronous). */
pm_status pm_predict_host_async(pm_ctx *ctx, const pm_model *model, const float *goals,
                                const float *beta, const float *obs_xy, int32_t n_obs,
                                const float *log_prior, int32_t n_particles, int32_t horizon,
                                const pm_grid *grid, uint64_t seed, uint32_t human_id,
                                float *posterior_out, uint32_t *counts_out, uint32_t *oob_out,
                                void *stream);

/* Make `stream` wait for every copy-out that pm_predict_host_async has queued
 * on this context (no host wait). */
pm_status pm_host_fence(pm_ctx *ctx, void *stream);

/* ---- many humans in one launch -------------------------------------------- */

/* One human of a batch. Device pointers unless stated.
 *   goals [G][2], beta [B]      the human's goals and rationality grid
 *   obs_xy [n_obs+1][2], n_obs  observed states for pm_batch_update_posterior
 *                               (n_obs = 0: no update for this human)
 *   log_belief [G*B]            in/out belief (read by pm_batch_predict)
 *   z0_xy [2]                   start state of the rollout, read on the device
 *                               at every pm_batch_predict (e.g. the last
 *                               observed state, updated in place between runs)
 *   n_particles, horizon        N and T
 *   grid                        binning grid (x0, y0, res) and output size W x H
 *   center                      1: the W x H output is the window of grid cells
 *                               centred on z0's cell (W, H odd), recomputed on
 *                               the device at every run; 0: output cell =
 *                               grid cell - (cx_off, cy_off)
 *   seed, human_id              Philox key (as pm_predict_occupancy)
 *   counts [horizon][H][W], oob [horizon]  outputs, zeroed by pm_batch_predict;
 *                               states outside the output count in oob.
 *   speed_off                   bit s: speed s disabled for this human on top
 *                               of the shared model's speed_off (a human seen
 *                               standing still keeps only the slow controls,
 *                               Sec. IV-B); 0 unless the shared model has
 *                               several speeds, and at least one speed must
 *                               stay enabled (else PM_EINVAL). */
typedef struct pm_human {
    const float *goals;
    const float *beta;
    int32_t G;
    int32_t B;
    const float *obs_xy;
    int32_t n_obs;
    float *log_belief;
    const float *z0_xy;
    int32_t n_particles;
    int32_t horizon;
    pm_grid grid;
    int32_t center;
    int32_t cx_off;
    int32_t cy_off;
    uint64_t seed;
    uint32_t human_id;
    uint32_t *counts;
    uint32_t *oob;
    uint32_t speed_off;
} pm_human;

/* Opaque batch plan: device descriptors, the tile work list, scratch for the
 * batched belief update and the tuned launch shape. */
typedef struct pm_batch pm_batch;

/* Create a plan for up to max_humans humans sharing the model fields K,
 * speed, dt, w1, w2 and heading_off of `shared` (its goals/beta/G/B are
 * ignored). Allocates the plan's device and page-locked host buffers. */
pm_status pm_batch_create(pm_ctx *ctx, const pm_model *shared, int32_t max_humans, pm_batch **out);

/* Set the batch contents (host array of n_humans descriptors, copied):
 * validates them, builds the work list of tiles sorted by horizon (longest
 * first) and queues the upload on `stream`. A CUDA graph that captured
 * pm_batch_update_posterior / pm_batch_predict reads the descriptors, the
 * tile list and the counts from device memory and stays valid across calls
 * to pm_batch_set while the tile list fits the capacity reached before the
 * capture (max_humans * 2048 tiles at creation; a larger batch reallocates
 * the list, after which the graph must be captured again). */
pm_status pm_batch_set(pm_batch *b, const pm_human *humans, int32_t n_humans, void *stream);

/* Belief update (Eq. 3 / Eq. 7) of every human with n_obs > 0, one launch. */
pm_status pm_batch_update_posterior(pm_batch *b, void *stream);

/* Zero the outputs (every cell, or the reachable ones: pm_batch_set_zeroing),
 * then one persistent launch of Algorithm 1 over all tiles of all humans.
 * Each human's counts equal those of pm_predict_occupancy with the same
 * inputs (bit-identical). Enqueues only a memset and two kernels: it may be
 * captured in a CUDA graph. */
pm_status pm_batch_predict(pm_batch *b, void *stream);

/* The two halves of pm_batch_predict, for a caller that overlaps the zeroing
 * with other work (e.g. on a second stream, beside pm_batch_update_posterior,
 * joined before the rollout): pm_batch_zero enqueues the zeroing of the
 * outputs (by the mode of pm_batch_set_zeroing), pm_batch_rollout the
 * persistent launch of Algorithm 1. pm_batch_rollout adds to the counts: the
 * outputs must have been zeroed by pm_batch_zero after the previous
 * prediction and before it (stream order or an event). Both may be captured
 * in a CUDA graph. */
pm_status pm_batch_zero(pm_batch *b, void *stream);
pm_status pm_batch_rollout(pm_batch *b, void *stream);

/* reach = 0 (the default): pm_batch_predict zeroes every cell of every
 * human's counts before the rollout. reach = 1: it zeroes only the cells of
 * step t that a particle can occupy after t steps of the longest control,
 * from this prediction's start or from the previous prediction's start into
 * the same slot (a box of radius t * max step plus rounding margins, clipped
 * to the output); a particle never leaves that box, so every other cell
 * still holds the zero of an earlier pass. The batch records each slot's
 * start in device memory (so a graph replay with new starts is covered).
 * The first prediction after this call, after pm_batch_set or after
 * pm_batch_set_block_flags zeroes every cell. In this mode the caller must
 * not write into the counts between predictions (reading them is fine);
 * after it has, call this function again. Stream-ordered; PM_EINVAL for
 * another value. */
pm_status pm_batch_set_zeroing(pm_batch *b, int32_t reach, void *stream);

/* Time candidate launch shapes (emplacement mode, threads per CTA and
 * shared-memory window size) on the current batch with CUDA events and keep
 * the fastest; it runs pm_batch_predict several times (outputs are
 * overwritten). Synchronous. */
pm_status pm_batch_autotune(pm_batch *b, void *stream);

/* Read or set the launch shape: threads per CTA (multiple of 32, <= 256;
 * a new batch starts with 128 threads, warp-combined emplacement),
 * the emplacement mode, resident CTAs per SM used for the grid (0 = as many
 * as fit) and the window budget in KiB of shared memory. shared_window = 0:
 * persistent warps take 32-particle tiles and combine the lanes of a warp
 * that land in the same cell into one global reduction; 1: a CTA takes a
 * tile of `threads` particles and counts each step in its shared-memory
 * window, flushed once per touched cell. pm_batch_set_config rebuilds the
 * work list when the tile size changes (queued on the legacy stream); a CUDA
 * graph that captured pm_batch_predict must be captured again after a change
 * of shape. Every shape gives the same counts. */
pm_status pm_batch_get_config(const pm_batch *b, int32_t *threads, int32_t *shared_window, int32_t *ctas_per_sm,
                              int32_t *window_kib);
pm_status pm_batch_set_config(pm_batch *b, int32_t threads, int32_t shared_window, int32_t ctas_per_sm,
                              int32_t window_kib);

/* Release the plan (synchronises with its pending uploads). */
void pm_batch_destroy(pm_batch *b);

/* ---- differentiation ------------------------------------------------------ */

/* Marginal log-likelihood of M observed trajectories under the model (built
 * on Eq. 2 and the joint prior of Eq. 3):
 *   L = sum_m log sum_j exp(log_prior_j + sum_t log pi_j(u_mt | z_mt)),
 * the control u_mt recovered from (z_mt, z_m,t+1) as in pm_update_posterior.
 *   offsets  [M+1] int32 (device): trajectory m is points offsets[m] ..
 *            offsets[m+1]-1 of traj_xy; offsets are clamped to [0, n_points]
 *   traj_xy  [n_points][2] FP32 (device)
 *   log_prior [G*B] (device)
 *   loglik   [1] FP32 (device) output
 * Per-step log pi is computed in FP32 and summed over each trajectory in
 * FP64. Uses context scratch (M*(2G+4) doubles): calls on one context must
 * be ordered on one stream. */
pm_status pm_loglik_forward(pm_ctx *ctx, const pm_model *model, int32_t M, const int32_t *offsets,
                            int32_t n_points, const float *traj_xy, const float *log_prior,
                            float *loglik, void *stream);

/* L as above and grad_out * dL/d(parameter) for the goal coordinates
 * d_goals [G][2], the speed d_speed [1] and the Q weights d_w [2] = (w1, w2)
 * (all device, FP32). The adjoint of Eq. 2 is
 *   d log pi_j / dp = beta (dQ(theta_obs)/dp - sum_k pi_k dQ(theta_k)/dp),
 * weighted by each trajectory's posterior over (beta, g). dL/dw1 is zero in
 * exact arithmetic (w1 shifts every Q of a step equally) and is returned as
 * computed. Sums over trajectories run in a fixed order (deterministic). */
pm_status pm_loglik_backward(pm_ctx *ctx, const pm_model *model, int32_t M, const int32_t *offsets,
                             int32_t n_points, const float *traj_xy, const float *log_prior,
                             float grad_out, float *loglik, float *d_goals, float *d_speed,
                             float *d_w, void *stream);

/* ---- for callers that cannot allocate ------------------------------------- */

/* The paper has no counterpart to this call; it serves callers that must not
 * allocate device memory: a real-time loop that forbids allocation once it
 * runs, work enqueued during a stream capture whose mode rejects cudaMalloc,
 * or an application whose device memory belongs to its own pool. It computes
 * what pm_update_posterior computes (same arguments, same belief layout and
 * host-side validation) without a context, and allocates nothing: its
 * scratch is a static device array of this library, 164,096 bytes, which
 * every GPU that loads the library holds until the process exits. Limit:
 * G*B <= 256 (larger models are rejected with PM_EINVAL); the observed steps
 * are split over at most 32 CTAs. The first call on a device looks up the
 * array's device address (loading the library's device code, which
 * allocates), so make that first call before any stream capture; a first call
 * inside a capture returns PM_EINVAL. Later calls outside a capture look the
 * address up again, so the call stays valid after a device reset; inside a
 * capture they use the last address found on that device. Every call shares
 * the array, which keeps the last call's contents (the call clears the one
 * word that must start at zero): calls whose work overlaps on the GPU
 * (different streams, or several host threads) race on it and must be
 * serialised by the caller. Inputs that only the kernel can check are
 * handled as in pm_update_posterior (a step touching a non-finite observed
 * state is skipped; a NaN or +inf prior entry propagates) but are not
 * reported: there is no context whose status word pm_sync_status could read.
 * The belief may differ from pm_update_posterior's in the last bits (the
 * steps are summed in other chunks). */
pm_status pm_update_posterior_noalloc(const pm_model *model, const float *obs_xy, int32_t n_obs,
                                      float *log_belief, void *stream);

/* ---- grid epilogue: smoothing and multi-human union ---------------------- */

/* Gaussian convolution of one human's occupancy (Sec. III-B; the particles'
 * point masses are spread around their cells before the planner reads the
 * grid). prob[t][y][x] = sum_{i,j} w_i w_j counts[t][y+i][x+j] / n_particles
 * over the grid (cells off the grid count 0: mass blurred past the edge is
 * dropped), w_{-R..R} = exp(-i^2 / (2 sigma^2)) normalised to sum 1, R =
 * ceil(3 sigma) computed in double from the float sigma_cells, which must
 * satisfy 0 <= 3 sigma <= 16 (so R <= 16 cells; 0 = normalisation only). counts: device [horizon][grid->H][grid->W] (as written by
 * pm_predict_occupancy); prob: device float [horizon][grid->H][grid->W],
 * written entirely. Stream-ordered; PM_EINVAL for bad sizes or sigma. */
pm_status pm_smooth_occupancy(pm_ctx *ctx, const uint32_t *counts, int32_t n_particles, int32_t horizon,
                              const pm_grid *grid, float sigma_cells, float *prob, void *stream);

/* enable = 1: pm_batch_predict also marks, per human and step, the 16 x 16-cell
 * blocks of the output it emplaces into (a byte per block, in batch-owned
 * device memory; a few per cent of the rollout's time), so that
 * pm_batch_union skips the empty ones; 0 (the default): no marks, and
 * pm_batch_union reads every region. The warp-combined emplacement writes the
 * marks; with the shared-memory window form (pm_batch_set_config) the union
 * reads every region. Re-uploads the descriptors on `stream` like
 * pm_batch_set. The kernel variant is chosen when pm_batch_predict is
 * enqueued, so a CUDA graph that captured it must be captured again after a
 * change. PM_EINVAL for another value, PM_ENOMEM if the marks cannot be
 * allocated. */
pm_status pm_batch_set_block_flags(pm_batch *b, int32_t enable, void *stream);

/* Multi-human prediction on one shared grid (Sec. IV-B): every human of the
 * batch contributes its occupancy, blurred as pm_smooth_occupancy does (its
 * window widened by R cells, so mass blurred past the window is kept), at its
 * window's cell offset (cx_off, cy_off, or centred on its start cell), and
 * prob[t][y][x] is the pointwise maximum over the humans whose horizon
 * exceeds t (0 where none reaches). grid: the shared grid; every human's
 * grid must have the same origin and resolution. prob: device float
 * [horizon][grid->H][grid->W], written entirely. Reads the batch's device
 * descriptors, so it may be captured in the same CUDA graph as
 * pm_batch_predict (after it on the stream). With block flags on
 * (pm_batch_set_block_flags) it reads only the 16 x 16-cell blocks that
 * pm_batch_predict marked as holding a particle. PM_EINVAL for mismatched
 * grids, bad sizes or sigma. */
pm_status pm_batch_union(pm_batch *b, float sigma_cells, int32_t horizon, const pm_grid *grid, float *prob,
                         void *stream);

/* ---- local planner on the predictions ------------------------------------- */

/* MPPI (model predictive path integral) control of the robot of Eq. 8 against
 * the predicted occupancy, the local planner of Sec. III-C. Robot state
 * z = [x, y, v, theta], control u = [a, omega]; explicit Euler over dt:
 * x += v cos(theta) dt, y += v sin(theta) dt, v += a dt, theta += omega dt.
 * Sample i applies u_ref[t] + delta[t][i], t = 0..T-1; after step t it pays
 * (z - goal)^T diag(q) (z - goal) + u^T diag(r) u + step_cost, plus coll_cost
 * when the occupancy at the robot's cell (FP32 binning as the emplacement
 * step) at prediction step (t+1)*pred_stride - 1 is >= coll_threshold (no
 * cost outside the grid or past prob_T); the terminal cost is
 * (z_T - goal)^T diag(q_final) (z_T - goal). The update uses the
 * cost-to-go from each step: u_opt[t] = u_ref[t] + sum_i w_i delta[t][i] /
 * sum_i w_i, w_i = exp(-(S_i(t) - min_i S_i(t)) / temperature). */
typedef struct pm_mppi {
    int32_t n_samples;   /* N >= 1 */
    int32_t horizon;     /* T >= 1 MPPI steps */
    float dt;            /* seconds per MPPI step, > 0 */
    int32_t pred_stride; /* prediction steps per MPPI step, >= 1 */
    float q[4];          /* state weights (x, y, v, theta) */
    float q_final[4];    /* terminal state weights */
    float r[2];          /* control weights (a, omega) */
    float goal[4];       /* robot goal state */
    float coll_threshold, coll_cost, step_cost;
    float temperature;   /* tau > 0 */
} pm_mppi;

/* z0: robot state (host, 4 floats). u_ref: device [T][2]; delta: device
 * [T][N][2] (sample-minor, the caller draws it; 8-byte aligned, else PM_EINVAL); prob: device [prob_T][H][W]
 * predicted occupancy on `grid` (e.g. pm_batch_union's output), or NULL for
 * no collision cost. Outputs (device, caller-owned): cost_to_go [T][N]
 * (S_i(t); S_i(0) is sample i's total cost) and u_opt [T][2]. Two kernels,
 * stream-ordered, no allocation; PM_EINVAL for bad sizes or weights. */
pm_status pm_mppi_solve(pm_ctx *ctx, const pm_mppi *params, const float *z0, const float *u_ref,
                        const float *delta, const float *prob, int32_t prob_T, const pm_grid *grid,
                        float *cost_to_go, float *u_opt, void *stream);

/* ---- checks and measurement ---------------------------------------------- */

/* Raw Philox4x64-10 blocks for counters (particle0 + i, block, purpose, 0),
 * key (seed, human_id), i in [0, n): out [n][4] uint64 (device). */
pm_status pm_philox_blocks(pm_ctx *ctx, uint64_t seed, uint32_t human_id, uint32_t purpose,
                           uint64_t particle0, uint64_t block, int32_t n, uint64_t *out,
                           void *stream);

/* Throughput of one arithmetic operation measured on this device, in
 * results per second (eight independent chains per thread, 8 CTAs of 256
 * threads per SM): op 0 = ex2.approx.f32, 1 = sqrt.approx.f32,
 * 2 = rsqrt.approx.f32 (special-function unit), 3 = fma.rn.f32,
 * 4 = fma.rn.f32x2 (two results per instruction), 5 = add.u32.
 * PM_EINVAL for another op. Synchronous (times its own launch with events).
 * Ops 0-2 give the roofline of the rollout; 3-5 the FP32 and integer pipes
 * that its heading loop also loads. */
pm_status pm_probe_sfu(pm_ctx *ctx, int op, double *results_per_s);

/* Device properties the roofline uses: SM count, SM clock (kHz), and the
 * compute capability as 10*major + minor. Any output may be NULL. */
pm_status pm_device_info(pm_ctx *ctx, int *sm_count, int *clock_khz, int *cc);

#ifdef __cplusplus
}
#endif

#endif /* PM_H_ */
