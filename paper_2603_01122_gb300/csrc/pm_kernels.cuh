// pm_kernels.cuh -- arguments and launch wrappers of the kernels around the
// rollout: the belief update, the adjoint, the batched forms, the grid
// epilogue and the MPPI planner (private to the library). The rollout's own
// pieces are in pm_internal.cuh.
#pragma once

#include "pm_internal.cuh"

namespace pm {

// The control set of several speeds as the belief update and the adjoint see
// it (S = 0: one speed, multiplier 1).
struct SpeedSet {
    int S;
    uint32_t speed_on;         // bit q: speed q enabled
    float mult[PM_MAX_SPEEDS]; // multipliers m_q
    float sl[PM_MAX_SPEEDS];   // step lengths v*m_q*dt
    float w1;
};

// The enabled heading nearest to the direction (dx, dy): the largest
// e_k . (dx, dy), the lower index on a tie, decided in FP32 (the snapped
// reading of an observed control). Returns its unit vector.
__device__ __forceinline__ float2 nearest_heading(const float *ux, const float *uy, uint64_t enabled, int K, float dx,
                                                  float dy)
{
    float best = -INFINITY;
    int kb = 0;
    for (int k = 0; k < K; ++k) {
        const float c = fmaf(ux[k], dx, uy[k] * dy);
        if (((enabled >> k) & 1ull) && c > best) {
            best = c;
            kb = k;
        }
    }
    return make_float2(ux[kb], uy[kb]);
}

// Arguments of the belief-update kernel (Eq. 3 / Eq. 7).
struct PosteriorArgs {
    float ux[kMaxK], uy[kMaxK]; // unit heading vectors
    uint64_t enabled;
    float s, s2, two_s, w2;
    int K, G, B;
    SpeedSet sp;
    const float *goals;
    const float *beta;
    const float *obs;
    int n_obs;
    int steps_per_chunk; // observed steps handled by one CTA
    int snap;               // observed headings read as the nearest enabled heading
    const float *log_prior; // read by the fold (may equal log_b)
    float *log_b;
    float *part;         // scratch: per (chunk, component) accumulators
    unsigned *ticket;    // scratch: chunks finished so far (0 between calls)
    unsigned *status;    // context status word (or NULL)
};

// Arguments of the log-likelihood / adjoint kernel.
struct AdjointArgs {
    float ux[kMaxK], uy[kMaxK]; // unit heading vectors
    uint64_t enabled;
    float s, s2, two_s, w2, dt, v;
    int K, G, B;
    SpeedSet sp;
    const float *goals;
    const float *beta;
    int M;                 // trajectories
    const int32_t *offsets; // [M+1] point offsets
    int n_points;          // points in traj (offsets are clamped to it)
    const float *traj;     // [n_points][2]
    const float *log_prior; // [G*B]
    int want_grad;
    int snap;              // observed headings read as the nearest enabled heading
    float grad_out;
    double *part;          // scratch [M][2G+4]
    double *comp_A;        // scratch [M][J]: sum_t log pi per component
    float *comp_G;         // scratch [M][J][5]: the component's gradient sums
    unsigned *traj_ticket; // scratch [M]: CTAs of the trajectory finished (zeroed per call)
    unsigned *ticket;      // scratch ticket (0 between calls)
    unsigned *status;      // context status word (or NULL)
    float *loglik;
    float *d_goals;
    float *d_speed;
    float *d_w;
};

// One human of a batched belief update (device array).
struct PostHuman {
    const float *goals;
    const float *beta;
    int G, B;
    const float *obs;
    int n_obs;
    int steps_per_chunk;
    const float *log_prior; // read by the fold (the batch passes log_b)
    float *log_b;
    float *part;
    unsigned *ticket;
    uint32_t speed_on; // several speeds: bit q = speed q enabled for this human
};

// One human of a batched rollout (device array).
struct BatchHuman {
    const float *goals;
    const float *beta;
    int G, B;
    const float *log_b;
    const float *z0;      // device [2]
    int N, T;
    float gx0, gy0, inv_res;
    int W, H;             // output cells
    int center;           // output window centred on the start cell
    int cx_off, cy_off;   // output cell = grid cell - offset (center == 0)
    int reach_cells;      // ceil(T v dt / res) + 1
    uint64_t seed;
    uint32_t human;
    uint32_t *counts;
    uint32_t *oob;
    uint32_t speed_on;    // several speeds: bit q = speed q enabled for this human
    uint8_t *flags;       // [T][fby][fbx] block occupancy written with the counts, or NULL
    int fbx, fby;         // output blocks of kFlagBlock x kFlagBlock cells per row / column
};


// Grid epilogue (Gaussian smoothing, Sec. III-B; max-union, Sec. IV-B).
constexpr int kMaxSmoothR = 16; // blur radius ceil(3 sigma) in cells

struct SmoothSrc {
    const uint32_t *counts; // [T][H][W]
    float inv_n;            // 1 / particles
    int T, W, H;
    int ox, oy;             // window cell (x, y) = shared cell (x + ox, y + oy)
    int small;              // every count < 2^23 (N < 2^23): exact FP32 conversion by the mantissa
    const uint8_t *flags;   // block occupancy [T][fby][fbx], or NULL (stage every region)
    int fbx, fby;
};

struct SmoothArgs {
    const SmoothSrc *srcs; // device source records, or nullptr: `single`
    const int *n_srcs;     // device: number of records
    SmoothSrc single;
    float w[2 * kMaxSmoothR + 1]; // normalised taps w_{-R..R}
    int R;
    float *out; // shared grid [T][H][W]
    int T, W, H;
};

// MPPI local planner on the predicted occupancy (Sec. III-C, Eq. 8).
struct MppiArgs {
    int N, T, pred_stride;
    float dt;
    float z0[4]; // x, y, v, theta
    float q[4], q_final[4], r[2], goal[4];
    float coll_threshold, coll_cost, step_cost, temperature;
    const float *u_ref; // [T][2]
    const float *delta; // [T][N][2]
    const float *prob;  // [prob_T][H][W] or nullptr
    int prob_T, W, H;
    float gx0, gy0, inv_res;
    float *ctg;   // [T][N] cost-to-go (out)
    float *u_opt; // [T][2] (out)
};

struct BatchArgs {
    HeadingTab tab;
    uint64_t enabled;
    float s2, w2_log2e, w1_vdt_log2e;
    int K;
    const BatchHuman *humans;
    const int2 *items;   // (human, first particle), longest horizon first
    const int *n_items;
    unsigned *head;      // next tile (zeroed before every launch)
    int win_radius_cap;  // (2r+1)^2 cells fit the dynamic shared memory
    unsigned *status;    // context status word (or NULL)
    int marks;           // write block occupancy flags (the humans' flags are set)
};

// Launch shape of the rollout: threads per CTA, particles per thread (1 or
// 2) and the emplacement mode (warp-combined global reductions, or the
// shared-memory window).
struct RolloutShape {
    int threads;
    int ppt;
    bool warp_hist;
};

// Launch wrappers (defined next to their kernels).
cudaError_t launch_smooth_union(const SmoothArgs &a, cudaStream_t s);
cudaError_t launch_mppi(const MppiArgs &a, cudaStream_t s);
// One SmoothSrc per live human of a batch (window offsets resolved on the device).
cudaError_t launch_union_sources(const BatchHuman *humans, const int *n_humans, int max_humans, SmoothSrc *srcs,
                                 cudaStream_t s);
cudaError_t launch_posterior(const PosteriorArgs &a, int n_chunks, cudaStream_t s);
int posterior_chunks(int n_obs, int *steps_per_chunk);
cudaError_t launch_posterior_batch(const PosteriorArgs &a, const PostHuman *humans, const int *n_humans,
                                   int max_rows, int max_chunks, int max_J, cudaStream_t s);
size_t posterior_scratch_bytes(int n_chunks, int J);
cudaError_t launch_philox_blocks(uint64_t seed, uint32_t human, uint32_t purpose,
                                 uint64_t particle0, uint64_t block, int n, uint64_t *out,
                                 cudaStream_t s);
cudaError_t launch_sfu_probe(int op, int blocks, int threads, int iters, float *sink,
                             cudaStream_t s);
cudaError_t launch_adjoint(const AdjointArgs &a, cudaStream_t s);
int batch_rollout_occupancy(int K, uint64_t enabled, int S, bool marks, const RolloutShape &shape, size_t dyn);
size_t batch_warp_tables_bytes(int threads, bool multi_speed); // dynamic shared memory of the warp form
cudaError_t launch_batch_rollout(const BatchArgs &a, const RolloutShape &shape, int blocks, size_t dyn, cudaStream_t s);
// prev == NULL: every cell; else the reachable cells of humans with a
// recorded previous start, and the call then records z0 in prev. n_dev[0]:
// live humans, n_dev[1]: their longest horizon (device); max_rows and t_max
// size the grid only.
cudaError_t launch_batch_zero(const BatchHuman *humans, const int *n_dev, int max_rows, int sm_count, int t_max,
                              float2 *prev, unsigned *ticket, float smax, cudaStream_t s);
// One human's outputs before its rollout, in one launch: counts [words]
// (or NULL), oob [T] (or NULL) and the chunk counter.
cudaError_t launch_zero_outputs(uint32_t *counts, size_t words, uint32_t *oob, int T, unsigned *head, int sm_count,
                                cudaStream_t s);
size_t adjoint_scratch_bytes(int M, int G, int J);
void adjoint_scratch_layout(void *base, int M, int G, int J, AdjointArgs &a);

} // namespace pm
