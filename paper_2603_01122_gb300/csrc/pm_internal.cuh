// pm_internal.cuh -- device helpers and kernel argument blocks private to the
// CUDA library (never shared with the CPU oracle).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "pm.h"

namespace pm {

constexpr int kMaxK = PM_MAX_HEADINGS;
constexpr int kMaxJ = PM_MAX_COMPONENTS;
constexpr uint32_t kPurposeSelect = 1u;
constexpr uint32_t kPurposeStep = 2u;

// ---------------------------------------------------------------------------
// Philox4x64-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy
// as 1, 2, 3", SC'11): ten rounds of two 64x64->128 multiplies, the Weyl key
// schedule added between rounds.
// ---------------------------------------------------------------------------
struct U64x4 {
    uint64_t a, b, c, d;
};

__device__ __forceinline__ U64x4 philox4x64_10(U64x4 x, uint64_t k0, uint64_t k1)
{
    constexpr uint64_t kMulA = 0xD2E7470EE14C6C93ull;
    constexpr uint64_t kMulB = 0xCA5A826395121157ull;
    constexpr uint64_t kWeylA = 0x9E3779B97F4A7C15ull;
    constexpr uint64_t kWeylB = 0xBB67AE8584CAA73Bull;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint64_t pa_hi = __umul64hi(kMulA, x.a), pa_lo = kMulA * x.a;
        const uint64_t pc_hi = __umul64hi(kMulB, x.c), pc_lo = kMulB * x.c;
        x = U64x4{pc_hi ^ x.b ^ k0, pc_lo, pa_hi ^ x.d ^ k1, pa_lo};
        k0 += kWeylA;
        k1 += kWeylB;
    }
    return x;
}

// ---------------------------------------------------------------------------
// Special-function-unit approximations (one MUFU instruction each).
// ---------------------------------------------------------------------------
__device__ __forceinline__ float ex2_approx(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float sqrt_approx(float x)
{
    float y;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float rsqrt_approx(float x)
{
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Two FP32 values in one 64-bit register pair (low half first) and the
// packed FP32 arithmetic of sm_100+ (one instruction, two IEEE operations,
// each rounded exactly as the scalar instruction would).
typedef unsigned long long f32x2;

__device__ __forceinline__ f32x2 f2_pack(float lo, float hi)
{
    f32x2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}

__device__ __forceinline__ void f2_unpack(f32x2 v, float &lo, float &hi)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}

__device__ __forceinline__ f32x2 f2_fma(f32x2 a, f32x2 b, f32x2 c)
{
    f32x2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

__device__ __forceinline__ f32x2 f2_add(f32x2 a, f32x2 b)
{
    f32x2 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

__device__ __forceinline__ f32x2 f2_sub(f32x2 a, f32x2 b)
{
    f32x2 d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

__device__ __forceinline__ f32x2 f2_mul(f32x2 a, f32x2 b)
{
    f32x2 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

// Fire-and-forget global add (the result is not needed).
__device__ __forceinline__ void red_add(uint32_t *p, uint32_t v)
{
    asm volatile("red.relaxed.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// ---------------------------------------------------------------------------
// Heading tables computed on the host (in double, rounded once to FP32).
// ---------------------------------------------------------------------------
struct HeadingTab {
    float ux[kMaxK], uy[kMaxK]; // unit vector (cos, sin) of theta_k
    float sx[kMaxK], sy[kMaxK]; // one Euler step v*dt*(cos, sin)
    float tx[kMaxK], ty[kMaxK]; // 2*v*dt*(cos, sin)
    float s;                    // step length v*dt
    // 2 s sin(pi / 2K): with all K equally spaced headings enabled, the
    // nearest one to any direction is within pi/K, so min_k d_k exceeds the
    // triangle bound |r - s| by at most this much (zero when the headings are
    // not all enabled: the bound is then not used)
    float lb_gap;
    // Several speeds (S >= 2, or one speed with a multiplier != 1): control
    // u = s*K + k moves sl[s] = v*mult[s]*dt along theta_k.
    int S;
    uint32_t speed_on;              // bit s: speed s enabled
    float mult[PM_MAX_SPEEDS];      // speed multipliers
    float sl[PM_MAX_SPEEDS];        // v*mult[s]*dt
    float msx[PM_MAX_SPEEDS][kMaxK]; // Euler step of control (s, k), rounded once from double
    float msy[PM_MAX_SPEEDS][kMaxK];
};

// Device status word of a context: kernels OR these bits into it when they
// meet inputs they cannot use (the affected work is skipped or its result is
// meaningless); pm_sync_status reports and clears them.
constexpr unsigned kStatusModel = 1u;  // a goal or beta value is not finite
constexpr unsigned kStatusBelief = 2u; // a log-belief is NaN or +inf, or every one is -inf
constexpr unsigned kStatusObs = 4u;    // an observed state is not finite (its steps are skipped)
constexpr unsigned kStatusTraj = 8u;   // a trajectory point is not finite (its steps are skipped)

__device__ __forceinline__ void flag_status(unsigned *status, unsigned bit)
{
    if (status) atomicOr(status, bit);
}

// Arguments of the rollout kernel (Algorithm 1 + emplacement).
struct RolloutArgs {
    HeadingTab tab;
    uint64_t enabled; // bit k: heading k may be drawn (k < K and not disabled)
    float s2;         // (v*dt)^2
    float w2_log2e;   // w2 * log2(e): beta*w2*log2(e) scales distance differences
    float w1_vdt_log2e; // w1 * v * dt * log2(e) (several speeds: beta times it times m_s)
    int K, G, B;
    const float *goals;
    const float *beta;
    const float *log_b;
    float z0x, z0y;
    int N, T;
    float gx0, gy0, inv_res;
    int W, H;
    uint64_t seed;
    uint32_t human;
    uint32_t *counts;
    uint32_t *oob;
    int win_x0, win_y0;  // shared-memory window origin (grid cells)
    int win_side;        // window width | height << 16 (cells, each <= 255); 0 = no window
    int n_trace;
    float *tr_states;
    uint8_t *tr_head;
    int32_t *tr_comp;
    unsigned *status; // context status word (or NULL)
};

// The control set of several speeds as the belief update and the adjoint see
// it (S = 0: one speed, multiplier 1).
struct SpeedSet {
    int S;
    uint32_t speed_on;         // bit q: speed q enabled
    float mult[PM_MAX_SPEEDS]; // multipliers m_q
    float sl[PM_MAX_SPEEDS];   // step lengths v*m_q*dt
    float w1;
};

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

// Block occupancy flags of a batch's histograms: flags[t][by][bx] = 1 once a
// particle is emplaced in the output block of kFlagBlock x kFlagBlock cells
// (bx = cx >> kFlagShift); the union epilogue skips the blocks left at 0.
constexpr int kFlagShift = 4, kFlagBlock = 1 << kFlagShift;

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
// `head` is a zeroed device counter of 32-particle chunks.
cudaError_t launch_rollout(const RolloutArgs &a, unsigned *head, int sm_count, cudaStream_t s);
cudaError_t launch_smooth_union(const SmoothArgs &a, cudaStream_t s);
cudaError_t launch_mppi(const MppiArgs &a, cudaStream_t s);
// One SmoothSrc per live human of a batch (window offsets resolved on the device).
cudaError_t launch_union_sources(const BatchHuman *humans, const int *n_humans, int max_humans, SmoothSrc *srcs,
                                 cudaStream_t s);
size_t rollout_static_smem_estimate();
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
int rollout_kt_for(int K); // template bucket for K (8, 16, 36 or 64)
cudaError_t launch_adjoint(const AdjointArgs &a, cudaStream_t s);
int batch_rollout_occupancy(int K, uint64_t enabled, int S, bool marks, const RolloutShape &shape, size_t dyn);
size_t batch_warp_tables_bytes(int threads, bool multi_speed); // dynamic shared memory of the warp form
cudaError_t launch_batch_rollout(const BatchArgs &a, const RolloutShape &shape, int blocks, size_t dyn, cudaStream_t s);
cudaError_t launch_batch_zero(const BatchHuman *humans, const int *n_dev, int max_rows, int sm_count, cudaStream_t s);
size_t adjoint_scratch_bytes(int M, int G, int J);
void adjoint_scratch_layout(void *base, int M, int G, int J, AdjointArgs &a);

} // namespace pm
