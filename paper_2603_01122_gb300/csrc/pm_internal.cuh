// pm_internal.cuh -- device helpers and the rollout's argument block, private to the
// CUDA library (never shared with the CPU oracle).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "pm_limits.h"

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
// Fixed-point heading weights: a weight w in [0, 1] becomes the integer
// round(w 2^23) in the low mantissa bits of fma(w, kWScale, kWMagic) (the
// sum lies in [2^23, 2^24], where the float spacing is 1; w = 1 gives 2^24,
// whose bits minus kWBits are again 2^23). Sums of up to 511 weights fit
// 32 bits.
constexpr float kWScale = 8388608.0f;    // 2^23
constexpr float kWMagic = 8388608.0f;    // 2^23
constexpr uint32_t kWBits = 0x4B000000u; // bits of kWMagic

// Error-free sum (Knuth's TwoSum): a + b = s + e exactly, s = fl(a + b).
// Written with explicitly rounded operations so that no contraction or
// reassociation can change it.
__device__ __forceinline__ float two_sum(float a, float b, float &e)
{
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return s;
}

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
    float inv_mult[PM_MAX_SPEEDS];  // 1 / mult (FP32)
    float sl[PM_MAX_SPEEDS];        // v*mult[s]*dt
    float msx[PM_MAX_SPEEDS][kMaxK]; // Euler step of control (s, k), rounded once from double
    float msy[PM_MAX_SPEEDS][kMaxK];
    // w2 log2(e) and w1 v dt log2(e), each as a high and a low float (their
    // sum is the double value): the offsets between speeds are formed from
    // beta times these exactly
    float w2l[2], w1l[2];
    // the model's own values and the unit heading vectors in double-float
    // (hi, lo), for the settlement of a several-speed draw (draw_multi_exact)
    float v, dt, w1, w2;
    int K;
    float cdf[kMaxK][2], sdf[kMaxK][2];
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

// Block occupancy flags of a batch's histograms: flags[t][by][bx] = 1 once a
// particle is emplaced in the output block of kFlagBlock x kFlagBlock cells
// (bx = cx >> kFlagShift); the union epilogue skips the blocks left at 0.
constexpr int kFlagShift = 4, kFlagBlock = 1 << kFlagShift;

// Rollout launch (defined next to its kernels).
// `head` is a zeroed device counter of 32-particle chunks.
cudaError_t launch_rollout(const RolloutArgs &a, unsigned *head, int sm_count, cudaStream_t s);
int rollout_kt_for(int K); // template bucket for K (8, 16, 36 or 64)
size_t rollout_static_smem_estimate();

} // namespace pm
