// pm_rollout.cu -- Algorithm 1 (hardware-accelerated human prediction) with the
// bootstrapped belief of Sec. III-B and the per-step emplacement onto an
// occupancy grid, as one fused kernel: one thread per particle.
//
// Per particle and step (the hot loop), for every heading k:
//   distance from the next state to the goal, d_k = sqrt(D + 2 s e_k.(z - g))
//   with D = ||z - g||^2 + s^2, computed as a difference to a reference
//   distance plus one Newton correction, so that beta*w2*(d_j - d_k) keeps FP32
//   relative precision even when ||z - g|| >> s (a plain FP32 distance of a
//   5 m vector carries 5e-7 m of rounding, i.e. 5e-5 of logit at beta = 100);
//   logits beta*Q_k up to a common shift are -beta*w2*d_k (w1 cancels, Eq. 2);
//   the largest logit is found first, then ex2.approx on the SFU;
//   weights are rounded to 22-bit fixed point so that the running sums C_k of
//   the inverse CDF are exact integers (the sampling decision then depends
//   only on the rounded weights, not on summation order).
// The drawn heading moves the FP32 state by one Euler step (Eq. 1); the state
// is binned with FP32 operations (x - x0) * inv_res and counted in a
// per-CTA shared-memory window (16-bit counts packed two per word) whose
// touched cells are listed on first touch and flushed with one global
// reduction per touched cell at the end of the step.
#include <cuda_runtime.h>

#include "pm_internal.cuh"

namespace pm {
namespace {

constexpr int kRolloutThreads = 256;

struct __align__(16) RolloutShared {
    float4 comp[kMaxJ]; // (beta_b * w2 * log2 e, g_x, g_y, 0) of component j = g*B + b
    uint32_t cdf[kMaxJ]; // inclusive fixed-point running sum of the belief
    float2 step[kMaxK];  // Euler step of heading k
    uint32_t list_n[2];  // touched-cell list length, by step parity
    uint32_t oob_n[2];   // particles outside the grid, by step parity
};

// Warp 0 turns the log-belief into a fixed-point cumulative table:
// e_j = exp(log b_j - max) (accurate expf), E_j = round(e_j * 2^22),
// cdf[j] = E_0 + ... + E_j. Lane L owns the contiguous block j = 8L..8L+7.
__device__ void belief_cdf(const float *log_b, int J, uint32_t *cdf, int lane)
{
    float lb[8];
    float m = -INFINITY;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const int j = lane * 8 + q;
        lb[q] = (j < J) ? log_b[j] : -INFINITY;
        m = fmaxf(m, lb[q]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    uint32_t run = 0, pre[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const float e = (lb[q] == -INFINITY || m == -INFINITY) ? 0.0f : expf(lb[q] - m);
        run += __float2uint_rn(e * 4194304.0f);
        pre[q] = run;
    }
    uint32_t incl = run;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    const uint32_t excl = incl - run;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const int j = lane * 8 + q;
        if (j < J) cdf[j] = pre[q] + excl;
    }
}

// One heading draw of Eq. 2 at state (x, y) for goal (gx, gy) and
// cb = beta * w2 * log2(e). FULL: all KT headings enabled.
template <int KT, bool FULL>
__device__ __forceinline__ int draw_heading(const RolloutArgs &a, float x, float y, float gx,
                                            float gy, float cb, uint32_t word)
{
    const float dx = x - gx, dy = y - gy;
    const float D = fmaf(dx, dx, fmaf(dy, dy, a.s2));
    const float hD = 0.5f * rsqrt_approx(D); // 1/(2 d), D >= s^2 > 0
    float dv[KT];
    float dref = 0.0f;
    if (FULL && (KT % 2 == 0)) {
        // e_{k+K/2} = -e_k exactly in the tables: one dot product serves both
#pragma unroll
        for (int k = 0; k < KT / 2; ++k) {
            const float p = fmaf(a.tab.tx[k], dx, a.tab.ty[k] * dy); // 2 s e_k.(z - g)
            const float dk = sqrt_approx(fmaxf(D + p, 0.0f));
            const float dm = sqrt_approx(fmaxf(D - p, 0.0f));
            const float rk = fmaf(-dk, dk, D) + p;                  // residual D + p - dk^2
            const float rm = fmaf(-dm, dm, D) - p;
            if (k == 0) dref = dk;
            dv[k] = fmaf(rk, hD, dk - dref);                         // d_k - d_0, corrected
            dv[k + KT / 2] = fmaf(rm, hD, dm - dref);
        }
    } else {
#pragma unroll
        for (int k = 0; k < KT; ++k) {
            const float p = fmaf(a.tab.tx[k], dx, a.tab.ty[k] * dy);
            const float dk = sqrt_approx(fmaxf(D + p, 0.0f));
            const float rk = fmaf(-dk, dk, D) + p;
            if (k == 0) dref = dk;
            dv[k] = fmaf(rk, hD, dk - dref);
        }
    }
    float dmin = INFINITY;
#pragma unroll
    for (int k = 0; k < KT; ++k)
        if (FULL || ((a.enabled >> k) & 1ull)) dmin = fminf(dmin, dv[k]);
    const float base = dmin * cb;
    const float nc = -cb;
    uint32_t C[KT];
    uint32_t S = 0;
#pragma unroll
    for (int k = 0; k < KT; ++k) {
        const float e = ex2_approx(fmaf(dv[k], nc, base)); // exp(beta*(Q_k - Q_max))
        uint32_t E = __float_as_uint(fmaf(e, 4194304.0f, 12582912.0f)) - 0x4B400000u;
        if (!FULL && !((a.enabled >> k) & 1ull)) E = 0u;
        S += E;
        C[k] = S;
    }
    const uint32_t thr = (uint32_t)(((uint64_t)(word >> 8) * (uint64_t)S) >> 24);
    int sel = 0;
#pragma unroll
    for (int k = 0; k < KT; ++k) sel += (C[k] <= thr) ? 1 : 0;
    return sel;
}

template <int KT, bool FULL>
__global__ void __launch_bounds__(kRolloutThreads) rollout_kernel(const __grid_constant__ RolloutArgs a)
{
    __shared__ RolloutShared sh;
    extern __shared__ __align__(16) uint32_t dyn[];
    const int tid = threadIdx.x;
    const int nthr = blockDim.x;
    const int J = a.G * a.B;
    const bool hist = a.counts != nullptr;
    const int ww = a.win_side & 0xFFFF, wh = a.win_side >> 16; // window width/height (cells)
    const int win_cells = ww * wh;
    const int win_words = (win_cells + 1) >> 1;
    uint32_t *win32 = dyn;
    uint16_t *win16 = reinterpret_cast<uint16_t *>(dyn);
    uint16_t *list = reinterpret_cast<uint16_t *>(dyn + win_words);

    for (int j = tid; j < J; j += nthr) {
        const int g = j / a.B, b = j - g * a.B;
        sh.comp[j] = make_float4(a.beta[b] * a.w2_log2e, a.goals[2 * g], a.goals[2 * g + 1], 0.0f);
    }
    for (int k = tid; k < KT; k += nthr) sh.step[k] = make_float2(a.tab.sx[k], a.tab.sy[k]);
    if (hist)
        for (int w = tid; w < win_words; w += nthr) win32[w] = 0u;
    if (tid < 2) {
        sh.list_n[tid] = 0u;
        sh.oob_n[tid] = 0u;
    }
    if (tid < 32) belief_cdf(a.log_b, J, sh.cdf, tid);
    __syncthreads();

    const int64_t i = (int64_t)blockIdx.x * nthr + tid;
    const bool active = i < a.N;
    const bool traced = i < a.n_trace;
    float x = a.z0x, y = a.z0y, cb = 0.0f, gx = 0.0f, gy = 0.0f;
    if (active) {
        const U64x4 r = philox4x64_10(U64x4{(uint64_t)i, 0ull, kPurposeSelect, 0ull}, a.seed, a.human);
        const uint32_t thr = (uint32_t)(((uint64_t)((uint32_t)r.a >> 8) * (uint64_t)sh.cdf[J - 1]) >> 24);
        int lo = 0, hi = J - 1; // smallest j with cdf[j] > thr
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (sh.cdf[mid] > thr) hi = mid;
            else lo = mid + 1;
        }
        const float4 c = sh.comp[lo];
        cb = c.x;
        gx = c.y;
        gy = c.z;
        if (traced && a.tr_comp) a.tr_comp[i] = lo;
    }

    const size_t plane = (size_t)a.W * (size_t)a.H;
    uint32_t q0 = 0, q1 = 0, q2 = 0, q3 = 0, q4 = 0, q5 = 0, q6 = 0, q7 = 0;
    for (int t = 1; t <= a.T; ++t) {
        int cx = 0, cy = 0;
        bool in_grid = false;
        if (active) {
            if (((t - 1) & 7) == 0) {
                const U64x4 r = philox4x64_10(
                    U64x4{(uint64_t)i, (uint64_t)((t - 1) >> 3), kPurposeStep, 0ull}, a.seed, a.human);
                q0 = (uint32_t)r.a; q1 = (uint32_t)(r.a >> 32);
                q2 = (uint32_t)r.b; q3 = (uint32_t)(r.b >> 32);
                q4 = (uint32_t)r.c; q5 = (uint32_t)(r.c >> 32);
                q6 = (uint32_t)r.d; q7 = (uint32_t)(r.d >> 32);
            }
            const uint32_t word = q0;
            q0 = q1; q1 = q2; q2 = q3; q3 = q4; q4 = q5; q5 = q6; q6 = q7;
            const int k = draw_heading<KT, FULL>(a, x, y, gx, gy, cb, word);
            const float2 st = sh.step[k];
            x = __fadd_rn(x, st.x);
            y = __fadd_rn(y, st.y);
            if (traced) {
                const size_t o = (size_t)i * a.T + (t - 1);
                if (a.tr_states) reinterpret_cast<float2 *>(a.tr_states)[o] = make_float2(x, y);
                if (a.tr_head) a.tr_head[o] = (uint8_t)k;
            }
            if (hist) {
                const float vx = __fmul_rn(__fsub_rn(x, a.gx0), a.inv_res);
                const float vy = __fmul_rn(__fsub_rn(y, a.gy0), a.inv_res);
                cx = __float2int_rd(vx);
                cy = __float2int_rd(vy);
                in_grid = (vx == vx) && (vy == vy) && cx >= 0 && cx < a.W && cy >= 0 && cy < a.H;
            }
        }
        if (!hist) continue;
        __syncthreads(); // the flush of step t-1 has cleared the window
        if (tid == 0) sh.list_n[(t + 1) & 1] = 0u;
        if (active) {
            if (!in_grid) {
                atomicAdd(&sh.oob_n[t & 1], 1u);
            } else {
                const int wx = cx - a.win_x0, wy = cy - a.win_y0;
                if ((unsigned)wx < (unsigned)ww && (unsigned)wy < (unsigned)wh) {
                    const int w = wy * ww + wx;
                    const uint32_t sft = (uint32_t)(w & 1) << 4;
                    const uint32_t old = atomicAdd(&win32[w >> 1], 1u << sft);
                    if (((old >> sft) & 0xFFFFu) == 0u) {
                        const uint32_t slot = atomicAdd(&sh.list_n[t & 1], 1u);
                        list[slot] = (uint16_t)(wx | (wy << 8));
                    }
                } else {
                    red_add(a.counts + (size_t)(t - 1) * plane + (size_t)cy * a.W + cx, 1u);
                }
            }
        }
        __syncthreads(); // all of step t is in the window
        const uint32_t n = sh.list_n[t & 1];
        uint32_t *crow = a.counts + (size_t)(t - 1) * plane;
        for (uint32_t e = tid; e < n; e += nthr) {
            const uint32_t pk = list[e];
            const int wx = (int)(pk & 0xFFu), wy = (int)(pk >> 8);
            const int w = wy * ww + wx;
            const uint32_t c = win16[w];
            win16[w] = 0;
            red_add(crow + (size_t)(a.win_y0 + wy) * a.W + (a.win_x0 + wx), c);
        }
        if (tid == 0) {
            const uint32_t o = sh.oob_n[t & 1];
            if (o) red_add(a.oob + (t - 1), o);
            sh.oob_n[t & 1] = 0u;
        }
    }
}

template <int KT>
int occupancy_kt(bool full, int threads, size_t dyn_smem)
{
    int n = 0;
    if (full) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, rollout_kernel<KT, true>, threads, dyn_smem);
    else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, rollout_kernel<KT, false>, threads, dyn_smem);
    return n;
}

template <int KT>
cudaError_t launch_kt(const RolloutArgs &a, int threads, size_t dyn_smem, cudaStream_t s)
{
    const uint64_t all = (KT >= 64) ? ~0ull : ((1ull << KT) - 1ull);
    const bool full = (a.K == KT) && ((a.enabled & all) == all);
    const unsigned blocks = (unsigned)((a.N + threads - 1) / threads);
    if (full) {
        auto k = rollout_kernel<KT, true>;
        if (dyn_smem > 48 * 1024) {
            cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn_smem);
            if (e != cudaSuccess) return e;
        }
        k<<<blocks, threads, dyn_smem, s>>>(a);
    } else {
        auto k = rollout_kernel<KT, false>;
        if (dyn_smem > 48 * 1024) {
            cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn_smem);
            if (e != cudaSuccess) return e;
        }
        k<<<blocks, threads, dyn_smem, s>>>(a);
    }
    return cudaGetLastError();
}

} // namespace

int rollout_kt_for(int K)
{
    if (K <= 8) return 8;
    if (K <= 16) return 16;
    if (K <= 36) return 36;
    return 64;
}

size_t rollout_static_smem_estimate() { return sizeof(RolloutShared); }

int rollout_occupancy(const RolloutArgs &a, int threads, size_t dyn_smem)
{
    const int KT = rollout_kt_for(a.K);
    const uint64_t all = (KT >= 64) ? ~0ull : ((1ull << KT) - 1ull);
    const bool full = (a.K == KT) && ((a.enabled & all) == all);
    if (dyn_smem > 48 * 1024) {
        // the attribute must be raised before the occupancy query counts it
        switch (KT) {
        case 8: cudaFuncSetAttribute(full ? rollout_kernel<8, true> : rollout_kernel<8, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn_smem); break;
        case 16: cudaFuncSetAttribute(full ? rollout_kernel<16, true> : rollout_kernel<16, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn_smem); break;
        case 36: cudaFuncSetAttribute(full ? rollout_kernel<36, true> : rollout_kernel<36, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn_smem); break;
        default: cudaFuncSetAttribute(full ? rollout_kernel<64, true> : rollout_kernel<64, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn_smem); break;
        }
    }
    switch (KT) {
    case 8: return occupancy_kt<8>(full, threads, dyn_smem);
    case 16: return occupancy_kt<16>(full, threads, dyn_smem);
    case 36: return occupancy_kt<36>(full, threads, dyn_smem);
    default: return occupancy_kt<64>(full, threads, dyn_smem);
    }
}

cudaError_t launch_rollout(const RolloutArgs &a, int threads, size_t dyn_smem, cudaStream_t s)
{
    if (threads <= 0) threads = kRolloutThreads;
    switch (rollout_kt_for(a.K)) {
    case 8: return launch_kt<8>(a, threads, dyn_smem, s);
    case 16: return launch_kt<16>(a, threads, dyn_smem, s);
    case 36: return launch_kt<36>(a, threads, dyn_smem, s);
    default: return launch_kt<64>(a, threads, dyn_smem, s);
    }
}

} // namespace pm
