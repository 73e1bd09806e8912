// pm_rollout_dev.cuh -- device pieces of Algorithm 1 shared by the
// single-human and the batched rollout kernels (private to the library).
#pragma once

#include "pm_internal.cuh"

namespace pm {

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
__device__ inline void belief_cdf(const float *log_b, int J, uint32_t *cdf, int lane)
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
__device__ __forceinline__ int draw_heading(const HeadingTab &tab, uint64_t enabled, float s2, float x, float y,
                                            float gx, float gy, float cb, uint32_t word)
{
    const float dx = x - gx, dy = y - gy;
    const float D = fmaf(dx, dx, fmaf(dy, dy, s2));
    const float hD = 0.5f * rsqrt_approx(D); // 1/(2 d), D >= s^2 > 0
    float dv[KT];
    float dref = 0.0f;
    if (FULL && (KT % 2 == 0)) {
        // e_{k+K/2} = -e_k exactly in the tables: one dot product serves both
#pragma unroll
        for (int k = 0; k < KT / 2; ++k) {
            const float p = fmaf(tab.tx[k], dx, tab.ty[k] * dy); // 2 s e_k.(z - g)
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
            const float p = fmaf(tab.tx[k], dx, tab.ty[k] * dy);
            const float dk = sqrt_approx(fmaxf(D + p, 0.0f));
            const float rk = fmaf(-dk, dk, D) + p;
            if (k == 0) dref = dk;
            dv[k] = fmaf(rk, hD, dk - dref);
        }
    }
    float dmin = INFINITY;
#pragma unroll
    for (int k = 0; k < KT; ++k)
        if (FULL || ((enabled >> k) & 1ull)) dmin = fminf(dmin, dv[k]);
    const float base = dmin * cb;
    const float nc = -cb;
    uint32_t C[KT];
    uint32_t S = 0;
#pragma unroll
    for (int k = 0; k < KT; ++k) {
        const float e = ex2_approx(fmaf(dv[k], nc, base)); // exp(beta*(Q_k - Q_max))
        uint32_t E = __float_as_uint(fmaf(e, 4194304.0f, 12582912.0f)) - 0x4B400000u;
        if (!FULL && !((enabled >> k) & 1ull)) E = 0u;
        S += E;
        C[k] = S;
    }
    const uint32_t thr = (uint32_t)(((uint64_t)(word >> 8) * (uint64_t)S) >> 24);
    int sel = 0;
#pragma unroll
    for (int k = 0; k < KT; ++k) sel += (C[k] <= thr) ? 1 : 0;
    return sel;
}


// Per-tile state of one human for rollout_tile.
struct TileCtx {
    float z0x, z0y;
    int T;
    int64_t i;      // this thread's particle index (within its human)
    bool active;    // i < particles of the human
    bool traced;    // record the trajectory of this particle
    uint64_t seed;
    uint32_t human;
    int J;
    bool hist;
    float gx0, gy0, inv_res; // grid the states are binned on
    int W, H;                // output cells
    int cx_off, cy_off;      // output cell = grid cell - offset
    uint32_t *counts;
    uint32_t *oob;
    int win_x0, win_y0, ww, wh; // shared-memory window, output cells
    float *tr_states;
    uint8_t *tr_head;
    int32_t *tr_comp;
};

// Algorithm 1 for one particle per thread of the CTA: the (beta, g) draw from
// the belief table in shared memory, then T heading draws and Euler steps,
// each step emplaced in the CTA's shared-memory window (first touch appends
// the cell to a list; the list is flushed with one global reduction per
// touched cell) or, outside the window, directly in global memory. `sh` must
// hold the component table and belief CDF of the human, the window must be
// zero and list_n / oob_n zero on entry; the window is zero again on exit.
template <int KT, bool FULL>
__device__ __forceinline__ void rollout_tile(const HeadingTab &tab, uint64_t enabled, float s2,
                                             const TileCtx &c, RolloutShared &sh, uint32_t *dyn)
{
    const int tid = threadIdx.x;
    const int nthr = blockDim.x;
    const int ww = c.ww, wh = c.wh;
    const int win_words = (ww * wh + 1) >> 1;
    uint32_t *win32 = dyn;
    uint16_t *win16 = reinterpret_cast<uint16_t *>(dyn);
    uint16_t *list = reinterpret_cast<uint16_t *>(dyn + win_words);

    float x = c.z0x, y = c.z0y, cb = 0.0f, gx = 0.0f, gy = 0.0f;
    const uint64_t i = (uint64_t)c.i;
    if (c.active) {
        const U64x4 r = philox4x64_10(U64x4{i, 0ull, kPurposeSelect, 0ull}, c.seed, c.human);
        const uint32_t thr = (uint32_t)(((uint64_t)((uint32_t)r.a >> 8) * (uint64_t)sh.cdf[c.J - 1]) >> 24);
        int lo = 0, hi = c.J - 1; // smallest j with cdf[j] > thr
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (sh.cdf[mid] > thr) hi = mid;
            else lo = mid + 1;
        }
        const float4 cc = sh.comp[lo];
        cb = cc.x;
        gx = cc.y;
        gy = cc.z;
        if (c.traced && c.tr_comp) c.tr_comp[i] = lo;
    }

    const size_t plane = (size_t)c.W * (size_t)c.H;
    uint32_t q0 = 0, q1 = 0, q2 = 0, q3 = 0, q4 = 0, q5 = 0, q6 = 0, q7 = 0;
    for (int t = 1; t <= c.T; ++t) {
        int cx = 0, cy = 0;
        bool in_grid = false;
        if (c.active) {
            if (((t - 1) & 7) == 0) {
                const U64x4 r = philox4x64_10(U64x4{i, (uint64_t)((t - 1) >> 3), kPurposeStep, 0ull}, c.seed, c.human);
                q0 = (uint32_t)r.a; q1 = (uint32_t)(r.a >> 32);
                q2 = (uint32_t)r.b; q3 = (uint32_t)(r.b >> 32);
                q4 = (uint32_t)r.c; q5 = (uint32_t)(r.c >> 32);
                q6 = (uint32_t)r.d; q7 = (uint32_t)(r.d >> 32);
            }
            const uint32_t word = q0;
            q0 = q1; q1 = q2; q2 = q3; q3 = q4; q4 = q5; q5 = q6; q6 = q7;
            const int k = draw_heading<KT, FULL>(tab, enabled, s2, x, y, gx, gy, cb, word);
            const float2 st = sh.step[k];
            x = __fadd_rn(x, st.x);
            y = __fadd_rn(y, st.y);
            if (c.traced) {
                const size_t o = (size_t)i * c.T + (t - 1);
                if (c.tr_states) reinterpret_cast<float2 *>(c.tr_states)[o] = make_float2(x, y);
                if (c.tr_head) c.tr_head[o] = (uint8_t)k;
            }
            if (c.hist) {
                const float vx = __fmul_rn(__fsub_rn(x, c.gx0), c.inv_res);
                const float vy = __fmul_rn(__fsub_rn(y, c.gy0), c.inv_res);
                cx = __float2int_rd(vx) - c.cx_off;
                cy = __float2int_rd(vy) - c.cy_off;
                in_grid = (vx == vx) && (vy == vy) && cx >= 0 && cx < c.W && cy >= 0 && cy < c.H;
            }
        }
        if (!c.hist) continue;
        __syncthreads(); // the flush of step t-1 has cleared the window
        if (tid == 0) sh.list_n[(t + 1) & 1] = 0u;
        if (c.active) {
            if (!in_grid) {
                atomicAdd(&sh.oob_n[t & 1], 1u);
            } else {
                const int wx = cx - c.win_x0, wy = cy - c.win_y0;
                if ((unsigned)wx < (unsigned)ww && (unsigned)wy < (unsigned)wh) {
                    const int w = wy * ww + wx;
                    const uint32_t sft = (uint32_t)(w & 1) << 4;
                    const uint32_t old = atomicAdd(&win32[w >> 1], 1u << sft);
                    if (((old >> sft) & 0xFFFFu) == 0u) {
                        const uint32_t slot = atomicAdd(&sh.list_n[t & 1], 1u);
                        list[slot] = (uint16_t)(wx | (wy << 8));
                    }
                } else {
                    red_add(c.counts + (size_t)(t - 1) * plane + (size_t)cy * c.W + cx, 1u);
                }
            }
        }
        __syncthreads(); // all of step t is in the window
        const uint32_t n = sh.list_n[t & 1];
        uint32_t *crow = c.counts + (size_t)(t - 1) * plane;
        for (uint32_t e = tid; e < n; e += nthr) {
            const uint32_t pk = list[e];
            const int wx = (int)(pk & 0xFFu), wy = (int)(pk >> 8);
            const int w = wy * ww + wx;
            const uint32_t v = win16[w];
            win16[w] = 0;
            red_add(crow + (size_t)(c.win_y0 + wy) * c.W + (c.win_x0 + wx), v);
        }
        if (tid == 0) {
            const uint32_t o = sh.oob_n[t & 1];
            if (o) red_add(c.oob + (t - 1), o);
            sh.oob_n[t & 1] = 0u;
        }
    }
}

} // namespace pm
