// pm_rollout_dev.cuh -- device pieces of Algorithm 1 shared by the
// single-human and the batched rollout kernels (private to the library).
#pragma once

#include "pm_internal.cuh"

namespace pm {

struct __align__(16) RolloutShared {
    float4 comp[kMaxJ]; // (beta_b * w2 * log2 e, g_x, g_y, 0) of component j = g*B + b
    uint32_t cdf[kMaxJ]; // inclusive fixed-point running sum of the belief
    float2 step[kMaxK];  // Euler step of heading k
    uint32_t list_n[3];  // touched-cell list length, by step mod 3
    uint32_t oob_n[2];   // particles outside the grid, by step parity
};

// Warp 0 turns the log-belief into a fixed-point cumulative table:
// e_j = exp(log b_j - max) (accurate expf), E_j = round(e_j * 2^22),
// cdf[j] = E_0 + ... + E_j. Lane L owns the contiguous block j = 8L..8L+7.
// Returns kStatusBelief (the same on every lane) for a NaN or +inf entry or a
// belief with no finite entry, else 0; the caller latches it.
__device__ inline unsigned belief_cdf(const float *log_b, int J, uint32_t *cdf, int lane)
{
    float lb[8];
    float m = -INFINITY;
    bool bad = false;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const int j = lane * 8 + q;
        lb[q] = (j < J) ? log_b[j] : -INFINITY;
        bad = bad || isnan(lb[q]) || lb[q] == INFINITY;
        m = fmaxf(m, lb[q]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    const unsigned bits = (__any_sync(0xffffffffu, bad) || m == -INFINITY) ? kStatusBelief : 0u;
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
    return bits;
}

// One heading draw of Eq. 2 at state (x, y) for goal (gx, gy) and
// cb = beta * w2 * log2(e). FULL: all KT headings enabled.
//
// d_k - d_0 is formed from the residual of the approximate square root with
// the per-heading factor 1/(2 d_k) (to first order in p_k, as in
// corrected_minus: this draw serves the components of large |beta|), so
// beta*w2*(d_j - d_k) keeps FP32 relative precision; the weights
// exp(beta (Q_k - Q_max)) are rounded to 23-bit fixed point, so the running
// sums C_k are exact and the draw (smallest k with C_k > (u24 * S) >> 24)
// depends only on the rounded weights. For even KT with every heading
// enabled the FP32 work runs on packed pairs of consecutive headings
// (fma/add/sub/mul .f32x2: the same IEEE operations, half the instructions);
// otherwise it runs scalar, skipping disabled headings. Both give identical
// results.
template <int KT, bool FULL>
__device__ __forceinline__ int draw_heading(const HeadingTab &tab, uint64_t enabled, float s2, float x, float y,
                                            float gx, float gy, float cb, uint32_t word)
{
    const float dx = x - gx, dy = y - gy;
    const float D = fmaf(dx, dx, fmaf(dy, dy, s2));
    const float hD = 0.5f * rsqrt_approx(D); // 1/(2 d), D >= s^2 > 0
    const float c3 = -2.0f * hD * hD * hD;    // 1/(2 d_k) = hD + c3 p_k to first order
    if constexpr (FULL && (KT % 2 == 0)) {
        const f32x2 DX = f2_pack(dx, dx), DY = f2_pack(dy, dy);
        const f32x2 DD = f2_pack(D, D), NDD = f2_pack(-D, -D), HD = f2_pack(hD, hD), C3 = f2_pack(c3, c3);
        const f32x2 *TX = reinterpret_cast<const f32x2 *>(tab.tx);
        const f32x2 *TY = reinterpret_cast<const f32x2 *>(tab.ty);
        f32x2 dv[KT / 2];
        f32x2 DREF = 0ull;
        float dmin[4] = {INFINITY, INFINITY, INFINITY, INFINITY}; // independent partial minima
#pragma unroll
        for (int q = 0; q < KT / 2; ++q) {
            const f32x2 P = f2_fma(TX[q], DX, f2_mul(TY[q], DY)); // 2 s e_k.(z - g), k = 2q, 2q+1
            float x0, x1;
            f2_unpack(f2_add(DD, P), x0, x1);
            // |x| only differs from max(x, 0) when rounding made a (near-zero) square negative
            const float d0 = sqrt_approx(fabsf(x0)), d1 = sqrt_approx(fabsf(x1));
            const f32x2 DK = f2_pack(d0, d1);
            if (q == 0) DREF = f2_pack(d0, d0);
            const f32x2 R = f2_sub(P, f2_fma(DK, DK, NDD));       // D + p - dk^2
            dv[q] = f2_fma(R, f2_fma(P, C3, HD), f2_sub(DK, DREF)); // d_k - d_0, corrected
            float v0, v1;
            f2_unpack(dv[q], v0, v1);
            dmin[q & 3] = fminf(dmin[q & 3], fminf(v0, v1));
        }
        float dm = fminf(fminf(dmin[0], dmin[1]), fminf(dmin[2], dmin[3]));
        if (cb < 0.0f) { // beta < 0: the farthest heading is the most probable
            dm = -INFINITY;
#pragma unroll
            for (int q = 0; q < KT / 2; ++q) {
                float v0, v1;
                f2_unpack(dv[q], v0, v1);
                dm = fmaxf(dm, fmaxf(v0, v1));
            }
        }
        const f32x2 NC = f2_pack(-cb, -cb);
        const float base = __fmul_rd(dm, cb); // rounded down: every exponent below is <= 0
        const f32x2 BASE = f2_pack(base, base);
        const f32x2 SC = f2_pack(kWScale, kWScale), MG = f2_pack(kWMagic, kWMagic);
        constexpr int H2 = KT / 2; // the running sums restart at the half: two independent chains
        uint32_t bits[KT];
        uint32_t S0 = 0u, S1 = 0u;
#pragma unroll
        for (int q = 0; q < KT / 2; ++q) {
            float a0, a1;
            f2_unpack(f2_fma(dv[q], NC, BASE), a0, a1);             // log2 of exp(beta (Q_k - Q_max))
            float w0, w1;
            f2_unpack(f2_fma(f2_pack(ex2_approx(a0), ex2_approx(a1)), SC, MG), w0, w1);
            bits[2 * q] = __float_as_uint(w0);                      // kWBits + round(e * 2^23)
            bits[2 * q + 1] = __float_as_uint(w1);
            if (2 * q < H2) S0 += bits[2 * q]; else S1 += bits[2 * q];
            if (2 * q + 1 < H2) S0 += bits[2 * q + 1]; else S1 += bits[2 * q + 1];
        }
        S0 -= (uint32_t)H2 * kWBits;                           // weight of headings [0, K/2)
        S1 -= (uint32_t)(KT - H2) * kWBits;                    // weight of headings [K/2, K)
        const uint32_t S = S0 + S1;                                 // total weight (exact integer)
        const uint32_t thr = (uint32_t)(((uint64_t)(word >> 8) * (uint64_t)S) >> 24);
        // C_k - thr - 1 once E_k is added: negative iff C_k <= thr
        uint32_t acc0 = ~thr, acc1 = ~thr + S0;
        int sel0 = 0, sel1 = 0;
#pragma unroll
        for (int k = 0; k < H2; ++k) {
            acc0 += bits[k] - kWBits;
            sel0 += (int)(acc0 >> 31);
            acc1 += bits[H2 + k] - kWBits;
            sel1 += (int)(acc1 >> 31);
        }
        return sel0 + sel1;
    } else {
        float dv[KT];
        float dref = 0.0f;
#pragma unroll
        for (int k = 0; k < KT; ++k) {
            const float p = fmaf(tab.tx[k], dx, tab.ty[k] * dy);
            const float dk = sqrt_approx(fmaxf(D + p, 0.0f));
            const float rk = fmaf(-dk, dk, D) + p;
            if (k == 0) dref = dk;
            dv[k] = fmaf(rk, fmaf(p, c3, hD), dk - dref);
        }
        // the most probable heading: the nearest for beta >= 0, the farthest
        // for beta < 0, so that every exponent below is <= 0
        float dext = (cb >= 0.0f) ? INFINITY : -INFINITY;
#pragma unroll
        for (int k = 0; k < KT; ++k)
            if (FULL || ((enabled >> k) & 1ull)) dext = (cb >= 0.0f) ? fminf(dext, dv[k]) : fmaxf(dext, dv[k]);
        const float base = __fmul_rd(dext, cb); // rounded down: every exponent below is <= 0
        const float nc = -cb;
        uint32_t C[KT];
        uint32_t S = 0;
#pragma unroll
        for (int k = 0; k < KT; ++k) {
            const float e = ex2_approx(fmaf(dv[k], nc, base));
            uint32_t E = __float_as_uint(fmaf(e, kWScale, kWMagic)) - kWBits;
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
}

// The same draw for even KT with all KT equally spaced headings enabled, the
// weights normalised by a bound of the distances instead of their exact
// extreme, which fuses the distance, exponential and summation passes into one.
// By the triangle inequality every d_k lies in [|r - s|, r + s] (r = ||z - g||,
// s = v dt), and the heading nearest the extreme direction lies within pi/K of
// it, so the extreme d_k is within lb_gap = 2 s sin(pi/2K) of the bound. The
// reference ref is the lower bound for beta >= 0 and the upper bound for
// beta < 0, pushed outwards by a few ulps of r + s so that every exponent
// -cb (d_k - ref) is <= 0 after rounding; the largest weight is then at least
// 2^(-|cb| lb_gap) (callers use this form only where that is >= 1/2). A
// common shift of all logits leaves the distribution of Eq. 2 unchanged.
struct LbStep {
    float dx, dy; // z - g
    float D;      // ||z - g||^2 + s^2
    float r;      // ||z - g||
    float ref;    // reference distance (see above)
};

__device__ __forceinline__ LbStep lb_step_d(const HeadingTab &tab, float s2, float dx, float dy, float cb)
{
    LbStep q;
    q.dx = dx;
    q.dy = dy;
    q.D = fmaf(q.dx, q.dx, fmaf(q.dy, q.dy, s2));
    q.r = sqrt_approx(fmaf(q.dx, q.dx, q.dy * q.dy));
    const float margin = (q.r + tab.s) * 0x1p-20f;
    q.ref = (cb >= 0.0f) ? fabsf(q.r - tab.s) - margin : q.r + tab.s + margin;
    return q;
}

__device__ __forceinline__ LbStep lb_step(const HeadingTab &tab, float s2, float x, float y, float gx, float gy,
                                          float cb)
{
    return lb_step_d(tab, s2, x - gx, y - gy, cb);
}

// Segments of the several-speed fused draw (draw_multi_lb): KT/G segments of
// G headings per speed (G even, so a pair of headings never straddles two);
// pass 1 keeps their sums and pass 2 recomputes the G weights of the one
// holding the threshold.
template <int KT>
struct CdfSegs {
    static constexpr int G = (KT == 8) ? 4 : (KT == 16) ? 4 : (KT == 36) ? 6 : 8;
    static constexpr int N = KT / G;
    static_assert(KT % G == 0 && G % 2 == 0, "segments hold whole pairs");
};

// Segments of the one-speed draw's inverse CDF (draw_heading_lb): chosen to
// minimise the instructions of select_fixed (its count grows with the
// segments, for the search and the pick, and with their length, for the scan).
template <int KT>
struct SelSegs {
    static constexpr int G = (KT == 8) ? 4 : (KT == 16) ? 8 : (KT == 36) ? 12 : 16;
    static constexpr int N = KT / G;
    static_assert(KT % G == 0 && G % 2 == 0, "segments hold whole pairs");
};

// Inverse CDF over the 23-bit fixed-point weights (bits = kWBits + w_k):
// the smallest k with C_k > thr = (u24 * S) >> 24, i.e. the number of
// running sums C_k <= thr. Seg[q] is the raw sum of the bits of segment q.
// The segment holding thr is the last one whose start sum is <= thr (every
// running sum before it is <= thr, every one after it is > thr); its G
// weights are picked by predicated selects (registers cannot be indexed)
// and scanned from its start sum: about NS + 3 NS + NS G + 2 G instructions
// instead of 2 KT for counting every heading.
template <int KT>
__device__ __forceinline__ int select_fixed(const uint32_t (&bits)[KT], const uint32_t (&seg)[SelSegs<KT>::N],
                                            uint32_t word)
{
    constexpr int G = SelSegs<KT>::G, NS = SelSegs<KT>::N;
    uint32_t start[NS]; // C at the start of each segment
    uint32_t S = 0u;
#pragma unroll
    for (int q = 0; q < NS; ++q) {
        start[q] = S;
        S += seg[q] - (uint32_t)G * kWBits;
    }
    const uint32_t thr = (uint32_t)(((uint64_t)(word >> 8) * (uint64_t)S) >> 24);
    int qs = 0;
    uint32_t base = 0u;
#pragma unroll
    for (int q = 1; q < NS; ++q) {
        const bool in = start[q] <= thr;
        qs = in ? q : qs;
        base = in ? start[q] : base;
    }
    uint32_t b[G];
#pragma unroll
    for (int j = 0; j < G; ++j) b[j] = bits[j];
#pragma unroll
    for (int q = 1; q < NS; ++q) {
        const bool p = qs == q;
#pragma unroll
        for (int j = 0; j < G; ++j) b[j] = p ? bits[q * G + j] : b[j];
    }
    // C_k - thr - 1 once w_k is added: negative iff C_k <= thr
    uint32_t acc = base + ~thr;
    int sel = 0;
#pragma unroll
    for (int j = 0; j < G; ++j) {
        acc += b[j] - kWBits;
        sel += (int)(acc >> 31);
    }
    return qs * G + sel;
}

// Bound-normalised draw with the distances from the approximate square root
// and one Newton correction: with p_k = 2 s e_k.(z - g), d_k^2 = D + p_k and
// the residual R_k = D + p_k - dk^2 of the approximation dk,
//   -cb (d_k - ref) = R_k (-cb / 2d) + (dk (-cb) + cb ref).
// K is a multiple of 4 and the headings are equally spaced, so heading
// k + K/2 is -e_k exactly (the table is built by quarter turns) and shares
// p_k with the opposite sign: one p serves two pairs of headings, whose
// weights go to the two summation chains.
template <int KT>
__device__ __forceinline__ int draw_heading_lb(const HeadingTab &tab, const LbStep &q, float cb, uint32_t word)
{
    static_assert(KT % 4 == 0, "pairs of headings must not straddle the two summation chains");
    // 1/(2 d) with D >= s^2 > 0, on the integer and FP32 pipes (the XU is the
    // busiest unit): the exponent-halving guess of 1/sqrt(D) (Lomont's
    // constant) and one Newton step, relative error below 1.8e-3. It only
    // scales the residual correction, a few ulps of d_k, and is of the order
    // of the step's own approximation 1/(2 sqrt(D)) ~ 1/(2 d_k) (s / |z - g|).
    float hD = __int_as_float(0x5F375A86 - (__float_as_int(q.D) >> 1));
    hD = hD * fmaf(-0.25f * q.D * hD, hD, 0.75f);
    const f32x2 DX = f2_pack(q.dx, q.dx), DY = f2_pack(q.dy, q.dy);
    const f32x2 DD = f2_pack(q.D, q.D), NDD = f2_pack(-q.D, -q.D);
    const f32x2 SC = f2_pack(kWScale, kWScale), MG = f2_pack(kWMagic, kWMagic);
    const f32x2 *TX = reinterpret_cast<const f32x2 *>(tab.tx);
    const f32x2 *TY = reinterpret_cast<const f32x2 *>(tab.ty);
    constexpr int H2 = KT / 2;
    constexpr int G = SelSegs<KT>::G;
    uint32_t bits[KT];
    uint32_t seg[SelSegs<KT>::N];
#pragma unroll
    for (int q = 0; q < SelSegs<KT>::N; ++q) seg[q] = 0u;
    const f32x2 HDNC = f2_pack(-cb * hD, -cb * hD), NHDNC = f2_pack(cb * hD, cb * hD);
    const f32x2 NC = f2_pack(-cb, -cb), RC = f2_pack(cb * q.ref, cb * q.ref);
#pragma unroll
    for (int k2 = 0; k2 < KT / 4; ++k2) {
        const f32x2 P = f2_fma(TX[k2], DX, f2_mul(TY[k2], DY)); // heading k; k + K/2 has -P
        float x0, x1, y0, y1;
        f2_unpack(f2_add(DD, P), x0, x1);
        f2_unpack(f2_sub(DD, P), y0, y1);
        const f32x2 DA = f2_pack(sqrt_approx(fabsf(x0)), sqrt_approx(fabsf(x1)));
        const f32x2 DB = f2_pack(sqrt_approx(fabsf(y0)), sqrt_approx(fabsf(y1)));
        float a0, a1, b0, b1;
        f2_unpack(f2_fma(f2_sub(P, f2_fma(DA, DA, NDD)), HDNC, f2_fma(DA, NC, RC)), a0, a1);
        f2_unpack(f2_fma(f2_add(P, f2_fma(DB, DB, NDD)), NHDNC, f2_fma(DB, NC, RC)), b0, b1);
        float w0, w1, v0, v1;
        f2_unpack(f2_fma(f2_pack(ex2_approx(a0), ex2_approx(a1)), SC, MG), w0, w1);
        f2_unpack(f2_fma(f2_pack(ex2_approx(b0), ex2_approx(b1)), SC, MG), v0, v1);
        bits[2 * k2] = __float_as_uint(w0);
        bits[2 * k2 + 1] = __float_as_uint(w1);
        bits[H2 + 2 * k2] = __float_as_uint(v0);
        bits[H2 + 2 * k2 + 1] = __float_as_uint(v1);
        seg[(2 * k2) / G] += bits[2 * k2] + bits[2 * k2 + 1];
        seg[(H2 + 2 * k2) / G] += bits[H2 + 2 * k2] + bits[H2 + 2 * k2 + 1];
    }
    return select_fixed<KT>(bits, seg, word);
}

// Component flag of the belief table: the bound-normalised draw keeps the
// largest weight >= 1/2 (23-bit weights keep >= 22 significant bits).
__device__ __forceinline__ float lb_flag(const HeadingTab &tab, float cb)
{
    return (fabsf(cb) * tab.lb_gap <= 1.0f) ? 1.0f : 0.0f;
}

// A component's table entry must be finite (goal and beta w2 log2(e)).
__device__ __forceinline__ bool bad_component(float cb, float gx, float gy) { return !isfinite(cb + gx + gy); }

// The heading draw of one particle: the fused bound form where it applies.
template <int KT, bool FULL>
__device__ __forceinline__ int draw(const HeadingTab &tab, uint64_t enabled, float s2, float x, float y, float gx,
                                    float gy, float cb, bool lb, uint32_t word)
{
    int k;
    if constexpr (FULL && (KT % 4 == 0)) {
        if (lb) k = draw_heading_lb<KT>(tab, lb_step(tab, s2, x, y, gx, gy, cb), cb, word);
        else k = draw_heading<KT, FULL>(tab, enabled, s2, x, y, gx, gy, cb, word);
    } else {
        k = draw_heading<KT, FULL>(tab, enabled, s2, x, y, gx, gy, cb, word);
    }
    // k < K whenever the total weight S > 0, which finite inputs guarantee;
    // the clamp keeps the step-table read in bounds for any input
    return min(k, KT - 1);
}

// ---------------------------------------------------------------------------
// Several speeds: Eq. 2 over the controls u = s*K + k (speed-major), each
// moving sl[s] = v*m_s*dt along theta_k, with
//   beta Q_u log2(e) = -(cb d_{k,s} + cw1 m_s),  cb = beta w2 log2(e),
//   cw1 = beta w1 v dt log2(e).
// Per speed the distances use the same corrected form as the one-speed draw
// against a reference REF_s (the triangle bound |r - s_s| pushed out by a few
// ulps, or with lb false the exact extreme over the speed's headings); the
// speeds are tied together by C_s = cb (REF_s - REF_b) + cw1 (m_s - m_b) - min,
// formed from differences of nearby floats (exact), so the exponent
//   a_{k,s} = -cb U_{k,s} - C_s <= 0,  U_{k,s} = d_{k,s} - REF_s.
// Pass 1 sums each speed's 23-bit fixed-point weights; the threshold picks
// the speed from the running per-speed totals, and pass 2 recomputes that
// speed's weights in heading order until the running sum passes it: the same
// decision as the inverse CDF over all S*K controls, without storing them.
// Heading loops run over the runtime K (K a multiple of 4, all enabled).
// ---------------------------------------------------------------------------
// D_q = r^2 + sl_q^2 from the common r^2, with its rounding residual eq
// (exact: the smaller term minus what the sum kept of it, Fast2Sum).
__device__ __forceinline__ float speed_D(const HeadingTab &tab, int q, float r2, float &eq)
{
    const float sl = tab.sl[q];
    const float s2 = __fmul_rn(sl, sl);
    const float D = __fadd_rn(r2, s2);
    eq = __fsub_rn(fminf(r2, s2), __fsub_rn(D, fmaxf(r2, s2)));
    return D;
}

struct SpeedStep {
    float D[PM_MAX_SPEEDS], hD[PM_MAX_SPEEDS], c3[PM_MAX_SPEEDS], REF[PM_MAX_SPEEDS];
    float C[PM_MAX_SPEEDS];  // offset of the speed's exponents (high part)
    float SC[PM_MAX_SPEEDS]; // fixed-point scale 2^23 2^(-low part of the offset)
};

// Corrected distance of one control from the approximate square root dk of
// D + P: dk + (D + P - dk^2) / (2 d_k), with 1/(2 d_k) = hD (1 + P/D)^(-1/2)
// taken to first order, hD - 2 hD^3 P (hD = 1/(2 sqrt(D)), 1/D = 4 hD^2); a
// common 1/(2 sqrt(D)) would leave (s/r) times the square root's error, which
// beta w2 turns into 1e-4 of the logit at beta = 10^4. c3 = -2 hD^3.
__device__ __forceinline__ float corrected_minus(float D, float P, float hD, float c3, float ref)
{
    const float dk = sqrt_approx(fabsf(D + P));
    const float R = P - fmaf(dk, dk, -D);
    return fmaf(R, fmaf(P, c3, hD), dk - ref);
}

__device__ __forceinline__ uint32_t multi_weight(const HeadingTab &tab, int k, int sp, float dx, float dy,
                                                 const SpeedStep &q, float cb)
{
    const float P = __fmul_rn(fmaf(tab.tx[k], dx, tab.ty[k] * dy), tab.mult[sp]); // 2 s_s e_k.(z - g)
    const float U = corrected_minus(q.D[sp], P, q.hD[sp], q.c3[sp], q.REF[sp]);
    // <= 0 up to the rounding of REF (exact extreme form); the clamp keeps the
    // weight within 23 bits for any beta
    const float a = fminf(fmaf(U, -cb, -q.C[sp]), 0.0f);
    return __float_as_uint(fmaf(ex2_approx(a), q.SC[sp], kWMagic)) - kWBits;
}

// Exact offsets between the speeds. Each speed's D_q = r^2 + sl_q^2 is
// rounded on its own, so its residual eq_q (exact, by TwoSum from the common
// r^2) shifts that speed's distances by hD_q eq_q; the offset of speed q is
//   beta [W2 (REF_q - REF_b) + W1 (m_q - m_b)] + cb hD_q eq_q - min,
// with W2 = w2 log2(e) and W1 = w1 v dt log2(e) given as high and low floats
// and beta the component's (exact) FP32 value, carried as a high part (added
// to the exponents) and a low part (folded into the fixed-point scale), every
// product split exactly by an FMA. Without this, the independent roundings of
// the D_q (beta w2 ulp(r^2) / 2d) and of beta w2, beta w1 v dt in FP32 move
// the speeds' weights against one another.
// heq[q] = cb hD_q eq_q.
__device__ __forceinline__ void speed_offsets(const HeadingTab &tab, uint32_t speed_on, float refb, float mb,
                                              float beta, const float (&REF)[PM_MAX_SPEEDS],
                                              const float (&heq)[PM_MAX_SPEEDS], float (&hi)[PM_MAX_SPEEDS],
                                              float (&lo)[PM_MAX_SPEEDS], float bias)
{
    float cmin = INFINITY;
    const float w2h = tab.w2l[0], w2lo = tab.w2l[1], w1h = tab.w1l[0], w1lo = tab.w1l[1];
#pragma unroll
    for (int q = 0; q < PM_MAX_SPEEDS; ++q) {
        float dl, ml, xl;
        const float dr = two_sum(REF[q], -refb, dl);
        const float dm = two_sum(tab.mult[q], -mb, ml);
        const float x1 = __fmul_rn(w2h, dr), x2 = __fmul_rn(w1h, dm);
        const float x1l = __fadd_rn(fmaf(w2h, dr, -x1), fmaf(w2h, dl, __fmul_rn(w2lo, dr)));
        const float x2l = __fadd_rn(fmaf(w1h, dm, -x2), fmaf(w1h, ml, __fmul_rn(w1lo, dm)));
        const float xh = two_sum(x1, x2, xl);
        const float xlo = __fadd_rn(xl, __fadd_rn(x1l, x2l));
        const float ch = __fmul_rn(beta, xh);
        hi[q] = ch;
        lo[q] = __fadd_rn(fmaf(beta, xh, -ch), fmaf(beta, xlo, heq[q]));
        if (q < tab.S && ((speed_on >> q) & 1u)) cmin = fminf(cmin, ch);
    }
#pragma unroll
    for (int q = 0; q < PM_MAX_SPEEDS; ++q) {
        float l;
        hi[q] = two_sum(hi[q], -cmin, l);
        lo[q] = __fadd_rn(__fadd_rn(lo[q], l), bias);
    }
}

// ---------------------------------------------------------------------------
// Double-float arithmetic (a value is hi + lo, |lo| <= ulp(hi)/2: about 48
// significant bits), from the error-free transformations of Knuth (TwoSum)
// and Dekker (TwoProduct, here with one FMA). Every operation is explicitly
// rounded so that no contraction or reassociation can change it.
// ---------------------------------------------------------------------------
struct DF {
    float hi, lo;
};

__device__ __forceinline__ DF df_norm(float a, float b) // |a| >= |b| or a == 0
{
    const float s = __fadd_rn(a, b);
    return DF{s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ DF df_add(DF x, DF y)
{
    float e;
    const float s = two_sum(x.hi, y.hi, e);
    return df_norm(s, __fadd_rn(e, __fadd_rn(x.lo, y.lo)));
}

__device__ __forceinline__ DF df_neg(DF x) { return DF{-x.hi, -x.lo}; }

__device__ __forceinline__ DF df_mulf(DF x, float f)
{
    const float p = __fmul_rn(x.hi, f);
    return df_norm(p, fmaf(x.lo, f, fmaf(x.hi, f, -p)));
}

__device__ __forceinline__ DF df_mul(DF x, DF y)
{
    const float p = __fmul_rn(x.hi, y.hi);
    const float e = fmaf(x.hi, y.hi, -p);
    return df_norm(p, fmaf(x.hi, y.lo, fmaf(x.lo, y.hi, e)));
}

__device__ __forceinline__ DF df_sqrt(DF x) // x > 0: one Newton step from the rounded square root
{
    const float r = __fsqrt_rn(x.hi);
    if (!(r > 0.0f)) return DF{r, 0.0f};
    const float rr = __fmul_rn(r, r);
    const float res = __fadd_rn(__fadd_rn(__fsub_rn(x.hi, rr), -fmaf(r, r, -rr)), x.lo); // x - r^2
    return df_norm(r, __fdiv_rn(res, __fmul_rn(2.0f, r)));
}

__device__ __forceinline__ bool df_less(DF x, DF y) { return x.hi < y.hi || (x.hi == y.hi && x.lo < y.lo); }

// e^x for a double-float x <= about 88: x = n ln 2 + r with |r| <= ln(2)/2,
// e^r from its Taylor series (terms from r^6 on in FP32, where their size
// keeps the absolute error below 1e-13; the first six in double-float),
// scaled by 2^n. Relative error about 1e-13; 0 below e^-150.
__device__ __forceinline__ DF df_exp(DF x)
{
    if (x.hi < -150.0f) return DF{0.0f, 0.0f};
    const float n = rintf(__fmul_rn(x.hi, 1.44269502f));
    const DF ln2{0.693147182f, -1.90465421e-09f}; // ln 2 = hi + lo
    const DF r = df_add(x, df_neg(df_mulf(ln2, n)));
    // 1/k! for k = 12 .. 6 in FP32, Horner in r.hi
    float t = 2.08767559e-09f;
    t = fmaf(t, r.hi, 2.50521079e-08f);
    t = fmaf(t, r.hi, 2.75573200e-07f);
    t = fmaf(t, r.hi, 2.75573188e-06f);
    t = fmaf(t, r.hi, 2.48015876e-05f);
    t = fmaf(t, r.hi, 1.98412701e-04f);
    t = fmaf(t, r.hi, 1.38888892e-03f);
    // then 1/5!, 1/4!, 1/3!, 1/2!, 1, 1 in double-float
    DF p{t, 0.0f};
    const DF c5{8.33333377e-03f, -4.34617203e-10f}, c4{4.16666679e-02f, -1.24176347e-09f};
    const DF c3{1.66666672e-01f, -4.96705388e-09f}, c2{0.5f, 0.0f}, c1{1.0f, 0.0f};
    p = df_add(df_mul(p, r), c5);
    p = df_add(df_mul(p, r), c4);
    p = df_add(df_mul(p, r), c3);
    p = df_add(df_mul(p, r), c2);
    p = df_add(df_mul(p, r), c1);
    p = df_add(df_mul(p, r), c1);
    const int ni = (int)n;
    return DF{ldexpf(p.hi, ni), ldexpf(p.lo, ni)};
}

// Eq. 2 for the several-speed control set in double-float at the FP32
// particle state of lane `src`, with the inverse-CDF rule of the FP32 draws
// (the smallest u with u24 2^-24 S < C_u), computed by the whole warp: lane L
// takes the controls [L per, L per + per) (per = ceil(U / 32)), a warp scan
// of the lanes' sums gives the running sums, and the first lane whose range
// holds the threshold names the control. Logits beta Q_u, Q_u = -w1 v m_q
// dt - w2 ||z + v m_q dt e_k - g||, shifted by the logit of the control
// `guess` (the FP32 draw's choice, whose weight is within 2^-23 of the
// largest, so no weight overflows), with the unit heading vectors of the
// double-float table. The several-speed draws ask for it only for a step
// whose FP32 threshold falls within the error band of a CDF boundary (a few
// in 10^6 steps), so that their decision does not rest on FP32 rounding
// there: with 96 nearly equal weights (small |beta|) the ex2 and fixed-point
// errors move the CDF by a few 10^-9; at |beta| ~ 10^4 the FP32 heading
// table and products move the logits between speeds by ~3e-5. Every lane of
// the warp must call it with the same src. Not inlined: its registers stay
// out of the hot loop.
static __device__ __noinline__ int settle_multi_warp(const HeadingTab &tab, uint32_t speed_on, int K, float x,
                                                     float y, float gx, float gy, float beta, uint32_t word,
                                                     int guess, int src)
{
    constexpr unsigned kAll = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    x = __shfl_sync(kAll, x, src);
    y = __shfl_sync(kAll, y, src);
    gx = __shfl_sync(kAll, gx, src);
    gy = __shfl_sync(kAll, gy, src);
    beta = __shfl_sync(kAll, beta, src);
    word = __shfl_sync(kAll, word, src);
    guess = __shfl_sync(kAll, guess, src);
    float ex_lo, ey_lo;
    const float ex_hi = two_sum(x, -gx, ex_lo), ey_hi = two_sum(y, -gy, ey_lo);
    const DF zgx{ex_hi, ex_lo}, zgy{ey_hi, ey_lo};
    const int U = tab.S * K;
    auto logit = [&](int u) {
        const int q = u / K, k = u - q * K;
        const DF st = df_mulf(df_mulf(DF{tab.v, 0.0f}, tab.mult[q]), tab.dt); // v m_q dt
        const DF dx = df_add(zgx, df_mul(st, DF{tab.cdf[k][0], tab.cdf[k][1]}));
        const DF dy = df_add(zgy, df_mul(st, DF{tab.sdf[k][0], tab.sdf[k][1]}));
        const DF d = df_sqrt(df_add(df_mul(dx, dx), df_mul(dy, dy)));
        const DF Q = df_neg(df_add(df_mulf(st, tab.w1), df_mulf(d, tab.w2)));
        return df_mulf(Q, beta);
    };
    const DF shift = df_neg(logit(guess));
    const int per = (U + 31) / 32; // at most 8 (U <= 256)
    DF e[8];
    DF bs{0.0f, 0.0f};
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        e[j] = DF{0.0f, 0.0f};
        const int u = lane * per + j;
        if (j < per && u < U && ((speed_on >> (u / K)) & 1u)) {
            e[j] = df_exp(df_add(logit(u), shift));
            bs = df_add(bs, e[j]);
        }
    }
    DF incl = bs; // inclusive scan over the lanes, earlier lanes first
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const DF v{__shfl_up_sync(kAll, incl.hi, o), __shfl_up_sync(kAll, incl.lo, o)};
        if (lane >= o) incl = df_add(v, incl);
    }
    DF C{__shfl_up_sync(kAll, incl.hi, 1), __shfl_up_sync(kAll, incl.lo, 1)};
    if (lane == 0) C = DF{0.0f, 0.0f};
    const DF S{__shfl_sync(kAll, incl.hi, 31), __shfl_sync(kAll, incl.lo, 31)};
    const DF target = df_mulf(S, (float)(word >> 8) * 0x1p-24f);
    int cand = -1, lastpos = -1;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const int u = lane * per + j;
        if (j < per && u < U) {
            if (e[j].hi > 0.0f) lastpos = u;
            C = df_add(C, e[j]);
            if (cand < 0 && e[j].hi > 0.0f && df_less(target, C)) cand = u;
        }
    }
    const unsigned has = __ballot_sync(kAll, cand >= 0);
    if (has) return __shfl_sync(kAll, cand, __ffs(has) - 1);
    // rounding left the threshold at the total: the last control with weight
    const unsigned pos = __ballot_sync(kAll, lastpos >= 0);
    return pos ? __shfl_sync(kAll, lastpos, 31 - __clz(pos)) : guess;
}

// Whether an FP32 draw's threshold thr lies clear of both boundaries of the
// chosen interval [lo, hi) of the fixed-point CDF (total S): by more than 24
// units (the ex2 and quantisation errors of up to 256 weights accumulate to
// a standard deviation of about 4 units at a boundary) plus |cb| S 2^-26
// (the FP32 distance and table errors, a few 1e-9 m, turned into relative
// weight errors by |cb| ln 2, with a factor 10 to spare).
__device__ __forceinline__ bool draw_is_clear(uint32_t thr, uint32_t lo, uint32_t hi, uint32_t S, float cb)
{
    const float band = fmaf((float)S * 0x1p-26f, fabsf(cb), 24.0f);
    return (float)(thr - lo) >= band && (float)(hi - 1u - thr) >= band;
}

__device__ __forceinline__ int draw_multi(const HeadingTab &tab, uint32_t speed_on, int K, float x, float y,
                                          float gx, float gy, float beta, float cb, float cw1, bool lb,
                                          uint32_t word, bool &settle)
{
    const float dx = x - gx, dy = y - gy;
    const float r2 = fmaf(dx, dx, dy * dy); // common to every speed
    const float r = sqrt_approx(r2);
    SpeedStep q;
    float eq[PM_MAX_SPEEDS];
    int best = max(__ffs((int)speed_on) - 1, 0); // an enabled speed, whatever the inputs
    float vbest = -INFINITY, refb = 0.0f, mb = tab.mult[0];
#pragma unroll
    for (int sp = 0; sp < PM_MAX_SPEEDS; ++sp) {
        q.D[sp] = q.hD[sp] = q.c3[sp] = q.REF[sp] = q.C[sp] = eq[sp] = 0.0f;
        q.SC[sp] = 0.0f;
        if (sp >= tab.S || !((speed_on >> sp) & 1u)) continue;
        const float sl = tab.sl[sp];
        q.D[sp] = speed_D(tab, sp, r2, eq[sp]);
        q.hD[sp] = 0.5f * rsqrt_approx(q.D[sp]);
        q.c3[sp] = -2.0f * q.hD[sp] * q.hD[sp] * q.hD[sp];
        eq[sp] = __fmul_rn(__fmul_rn(cb, q.hD[sp]), eq[sp]); // cb hD eq
        if (lb) {
            const float margin = (r + sl) * 0x1p-20f;
            q.REF[sp] = (cb >= 0.0f) ? fabsf(r - sl) - margin : r + sl + margin;
        } else {
            // the exact extreme of the corrected distances of this speed
            float ext = (cb >= 0.0f) ? INFINITY : -INFINITY;
            q.REF[sp] = 0.0f;
            for (int k = 0; k < K; ++k) {
                const float P = __fmul_rn(fmaf(tab.tx[k], dx, tab.ty[k] * dy), tab.mult[sp]);
                const float d = corrected_minus(q.D[sp], P, q.hD[sp], q.c3[sp], 0.0f);
                ext = (cb >= 0.0f) ? fminf(ext, d) : fmaxf(ext, d);
            }
            q.REF[sp] = ext;
        }
        const float v = -fmaf(cb, q.REF[sp], cw1 * tab.mult[sp]);
        if (v > vbest) {
            vbest = v;
            best = sp;
            refb = q.REF[sp];
            mb = tab.mult[sp];
        }
    }
    // offsets between speeds (high part in the exponent, low part in the
    // scale); a common factor 2^-2^-18 on every weight keeps the largest one
    // below 2^23 whatever the sign of the low parts (it does not change the
    // distribution)
    float lo[PM_MAX_SPEEDS];
    speed_offsets(tab, speed_on, refb, mb, beta, q.REF, eq, q.C, lo, 0x1p-18f);
    uint32_t W[PM_MAX_SPEEDS];
    uint32_t total = 0u;
#pragma unroll
    for (int sp = 0; sp < PM_MAX_SPEEDS; ++sp) {
        W[sp] = 0u;
        if (sp >= tab.S || !((speed_on >> sp) & 1u)) continue;
        q.SC[sp] = kWScale * exp2f(-lo[sp]);
        uint32_t w = 0u;
        for (int k = 0; k < K; ++k) w += multi_weight(tab, k, sp, dx, dy, q, cb);
        W[sp] = w;
        total += w;
    }
    const uint32_t thr = (uint32_t)(((uint64_t)(word >> 8) * (uint64_t)total) >> 24);
    // the speed whose running-sum interval holds thr (total > thr always)
    uint32_t C0 = 0u;
    int ss = best;
    {
        uint32_t run = 0u;
        bool found = false;
#pragma unroll
        for (int sp = 0; sp < PM_MAX_SPEEDS; ++sp) {
            if (!found && sp < tab.S && ((speed_on >> sp) & 1u)) {
                if (thr < run + W[sp]) {
                    ss = sp;
                    C0 = run;
                    found = true;
                } else {
                    run += W[sp];
                }
            }
        }
    }
    // that speed's headings in order until the running sum passes thr
    uint32_t acc = C0, below = C0;
    int kk = K - 1;
    bool hit = false;
    for (int k = 0; k < K; ++k) {
        below = acc;
        acc += multi_weight(tab, k, ss, dx, dy, q, cb);
        if (thr < acc) {
            kk = k;
            hit = true;
            break;
        }
    }
    settle = !hit || !draw_is_clear(thr, below, acc, total, cb);
    return ss * K + kk;
}

// The several-speed draw fused like draw_heading_lb, for KT headings all
// enabled (KT % 4 == 0) and a component with the bound-normalised flag.
// Per enabled speed q the loop is the one-speed loop with that speed's
// constants: P_{k,q} = 2 s e_k.(m_q (z - g)) (the scaled offset rounded once,
// so heading k + K/2 still has exactly -P), D_q = ||z - g||^2 + sl_q^2 (from
// the common ||z - g||^2; its rounding residual is part of the offset) and
// the bound REF_q of that speed. The exponent of control (q, k) is
//   -cb (d_{k,q} - REF_q) - C_q,   C_q = cb (REF_q - REF_b) + cw1 (m_q - m_b) - min,
// evaluated as fma(R, -cb/2d, fma(d~, -cb, RC_q)) with RC_q = round(cb REF_q);
// the rounding e_q of RC_q, the shift -cb/(2d) eq_q of the residual eq_q of
// D_q and the offset C_q are folded into the fixed-point scale
// 2^23 2^(e_q - cb eq_q/2d - C_q), so they cost nothing per control and the
// independent roundings of the D_q do not move the speeds against one
// another (by beta w2 ulp(r^2)/2d, 1e-5 of the logit at beta = 100 and r = 5
// m, before this correction). Pass 1 keeps segment sums of G
// headings per speed (the bits are not stored); the threshold picks the
// segment and pass 2 recomputes only its G weights, bit for bit.
template <int KT>
struct MultiLbConsts {
    float D, HDNC, RC, SC, mx, my; // D_q, -cb/(2 d_q), round(cb REF_q), scale, m_q (z - g)
};


// The residual eq of D_q shifts every exponent of the speed by HDNC eq (the
// distances' residual correction of the exact D_q); it goes into the scale
// with the rounding e of RC and the speed's offset C.
template <int KT>
__device__ __forceinline__ MultiLbConsts<KT> multi_lb_consts(const HeadingTab &tab, int q, float r2, float dx,
                                                             float dy, float cb, float REF, float C)
{
    MultiLbConsts<KT> c;
    float eq;
    c.D = speed_D(tab, q, r2, eq);
    c.HDNC = -cb * (0.5f * rsqrt_approx(c.D));
    c.RC = cb * REF;
    const float e = fmaf(cb, REF, -c.RC); // cb REF - RC, exact
    c.SC = kWScale * exp2f(fmaf(c.HDNC, eq, e) - C);
    c.mx = __fmul_rn(dx, tab.mult[q]);
    c.my = __fmul_rn(dy, tab.mult[q]);
    return c;
}

// Fixed-point weight of heading k under the constants of one speed (pass 2).
template <int KT>
__device__ __forceinline__ uint32_t multi_lb_weight(const HeadingTab &tab, int k, const MultiLbConsts<KT> &c,
                                                    float cb)
{
    const float P = fmaf(tab.tx[k], c.mx, __fmul_rn(tab.ty[k], c.my));
    const float d = sqrt_approx(fabsf(c.D + P));
    const float a = fmaf(P - fmaf(d, d, -c.D), c.HDNC, fmaf(d, -cb, c.RC));
    return __float_as_uint(fmaf(ex2_approx(a), c.SC, kWMagic)) - kWBits;
}

template <int KT>
__device__ __forceinline__ int draw_multi_lb(const HeadingTab &tab, uint32_t speed_on, float x, float y, float gx,
                                             float gy, float beta, float cb, float cw1, uint32_t word, bool &settle)
{
    static_assert(KT % 4 == 0, "pairs of headings must not straddle the two halves");
    constexpr int G = CdfSegs<KT>::G, NS = KT / G, H2 = KT / 2;
    const float dx = x - gx, dy = y - gy;
    const float r2 = fmaf(dx, dx, dy * dy); // common to every speed
    const float r = sqrt_approx(r2);
    // bounds per speed and the offsets between speeds
    float REF[PM_MAX_SPEEDS], C[PM_MAX_SPEEDS];
    float vbest = -INFINITY, refb = 0.0f, mb = 0.0f;
#pragma unroll
    for (int q = 0; q < PM_MAX_SPEEDS; ++q) {
        const float sl = tab.sl[q];
        const float margin = (r + sl) * 0x1p-20f;
        REF[q] = (cb >= 0.0f) ? fabsf(r - sl) - margin : r + sl + margin;
        const float v = -fmaf(cb, REF[q], cw1 * tab.mult[q]);
        if (q < tab.S && ((speed_on >> q) & 1u) && v > vbest) {
            vbest = v;
            refb = REF[q];
            mb = tab.mult[q];
        }
    }
    float cmin = INFINITY;
#pragma unroll
    for (int q = 0; q < PM_MAX_SPEEDS; ++q) {
        C[q] = fmaf(cb, REF[q] - refb, cw1 * (tab.mult[q] - mb));
        if (q < tab.S && ((speed_on >> q) & 1u)) cmin = fminf(cmin, C[q]);
    }
    const f32x2 NC = f2_pack(-cb, -cb), MG = f2_pack(kWMagic, kWMagic);
    const f32x2 *TX = reinterpret_cast<const f32x2 *>(tab.tx);
    const f32x2 *TY = reinterpret_cast<const f32x2 *>(tab.ty);
    uint32_t seg[PM_MAX_SPEEDS][NS];
#pragma unroll
    for (int q = 0; q < PM_MAX_SPEEDS; ++q) {
#pragma unroll
        for (int i = 0; i < NS; ++i) seg[q][i] = 0u;
        if (q >= tab.S || !((speed_on >> q) & 1u)) continue;
        const MultiLbConsts<KT> c = multi_lb_consts<KT>(tab, q, r2, dx, dy, cb, REF[q], C[q] - cmin);
        const f32x2 MX = f2_pack(c.mx, c.mx), MY = f2_pack(c.my, c.my);
        const f32x2 DD = f2_pack(c.D, c.D), NDD = f2_pack(-c.D, -c.D);
        const f32x2 HDNC = f2_pack(c.HDNC, c.HDNC), NHDNC = f2_pack(-c.HDNC, -c.HDNC);
        const f32x2 RC = f2_pack(c.RC, c.RC), SC = f2_pack(c.SC, c.SC);
#pragma unroll
        for (int k2 = 0; k2 < KT / 4; ++k2) {
            const f32x2 P = f2_fma(TX[k2], MX, f2_mul(TY[k2], MY)); // headings 2k2, 2k2+1; -P for + K/2
            float x0, x1, y0, y1;
            f2_unpack(f2_add(DD, P), x0, x1);
            f2_unpack(f2_sub(DD, P), y0, y1);
            const f32x2 DA = f2_pack(sqrt_approx(fabsf(x0)), sqrt_approx(fabsf(x1)));
            const f32x2 DB = f2_pack(sqrt_approx(fabsf(y0)), sqrt_approx(fabsf(y1)));
            float a0, a1, b0, b1;
            f2_unpack(f2_fma(f2_sub(P, f2_fma(DA, DA, NDD)), HDNC, f2_fma(DA, NC, RC)), a0, a1);
            f2_unpack(f2_fma(f2_add(P, f2_fma(DB, DB, NDD)), NHDNC, f2_fma(DB, NC, RC)), b0, b1);
            float w0, w1, v0, v1;
            f2_unpack(f2_fma(f2_pack(ex2_approx(a0), ex2_approx(a1)), SC, MG), w0, w1);
            f2_unpack(f2_fma(f2_pack(ex2_approx(b0), ex2_approx(b1)), SC, MG), v0, v1);
            seg[q][(2 * k2) / G] += (__float_as_uint(w0) - kWBits) + (__float_as_uint(w1) - kWBits);
            seg[q][(H2 + 2 * k2) / G] += (__float_as_uint(v0) - kWBits) + (__float_as_uint(v1) - kWBits);
        }
    }
    uint32_t S = 0u;
#pragma unroll
    for (int q = 0; q < PM_MAX_SPEEDS; ++q)
#pragma unroll
        for (int i = 0; i < NS; ++i) S += seg[q][i];
    const uint32_t thr = (uint32_t)(((uint64_t)(word >> 8) * (uint64_t)S) >> 24);
    // the segment whose running-sum interval holds thr
    int qs = 0, is = NS - 1;
    uint32_t C0 = 0u, run = 0u;
    bool found = false;
#pragma unroll
    for (int q = 0; q < PM_MAX_SPEEDS; ++q)
#pragma unroll
        for (int i = 0; i < NS; ++i) {
            const bool hit = !found && thr < run + seg[q][i];
            qs = hit ? q : qs;
            is = hit ? i : is;
            C0 = hit ? run : C0;
            found = found || hit;
            run += seg[q][i];
        }
    if (!found) { // S == 0: only for non-finite inputs; any valid control
        qs = max(__ffs((int)speed_on) - 1, 0);
        is = NS - 1;
        C0 = 0u;
    }
    float REFs = REF[0], Cs = C[0];
#pragma unroll
    for (int q = 1; q < PM_MAX_SPEEDS; ++q) {
        REFs = (qs == q) ? REF[q] : REFs;
        Cs = (qs == q) ? C[q] : Cs;
    }
    const MultiLbConsts<KT> c = multi_lb_consts<KT>(tab, qs, r2, dx, dy, cb, REFs, Cs - cmin);
    uint32_t acc = C0, below = C0;
    int kk = is * G + G - 1;
    bool hit = false;
    for (int k = is * G; k < is * G + G; ++k) {
        below = acc;
        acc += multi_lb_weight<KT>(tab, k, c, cb);
        if (thr < acc) {
            kk = k;
            hit = true;
            break;
        }
    }
    settle = !hit || !draw_is_clear(thr, below, acc, S, cb);
    return qs * KT + kk;
}

// Per-tile state of one human for rollout_tile.
struct TileCtx {
    float z0x, z0y;
    int T;
    int64_t i;       // the first particle of this thread (the others follow at +blockDim)
    int64_t N;       // particles of the human: indices >= N are idle
    int64_t n_trace; // particles below this index record their trajectory
    uint64_t seed;
    uint32_t human;
    int J;
    bool hist;
    float gx0, gy0, inv_res; // grid the states are binned on
    int W, H;                // output cells
    int cx_off, cy_off;      // output cell = grid cell - offset
    uint32_t *counts;
    uint32_t *oob;
    int win_x0, win_y0, ww, wh; // shared-memory window, output cells (window mode)
    float *tr_states;
    uint8_t *tr_head;
    int32_t *tr_comp;
    uint8_t *flags; // block occupancy [T][fby][fbx] (warp emplacement), or NULL
    int fbx;
    int fplane;     // fbx * fby
};

// Words of one shared-memory window of ww x wh 16-bit counts, padded to 16 B.
__device__ __host__ __forceinline__ int window_stride_words(int ww, int wh)
{
    return (((ww * wh + 1) >> 1) + 3) & ~3;
}

// Algorithm 1 for PPT particles per thread of the CTA (particles i, i+blockDim,
// ...; independent chains the scheduler interleaves): the (beta, g) draw from
// the belief table in shared memory, then T heading draws and Euler steps.
//
// Emplacement, two modes:
//  - WARP_HIST: the lanes of a warp that fall in the same cell at step t are
//    combined (match.any) and their leader adds the count to global memory
//    with one reduction; no shared window, no block barrier.
//  - window: each step is counted in the CTA's shared-memory window (first
//    touch appends the cell to the step's list; after one block barrier the
//    list is flushed with one global reduction per touched cell); cells
//    outside the window go straight to global memory. Two windows and two
//    lists alternate by step parity and three list counters rotate, so the
//    flush of step t overlaps the inserts of step t+1. `sh` must hold the
//    human's tables; both windows, list_n[0..2] and oob_n[0..1] must be zero
//    on entry; the windows are zero again on exit. dyn layout: window 0 |
//    window 1 (window_stride_words each) | list 0 | list 1 (PPT*blockDim each).
template <int KT, bool FULL, int PPT, bool WARP_HIST>
__device__ __forceinline__ void rollout_tile(const HeadingTab &tab, uint64_t enabled, float s2,
                                             const TileCtx &c, RolloutShared &sh, uint32_t *dyn)
{
    const int tid = threadIdx.x;
    const int nthr = blockDim.x;
    const int ww = c.ww, wh = c.wh;
    const int stride = window_stride_words(ww, wh);
    uint16_t *list0 = reinterpret_cast<uint16_t *>(dyn + 2 * stride);
    const int list_cap = PPT * nthr;

    float x[PPT], y[PPT], cb[PPT], gx[PPT], gy[PPT];
    uint64_t ip[PPT];
    bool act[PPT], trc[PPT], lb[PPT];
    uint32_t q[PPT][8];
#pragma unroll
    for (int p = 0; p < PPT; ++p) {
        ip[p] = (uint64_t)c.i + (uint64_t)p * nthr;
        act[p] = (int64_t)ip[p] < c.N;
        trc[p] = (int64_t)ip[p] < c.n_trace;
        x[p] = c.z0x;
        y[p] = c.z0y;
        cb[p] = gx[p] = gy[p] = 0.0f;
        lb[p] = false;
#pragma unroll
        for (int w = 0; w < 8; ++w) q[p][w] = 0u;
        if (act[p]) {
            const U64x4 r = philox4x64_10(U64x4{ip[p], 0ull, kPurposeSelect, 0ull}, c.seed, c.human);
            const uint32_t thr = (uint32_t)(((uint64_t)((uint32_t)r.a >> 8) * (uint64_t)sh.cdf[c.J - 1]) >> 24);
            int lo = 0, hi = c.J - 1; // smallest j with cdf[j] > thr
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (sh.cdf[mid] > thr) hi = mid;
                else lo = mid + 1;
            }
            const float4 cc = sh.comp[lo];
            cb[p] = cc.x;
            gx[p] = cc.y;
            gy[p] = cc.z;
            lb[p] = cc.w != 0.0f;
            if (trc[p] && c.tr_comp) c.tr_comp[ip[p]] = lo;
        }
    }

    const size_t plane = (size_t)c.W * (size_t)c.H;
    int li = 1; // t mod 3: the list counter of step t (window mode)
    for (int t = 1; t <= c.T; ++t) {
        int cx[PPT], cy[PPT];
        bool ing[PPT];
#pragma unroll
        for (int p = 0; p < PPT; ++p) {
            cx[p] = cy[p] = 0;
            ing[p] = false;
            if (act[p]) {
                if (((t - 1) & 7) == 0) {
                    const U64x4 r = philox4x64_10(U64x4{ip[p], (uint64_t)((t - 1) >> 3), kPurposeStep, 0ull},
                                                  c.seed, c.human);
                    q[p][0] = (uint32_t)r.a; q[p][1] = (uint32_t)(r.a >> 32);
                    q[p][2] = (uint32_t)r.b; q[p][3] = (uint32_t)(r.b >> 32);
                    q[p][4] = (uint32_t)r.c; q[p][5] = (uint32_t)(r.c >> 32);
                    q[p][6] = (uint32_t)r.d; q[p][7] = (uint32_t)(r.d >> 32);
                }
                const uint32_t word = q[p][0];
#pragma unroll
                for (int w = 0; w < 7; ++w) q[p][w] = q[p][w + 1];
                const int k = draw<KT, FULL>(tab, enabled, s2, x[p], y[p], gx[p], gy[p], cb[p], lb[p], word);
                const float2 st = sh.step[k];
                x[p] = __fadd_rn(x[p], st.x);
                y[p] = __fadd_rn(y[p], st.y);
                if (trc[p]) {
                    const size_t o = (size_t)ip[p] * c.T + (t - 1);
                    if (c.tr_states) reinterpret_cast<float2 *>(c.tr_states)[o] = make_float2(x[p], y[p]);
                    if (c.tr_head) c.tr_head[o] = (uint8_t)k;
                }
                if (c.hist) {
                    const float vx = __fmul_rn(__fsub_rn(x[p], c.gx0), c.inv_res);
                    const float vy = __fmul_rn(__fsub_rn(y[p], c.gy0), c.inv_res);
                    cx[p] = __float2int_rd(vx) - c.cx_off;
                    cy[p] = __float2int_rd(vy) - c.cy_off;
                    ing[p] = (vx == vx) && (vy == vy) && cx[p] >= 0 && cx[p] < c.W && cy[p] >= 0 && cy[p] < c.H;
                }
            }
        }
        if (c.hist) {
            if constexpr (WARP_HIST) {
                const int lane = tid & 31;
#pragma unroll
                for (int p = 0; p < PPT; ++p) {
                    const uint32_t key = !act[p] ? 0xFFFFFFFFu : (ing[p] ? (uint32_t)(cy[p] * c.W + cx[p]) : 0xFFFFFFFEu);
                    const uint32_t peers = __match_any_sync(0xffffffffu, key);
                    if (key != 0xFFFFFFFFu && (__ffs(peers) - 1) == lane) {
                        if (key == 0xFFFFFFFEu) red_add(c.oob + (t - 1), (uint32_t)__popc(peers));
                        else red_add(c.counts + (size_t)(t - 1) * plane + key, (uint32_t)__popc(peers));
                    }
                }
            } else {
                const int b = t & 1;
                uint32_t *win32 = dyn + b * stride;
                uint16_t *win16 = reinterpret_cast<uint16_t *>(win32);
                uint16_t *list = list0 + b * list_cap;
#pragma unroll
                for (int p = 0; p < PPT; ++p) {
                    if (!act[p]) continue;
                    if (!ing[p]) {
                        atomicAdd(&sh.oob_n[b], 1u);
                        continue;
                    }
                    const int wx = cx[p] - c.win_x0, wy = cy[p] - c.win_y0;
                    if ((unsigned)wx < (unsigned)ww && (unsigned)wy < (unsigned)wh) {
                        const int w = wy * ww + wx;
                        const uint32_t sft = (uint32_t)(w & 1) << 4;
                        const uint32_t old = atomicAdd(&win32[w >> 1], 1u << sft);
                        if (((old >> sft) & 0xFFFFu) == 0u) {
                            const uint32_t slot = atomicAdd(&sh.list_n[li], 1u);
                            list[slot] = (uint16_t)(wx | (wy << 8));
                        }
                    } else {
                        red_add(c.counts + (size_t)(t - 1) * plane + (size_t)cy[p] * c.W + cx[p], 1u);
                    }
                }
                __syncthreads(); // all of step t is in window b; step t-1's flush is done
                const int lr = (li == 0) ? 2 : li - 1; // counter of step t-1: free from here on
                if (tid == 0) sh.list_n[lr] = 0u;
                const uint32_t n = sh.list_n[li];
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
                    const uint32_t o = sh.oob_n[b];
                    if (o) red_add(c.oob + (t - 1), o);
                    sh.oob_n[b] = 0u;
                }
            }
        }
        li = (li == 2) ? 0 : li + 1;
    }
}
// Algorithm 1 for the particle of one lane: the (beta, g) draw from the
// belief table (comp, cdf), then T heading draws and Euler steps, each step
// emplaced with the lanes of the warp that land in the same cell combined
// (match.any) into one global reduction. Every lane of the warp must call
// it with the same c.T (idle lanes pass c.i >= c.N). No block barrier.
// MS: the control set of several speeds (betas holds each component's beta,
// step the S*K Euler steps, K the headings, speed_on the enabled speeds); KT >
// 0 is then K itself, with draw_multi_lb for the components it applies to,
// and KT = 0 runs draw_multi for any K.
template <int KT, bool FULL, bool MS = false>
__device__ __forceinline__ void rollout_lane(const HeadingTab &tab, uint64_t enabled, float s2, const TileCtx &c,
                                             const float4 *comp, const uint32_t *cdf, const float2 *step,
                                             const float *betas = nullptr, int K = 0, uint32_t speed_on = 0u)
{
    const int lane = threadIdx.x & 31;
    const uint64_t i = (uint64_t)c.i;
    const bool act = c.i < c.N;
    const bool trc = c.i < c.n_trace;
    float x = c.z0x, y = c.z0y, cb = 0.0f, gx = 0.0f, gy = 0.0f, cw = 0.0f, bt = 0.0f;
    bool lb = false;
    // several speeds with exactly one enabled: its index (else -1)
    const int one_speed = (MS && __popc(speed_on) == 1) ? __ffs((int)speed_on) - 1 : -1;
    if (act) {
        const U64x4 r = philox4x64_10(U64x4{i, 0ull, kPurposeSelect, 0ull}, c.seed, c.human);
        const uint32_t thr = (uint32_t)(((uint64_t)((uint32_t)r.a >> 8) * (uint64_t)cdf[c.J - 1]) >> 24);
        int lo = 0, hi = c.J - 1; // smallest j with cdf[j] > thr
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (cdf[mid] > thr) hi = mid;
            else lo = mid + 1;
        }
        const float4 cc = comp[lo];
        cb = cc.x;
        gx = cc.y;
        gy = cc.z;
        lb = cc.w != 0.0f;
        if constexpr (MS) {
            bt = betas[lo];
            cw = bt * tab.w1l[0]; // beta w1 v dt log2(e)
        }
        if (trc && c.tr_comp) c.tr_comp[i] = lo;
    }
    const size_t plane = (size_t)c.W * (size_t)c.H;
    uint32_t q0 = 0, q1 = 0, q2 = 0, q3 = 0, q4 = 0, q5 = 0, q6 = 0, q7 = 0;
    for (int t = 1; t <= c.T; ++t) {
        uint32_t key = 0xFFFFFFFFu; // idle lane
        int fkey = 0;               // block of the cell (flags only)
        int k = 0;
        bool settle = false; // several speeds: the FP32 draw was too close to a CDF boundary
        uint32_t word = 0u;
        if (act) {
            if (((t - 1) & 7) == 0) {
                const U64x4 r = philox4x64_10(U64x4{i, (uint64_t)((t - 1) >> 3), kPurposeStep, 0ull}, c.seed, c.human);
                q0 = (uint32_t)r.a; q1 = (uint32_t)(r.a >> 32);
                q2 = (uint32_t)r.b; q3 = (uint32_t)(r.b >> 32);
                q4 = (uint32_t)r.c; q5 = (uint32_t)(r.c >> 32);
                q6 = (uint32_t)r.d; q7 = (uint32_t)(r.d >> 32);
            }
            word = q0;
            q0 = q1; q1 = q2; q2 = q3; q3 = q4; q4 = q5; q5 = q6; q6 = q7;
            if constexpr (MS) {
                if constexpr (KT > 0) { // K == KT, all headings enabled: the fused form where it applies
                    if (lb && one_speed >= 0) {
                        // one enabled speed m (a human standing still keeps only the
                        // slow one): ||z + s m e_k - g|| = m ||(z - g) / m + s e_k||, so
                        // the one-speed draw at the scaled offset with cb m draws the
                        // same policy (the speed term is common to every control)
                        const float im = tab.inv_mult[one_speed], cbm = cb * tab.mult[one_speed];
                        k = one_speed * KT +
                            draw_heading_lb<KT>(tab, lb_step_d(tab, s2, (x - gx) * im, (y - gy) * im, cbm), cbm, word);
                    } else if (lb) {
                        k = draw_multi_lb<KT>(tab, speed_on, x, y, gx, gy, bt, cb, cw, word, settle);
                    } else {
                        k = draw_multi(tab, speed_on, K, x, y, gx, gy, bt, cb, cw, lb, word, settle);
                    }
                } else {
                    k = draw_multi(tab, speed_on, K, x, y, gx, gy, bt, cb, cw, lb, word, settle);
                }
            } else {
                k = draw<KT, FULL>(tab, enabled, s2, x, y, gx, gy, cb, lb, word);
            }
        }
        if constexpr (MS) {
            // a draw too close to a CDF boundary for FP32 is settled in
            // double-float by the whole warp, one flagged lane at a time
            unsigned need = __ballot_sync(0xffffffffu, settle);
            while (need) {
                const int src = __ffs((int)need) - 1;
                const int u = settle_multi_warp(tab, speed_on, K, x, y, gx, gy, bt, word, k, src);
                if (lane == src) k = u;
                need &= need - 1u;
            }
        }
        if (act) {
            const float2 st = step[k];
            x = __fadd_rn(x, st.x);
            y = __fadd_rn(y, st.y);
            if (trc) {
                const size_t o = (size_t)i * c.T + (t - 1);
                if (c.tr_states) reinterpret_cast<float2 *>(c.tr_states)[o] = make_float2(x, y);
                if (c.tr_head) c.tr_head[o] = (uint8_t)k;
            }
            if (c.hist) {
                const float vx = __fmul_rn(__fsub_rn(x, c.gx0), c.inv_res);
                const float vy = __fmul_rn(__fsub_rn(y, c.gy0), c.inv_res);
                // floor(v) for |v| < 2^22 on the FP32 pipe: v + 1.5 * 2^23 rounded
                // down is exact and holds floor(v) in its low mantissa bits;
                // larger |v| and NaN are outside every grid (W, H <= 2^22)
                const int cx = (__float_as_int(__fadd_rd(vx, 12582912.0f)) - 0x4B400000) - c.cx_off;
                const int cy = (__float_as_int(__fadd_rd(vy, 12582912.0f)) - 0x4B400000) - c.cy_off;
                const bool in = fabsf(vx) < 4194304.0f && fabsf(vy) < 4194304.0f && cx >= 0 && cx < c.W &&
                                cy >= 0 && cy < c.H;
                key = in ? (uint32_t)(cy * c.W + cx) : 0xFFFFFFFEu;
                if (c.flags) fkey = (cy >> kFlagShift) * c.fbx + (cx >> kFlagShift);
            }
        }
        if (c.hist) {
            const uint32_t peers = __match_any_sync(0xffffffffu, key);
            // the lowest lane of each group of equal keys adds the group's size
            if (key != 0xFFFFFFFFu && (peers & ((1u << lane) - 1u)) == 0u) {
                if (key == 0xFFFFFFFEu) {
                    red_add(c.oob + (t - 1), (uint32_t)__popc(peers));
                } else {
                    red_add(c.counts + (size_t)(t - 1) * plane + key, (uint32_t)__popc(peers));
                    if (c.flags) c.flags[(size_t)(t - 1) * c.fplane + fkey] = 1u; // idempotent
                }
            }
        }
    }
}

} // namespace pm
