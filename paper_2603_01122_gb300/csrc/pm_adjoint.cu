// pm_adjoint.cu -- marginal log-likelihood of observed trajectories under the
// Boltzmann model (Eq. 2) with the joint prior over (beta, g) of Eq. 3, and
// its gradient with respect to the goal coordinates, the walking speed v and
// the Q weights (w1, w2):
//
//   L = sum_m log sum_j exp(log prior_j + A_mj),  A_mj = sum_t log pi_j(u_mt | z_mt)
//   dL/dp = sum_m sum_j w_mj sum_t d log pi_j / dp,  w_mj = softmax_j(log prior_j + A_mj)
//   d log pi / dp = beta (dQ(theta_obs)/dp - sum_k pi_k dQ(theta_k)/dp)
//   dQ/dg = w2 u, dQ/dv = -w1 dt - w2 dt e.u, dQ/dw1 = -v dt, dQ/dw2 = -d,
//   with d = ||z + v dt e - g|| and u = (z + v dt e - g) / d; with several
//   speeds (Sec. IV-B) each control carries its multiplier m_q in the step
//   and in these derivatives, which makes dL/dw1 nonzero.
//
// A CTA per (trajectory, group of eight components); a warp per component
// (beta, g) with its lanes over the trajectory's steps and the headings
// unrolled in registers. The
// per-step log pi is FP32; its sum over a trajectory (up to hundreds of
// steps of about -log K each) is accumulated in FP64, the one place where
// FP32 would lose the differences between components. Per-trajectory
// partials go to scratch; the last CTA to finish (ticket, no waiting) sums
// them over trajectories in a fixed order and writes the outputs.
#include <cuda_runtime.h>

#include "pm_kernels.cuh"

namespace pm {
namespace {

constexpr int kAdjThreads = 256;
constexpr float kLog2e = 1.4426950408889634f, kLn2 = 0.6931471805599453f;

__device__ __forceinline__ float wsum(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ double wsum_d(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ double wmax_d(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

struct StepGrad {
    float logpi, gx, gy, gv, gw1, gw2;
};

// log pi_j(theta_obs | z) and its derivatives for one observed step.
template <int KT>
__device__ __forceinline__ StepGrad step_terms(const AdjointArgs &a, float zx, float zy, float ex, float ey,
                                               float gx, float gy, float beta, bool grad)
{
    const float px = zx - gx, py = zy - gy;
    const float D = fmaf(px, px, fmaf(py, py, a.s2));
    const float xo = fmaxf(D + a.two_s * fmaf(ex, px, ey * py), 0.0f);
    const float ro = rsqrtf(fmaxf(xo, 1e-30f));
    const float d_o = xo * ro;
    const float bw = beta * a.w2;
    const float bw2 = bw * kLog2e; // logits in base 2: exponentials on the SFU
    float lg[KT];
    float m = -INFINITY;
#pragma unroll
    for (int k = 0; k < KT; ++k) {
        const bool on = k < a.K && ((a.enabled >> k) & 1ull);
        const float xk = fmaxf(D + a.two_s * fmaf(a.ux[k], px, a.uy[k] * py), 0.0f);
        const float dk = xk * rsqrtf(fmaxf(xk, 1e-30f));
        // beta w2 (d_obs - d_k), formed as a difference of squares
        const float num = a.two_s * fmaf(ex - a.ux[k], px, (ey - a.uy[k]) * py);
        lg[k] = on ? bw2 * __fdividef(num, fmaxf(d_o + dk, 1e-30f)) : -INFINITY;
        m = fmaxf(m, lg[k]);
    }
    float S = 0.0f;
#pragma unroll
    for (int k = 0; k < KT; ++k) {
        lg[k] = (lg[k] == -INFINITY) ? 0.0f : ex2_approx(lg[k] - m);
        S += lg[k];
    }
    StepGrad r;
    r.logpi = -(m + log2f(S)) * kLn2;
    if (!grad) return r;
    const float inv = 1.0f / S;
    float sux = 0.f, suy = 0.f, seu = 0.f, sd = 0.f, sp = 0.f;
#pragma unroll
    for (int k = 0; k < KT; ++k) {
        const float pk = lg[k] * inv;
        const float xk = fmaxf(D + a.two_s * fmaf(a.ux[k], px, a.uy[k] * py), 0.0f);
        const float rk = rsqrtf(fmaxf(xk, 1e-30f));
        const float dk = xk * rk;
        const float qx = fmaf(a.s, a.ux[k], px), qy = fmaf(a.s, a.uy[k], py); // z + s e_k - g
        const float uxk = qx * rk, uyk = qy * rk;
        sux = fmaf(pk, uxk, sux);
        suy = fmaf(pk, uyk, suy);
        seu = fmaf(pk, fmaf(a.ux[k], uxk, a.uy[k] * uyk), seu);
        sd = fmaf(pk, dk, sd);
        sp += pk;
    }
    const float qox = fmaf(a.s, ex, px), qoy = fmaf(a.s, ey, py);
    const float uox = qox * ro, uoy = qoy * ro;
    r.gx = bw * (uox - sux);
    r.gy = bw * (uoy - suy);
    r.gv = bw * a.dt * (seu - fmaf(ex, uox, ey * uoy));
    r.gw1 = beta * a.v * a.dt * (sp - 1.0f); // dQ/dw1 is the same for every heading
    r.gw2 = beta * (sd - d_o);
    return r;
}

// The same terms for KT (even) headings that are all enabled, on packed FP32
// pairs of consecutive headings (the same IEEE operations per element as
// step_terms, in half the issue slots; only the order of the final sums of
// the expectations differs: two interleaved partial sums).
template <int KT>
__device__ __forceinline__ StepGrad step_terms_full(const AdjointArgs &a, float zx, float zy, float ex, float ey,
                                                    float gx, float gy, float beta, bool grad)
{
    static_assert(KT % 2 == 0, "pairs of headings");
    const float px = zx - gx, py = zy - gy;
    const float D = fmaf(px, px, fmaf(py, py, a.s2));
    const float xo = fmaxf(D + a.two_s * fmaf(ex, px, ey * py), 0.0f);
    const float ro = rsqrtf(fmaxf(xo, 1e-30f));
    const float d_o = xo * ro;
    const float bw = beta * a.w2;
    const float bw2 = bw * kLog2e;
    const f32x2 *UX = reinterpret_cast<const f32x2 *>(a.ux);
    const f32x2 *UY = reinterpret_cast<const f32x2 *>(a.uy);
    const f32x2 PX = f2_pack(px, px), PY = f2_pack(py, py), EX = f2_pack(ex, ex), EY = f2_pack(ey, ey);
    const f32x2 DD = f2_pack(D, D), TS = f2_pack(a.two_s, a.two_s), DO = f2_pack(d_o, d_o);
    const f32x2 BW2 = f2_pack(bw2, bw2);
    // X_k = D + 2 s e_k.(z - g), its reciprocal square root, d_k = X_k rsqrt(X_k)
    auto dist = [&](int k2, f32x2 &X, f32x2 &RK) {
        const f32x2 PU = f2_fma(UX[k2], PX, f2_mul(UY[k2], PY));
        float x0, x1;
        f2_unpack(f2_fma(TS, PU, DD), x0, x1);
        x0 = fmaxf(x0, 0.0f);
        x1 = fmaxf(x1, 0.0f);
        X = f2_pack(x0, x1);
        RK = f2_pack(rsqrtf(fmaxf(x0, 1e-30f)), rsqrtf(fmaxf(x1, 1e-30f)));
    };
    f32x2 LG[KT / 2];
    float m = -INFINITY;
#pragma unroll
    for (int k2 = 0; k2 < KT / 2; ++k2) {
        f32x2 X, RK;
        dist(k2, X, RK);
        const f32x2 DK = f2_mul(X, RK);
        // beta w2 (d_obs - d_k) in base 2, formed as a difference of squares
        const f32x2 NUM = f2_mul(TS, f2_fma(f2_sub(EX, UX[k2]), PX, f2_mul(f2_sub(EY, UY[k2]), PY)));
        float q0, q1, n0, n1;
        f2_unpack(f2_add(DO, DK), q0, q1);
        f2_unpack(NUM, n0, n1);
        LG[k2] = f2_mul(BW2, f2_pack(__fdividef(n0, fmaxf(q0, 1e-30f)), __fdividef(n1, fmaxf(q1, 1e-30f))));
        float l0, l1;
        f2_unpack(LG[k2], l0, l1);
        m = fmaxf(m, fmaxf(l0, l1));
    }
    f32x2 SS = f2_pack(0.0f, 0.0f);
    const f32x2 NM = f2_pack(-m, -m);
#pragma unroll
    for (int k2 = 0; k2 < KT / 2; ++k2) {
        float l0, l1;
        f2_unpack(f2_add(LG[k2], NM), l0, l1);
        LG[k2] = f2_pack(ex2_approx(l0), ex2_approx(l1));
        SS = f2_add(SS, LG[k2]);
    }
    float s0, s1;
    f2_unpack(SS, s0, s1);
    const float S = s0 + s1;
    StepGrad r;
    r.logpi = -(m + log2f(S)) * kLn2;
    if (!grad) return r;
    const float inv = 1.0f / S;
    const f32x2 INV = f2_pack(inv, inv), SV = f2_pack(a.s, a.s);
    f32x2 SUX = f2_pack(0.f, 0.f), SUY = SUX, SEU = SUX, SD = SUX, SP = SUX;
#pragma unroll
    for (int k2 = 0; k2 < KT / 2; ++k2) {
        const f32x2 PK = f2_mul(LG[k2], INV);
        f32x2 X, RK;
        dist(k2, X, RK);
        const f32x2 DK = f2_mul(X, RK);
        const f32x2 UXK = f2_mul(f2_fma(SV, UX[k2], PX), RK), UYK = f2_mul(f2_fma(SV, UY[k2], PY), RK);
        SUX = f2_fma(PK, UXK, SUX);
        SUY = f2_fma(PK, UYK, SUY);
        SEU = f2_fma(PK, f2_fma(UX[k2], UXK, f2_mul(UY[k2], UYK)), SEU);
        SD = f2_fma(PK, DK, SD);
        SP = f2_add(SP, PK);
    }
    auto fold = [](f32x2 v) {
        float lo, hi;
        f2_unpack(v, lo, hi);
        return lo + hi;
    };
    const float sux = fold(SUX), suy = fold(SUY), seu = fold(SEU), sd = fold(SD), sp = fold(SP);
    const float qox = fmaf(a.s, ex, px), qoy = fmaf(a.s, ey, py);
    const float uox = qox * ro, uoy = qoy * ro;
    r.gx = bw * (uox - sux);
    r.gy = bw * (uoy - suy);
    r.gv = bw * a.dt * (seu - fmaf(ex, uox, ey * uoy));
    r.gw1 = beta * a.v * a.dt * (sp - 1.0f); // dQ/dw1 is the same for every heading
    r.gw2 = beta * (sd - d_o);
    return r;
}

// Several speeds (control u = speed q x heading k moving sl_q = v m_q dt):
// Q_u = -w1 v m_q dt - w2 d_u, so
//   dQ_u/dg = w2 u_u, dQ_u/dv = -m_q dt (w1 + w2 e_k.u_u), dQ_u/dw1 = -v m_q dt,
//   dQ_u/dw2 = -d_u,
// and the observed control is the observed direction at the enabled speed
// nearest to the step's length. cu[u] = (cos, sin of theta_k, sl_q, m_q or 0
// when speed q is disabled); the controls are visited in three passes
// (maximum, sum, expectations) instead of being held in registers.
__device__ __forceinline__ StepGrad step_terms_ms(const AdjointArgs &a, const float4 *cu, int U, float zx, float zy,
                                                  float ex, float ey, float len, float gx, float gy, float beta,
                                                  bool grad)
{
    int q0 = 0;
    float best = INFINITY;
    const float r = len / a.s;
    for (int q = 0; q < a.sp.S; ++q) {
        const float d = fabsf(a.sp.mult[q] - r);
        if (((a.sp.speed_on >> q) & 1u) && d < best) {
            best = d;
            q0 = q;
        }
    }
    const float so = a.sp.sl[q0], mo = a.sp.mult[q0];
    const float px = zx - gx, py = zy - gy;
    const float P = fmaf(px, px, py * py);
    const float xo = fmaxf(fmaf(so, so, P) + 2.0f * so * fmaf(ex, px, ey * py), 0.0f);
    const float ro = rsqrtf(fmaxf(xo, 1e-30f));
    const float d_o = xo * ro;
    const float bw2 = beta * a.w2;
    // logits in base 2 (exponentials on the SFU)
    const float bl1 = beta * a.sp.w1 * kLog2e, bl2 = bw2 * kLog2e;
    auto logit = [&](const float4 &c, float &du, float &rk) {
        const float xk = fmaxf(fmaf(c.z, c.z, P) + 2.0f * c.z * fmaf(c.x, px, c.y * py), 0.0f);
        rk = rsqrtf(fmaxf(xk, 1e-30f));
        du = xk * rk;
        const float num = fmaf(so - c.z, so + c.z, 2.0f * fmaf(fmaf(so, ex, -c.z * c.x), px, fmaf(so, ey, -c.z * c.y) * py));
        return fmaf(bl1, so - c.z, bl2 * __fdividef(num, fmaxf(d_o + du, 1e-30f)));
    };
    float m = -INFINITY;
    for (int u = 0; u < U; ++u) {
        const float4 c = cu[u];
        if (c.w == 0.0f) continue;
        float du, rk;
        m = fmaxf(m, logit(c, du, rk));
    }
    float S = 0.0f;
    for (int u = 0; u < U; ++u) {
        const float4 c = cu[u];
        if (c.w == 0.0f) continue;
        float du, rk;
        S += ex2_approx(logit(c, du, rk) - m);
    }
    StepGrad res;
    res.logpi = -(m + log2f(S)) * kLn2;
    if (!grad) return res;
    const float inv = 1.0f / S;
    float sux = 0.f, suy = 0.f, smeu = 0.f, sm = 0.f, sd = 0.f;
    for (int u = 0; u < U; ++u) {
        const float4 c = cu[u];
        if (c.w == 0.0f) continue;
        float du, rk;
        const float pk = ex2_approx(logit(c, du, rk) - m) * inv;
        const float uxk = fmaf(c.z, c.x, px) * rk, uyk = fmaf(c.z, c.y, py) * rk; // (z + sl e_k - g) / d_u
        sux = fmaf(pk, uxk, sux);
        suy = fmaf(pk, uyk, suy);
        smeu = fmaf(pk * c.w, fmaf(c.x, uxk, c.y * uyk), smeu);
        sm = fmaf(pk, c.w, sm);
        sd = fmaf(pk, du, sd);
    }
    const float uox = fmaf(so, ex, px) * ro, uoy = fmaf(so, ey, py) * ro;
    res.gx = bw2 * (uox - sux);
    res.gy = bw2 * (uoy - suy);
    res.gv = beta * a.dt * fmaf(a.sp.w1, sm - mo, a.w2 * (smeu - mo * fmaf(ex, uox, ey * uoy)));
    res.gw1 = beta * a.v * a.dt * (sm - mo);
    res.gw2 = beta * (sd - d_o);
    return res;
}

// Grid: blockIdx.x = trajectory m, blockIdx.y = a group of kCompsPerCta
// components (a warp each). A CTA writes its components' sums to scratch; the
// last CTA of a trajectory (ticket per trajectory) combines them into the
// trajectory's partials, and the last trajectory to finish (global ticket)
// sums the partials in trajectory order. No CTA waits for another.
// FULL: KT headings, all enabled (the packed step_terms_full).
template <int KT, bool MS = false, bool FULL = false>
__global__ void __launch_bounds__(kAdjThreads) adjoint_kernel(const __grid_constant__ AdjointArgs a)
{
    __shared__ double A_s[kMaxJ];
    __shared__ float G_s[kMaxJ][5];
    __shared__ int last;
    __shared__ float4 cu[MS ? PM_MAX_SPEEDS * kMaxK : 1];
    const int U = MS ? a.sp.S * a.K : 0;
    if constexpr (MS) {
        for (int u = threadIdx.x; u < U; u += blockDim.x) {
            const int q = u / a.K, k = u - q * a.K;
            cu[u] = make_float4(a.ux[k], a.uy[k], a.sp.sl[q], ((a.sp.speed_on >> q) & 1u) ? a.sp.mult[q] : 0.0f);
        }
        __syncthreads();
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    const int J = a.G * a.B;
    const int m = blockIdx.x;
    const int P = 2 * a.G + 4; // per-trajectory partials: L, d_goals[2G], d_v, d_w1, d_w2
    const int p0 = min(max(a.offsets[m], 0), a.n_points);
    const int p1 = min(max(a.offsets[m + 1], p0), a.n_points);
    const int nsteps = max(p1 - p0 - 1, 0);
    const bool grad = a.want_grad != 0;
    double *cA = a.comp_A + (size_t)m * J; // this trajectory's per-component sums
    float *cG = a.comp_G + (size_t)m * J * 5;

    for (int j = blockIdx.y * nwarp + warp; j < min(J, (int)(blockIdx.y + 1) * nwarp); j += nwarp) {
        const int g = j / a.B, b = j - g * a.B;
        const float beta = a.beta[b];
        const float gx = a.goals[2 * g], gy = a.goals[2 * g + 1];
        double A = 0.0;
        float Gx = 0.f, Gy = 0.f, Gv = 0.f, Gw1 = 0.f, Gw2 = 0.f;
        for (int t = lane; t < nsteps; t += 32) {
            const float *z = a.traj + 2 * (size_t)(p0 + t);
            const float zx = z[0], zy = z[1];
            const float dx = z[2] - zx, dy = z[3] - zy;
            const float len = sqrtf(fmaf(dx, dx, dy * dy));
            if (!isfinite(len)) { // unusable point: its steps are skipped and reported
                flag_status(a.status, kStatusTraj);
                continue;
            }
            if (!(len >= 1e-6f)) continue; // stationary step: no information
            float ex = dx / len, ey = dy / len;
            if (a.snap) { // the discrete control nearest to the observed heading
                const float2 e = nearest_heading(a.ux, a.uy, a.enabled, a.K, dx, dy);
                ex = e.x;
                ey = e.y;
            }
            StepGrad s;
            if constexpr (MS) s = step_terms_ms(a, cu, U, zx, zy, ex, ey, len, gx, gy, beta, grad);
            else if constexpr (FULL) s = step_terms_full<KT>(a, zx, zy, ex, ey, gx, gy, beta, grad);
            else s = step_terms<KT>(a, zx, zy, ex, ey, gx, gy, beta, grad);
            A += (double)s.logpi;
            if (grad) {
                Gx += s.gx;
                Gy += s.gy;
                Gv += s.gv;
                Gw1 += s.gw1;
                Gw2 += s.gw2;
            }
        }
        A = wsum_d(A);
        if (grad) {
            Gx = wsum(Gx);
            Gy = wsum(Gy);
            Gv = wsum(Gv);
            Gw1 = wsum(Gw1);
            Gw2 = wsum(Gw2);
        }
        if (lane == 0) {
            cA[j] = A;
            cG[5 * j + 0] = Gx;
            cG[5 * j + 1] = Gy;
            cG[5 * j + 2] = Gv;
            cG[5 * j + 3] = Gw1;
            cG[5 * j + 4] = Gw2;
        }
    }

    // the last CTA of this trajectory combines its components
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = (atomicAdd(a.traj_ticket + m, 1u) == gridDim.y - 1);
    __syncthreads();
    if (!last) return;
    __threadfence();
    for (int j = threadIdx.x; j < J; j += blockDim.x) {
        A_s[j] = ((volatile double *)cA)[j];
#pragma unroll
        for (int c = 0; c < 5; ++c) G_s[j][c] = ((volatile float *)cG)[5 * j + c];
    }
    if (threadIdx.x == 0) a.traj_ticket[m] = 0u;
    __syncthreads();

    double *part = a.part + (size_t)m * P;
    if (warp == 0) {
        double mx = -INFINITY;
        for (int j = lane; j < J; j += 32) {
            const float lp = a.log_prior[j];
            if (isnan(lp) || lp == INFINITY) flag_status(a.status, kStatusBelief);
            mx = fmax(mx, (double)lp + A_s[j]);
        }
        mx = wmax_d(mx);
        float se = 0.0f;
        for (int j = lane; j < J; j += 32) {
            const double Lj = (double)a.log_prior[j] + A_s[j];
            if (Lj != -INFINITY) se += expf((float)(Lj - mx));
        }
        se = wsum(se);
        const double lse = mx + log((double)se);
        if (lane == 0) part[0] = lse;
        if (grad) {
            // posterior weights of the components for this trajectory
            for (int j = lane; j < J; j += 32) {
                const double Lj = (double)a.log_prior[j] + A_s[j];
                A_s[j] = (Lj == -INFINITY) ? 0.0 : (double)expf((float)(Lj - lse));
            }
            __syncwarp();
            float v = 0.f, w1 = 0.f, w2 = 0.f;
            for (int j = lane; j < J; j += 32) {
                const float w = (float)A_s[j];
                v = fmaf(w, G_s[j][2], v);
                w1 = fmaf(w, G_s[j][3], w1);
                w2 = fmaf(w, G_s[j][4], w2);
            }
            v = wsum(v);
            w1 = wsum(w1);
            w2 = wsum(w2);
            for (int g = 0; g < a.G; ++g) {
                float sx = 0.f, sy = 0.f;
                for (int b = lane; b < a.B; b += 32) {
                    const int j = g * a.B + b;
                    const float w = (float)A_s[j];
                    sx = fmaf(w, G_s[j][0], sx);
                    sy = fmaf(w, G_s[j][1], sy);
                }
                sx = wsum(sx);
                sy = wsum(sy);
                if (lane == 0) {
                    part[1 + 2 * g] = sx;
                    part[2 + 2 * g] = sy;
                }
            }
            if (lane == 0) {
                part[1 + 2 * a.G] = v;
                part[2 + 2 * a.G] = w1;
                part[3 + 2 * a.G] = w2;
            }
        }
    }

    // the last trajectory to finish sums the partials in trajectory order
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = (atomicAdd(a.ticket, 1u) == (unsigned)(gridDim.x - 1));
    __syncthreads();
    if (!last) return;
    __threadfence();
    const int nout = grad ? P : 1;
    for (int q = warp; q < nout; q += nwarp) {
        double s = 0.0;
        for (int mm = lane; mm < a.M; mm += 32) s += ((volatile double *)a.part)[(size_t)mm * P + q];
        s = wsum_d(s);
        if (lane == 0) {
            if (q == 0) {
                *a.loglik = (float)s;
            } else if (q <= 2 * a.G) {
                a.d_goals[q - 1] = (float)(s * (double)a.grad_out);
            } else if (q == 2 * a.G + 1) {
                *a.d_speed = (float)(s * (double)a.grad_out);
            } else {
                a.d_w[q - 2 * a.G - 2] = (float)(s * (double)a.grad_out);
            }
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) *a.ticket = 0u;
}

} // namespace

// Scratch: per-trajectory partials [M][2G+4] doubles, per-component sums
// [M][J] doubles and [M][J][5] floats, and one ticket word per trajectory.
size_t adjoint_scratch_bytes(int M, int G, int J)
{
    return (size_t)M * (2 * G + 4) * sizeof(double) + (size_t)M * J * sizeof(double) +
           (size_t)M * J * 5 * sizeof(float) + (size_t)M * sizeof(unsigned);
}

void adjoint_scratch_layout(void *base, int M, int G, int J, AdjointArgs &a)
{
    char *p = static_cast<char *>(base);
    a.part = reinterpret_cast<double *>(p);
    p += (size_t)M * (2 * G + 4) * sizeof(double);
    a.comp_A = reinterpret_cast<double *>(p);
    p += (size_t)M * J * sizeof(double);
    a.comp_G = reinterpret_cast<float *>(p);
    p += (size_t)M * J * 5 * sizeof(float);
    a.traj_ticket = reinterpret_cast<unsigned *>(p);
}

cudaError_t launch_adjoint(const AdjointArgs &a, cudaStream_t s)
{
    // the per-trajectory tickets start at zero whatever an earlier call left
    cudaError_t e = cudaMemsetAsync(a.traj_ticket, 0, (size_t)a.M * sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    const int J = a.G * a.B;
    const dim3 grid((unsigned)a.M, (unsigned)((J + kAdjThreads / 32 - 1) / (kAdjThreads / 32)));
    if (a.sp.S > 0) {
        adjoint_kernel<8, true><<<grid, kAdjThreads, 0, s>>>(a);
        return cudaGetLastError();
    }
    const int KT = rollout_kt_for(a.K);
    const uint64_t all = (KT >= 64) ? ~0ull : ((1ull << KT) - 1ull);
    const bool full = a.K == KT && (a.enabled & all) == all;
    switch (KT) {
    case 8: full ? adjoint_kernel<8, false, true><<<grid, kAdjThreads, 0, s>>>(a)
                 : adjoint_kernel<8><<<grid, kAdjThreads, 0, s>>>(a); break;
    case 16: full ? adjoint_kernel<16, false, true><<<grid, kAdjThreads, 0, s>>>(a)
                  : adjoint_kernel<16><<<grid, kAdjThreads, 0, s>>>(a); break;
    case 36: full ? adjoint_kernel<36, false, true><<<grid, kAdjThreads, 0, s>>>(a)
                  : adjoint_kernel<36><<<grid, kAdjThreads, 0, s>>>(a); break;
    default: full ? adjoint_kernel<64, false, true><<<grid, kAdjThreads, 0, s>>>(a)
                  : adjoint_kernel<64><<<grid, kAdjThreads, 0, s>>>(a); break;
    }
    return cudaGetLastError();
}

} // namespace pm
