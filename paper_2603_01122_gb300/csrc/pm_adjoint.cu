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
// unrolled in registers. Each step is one pass over the headings: the
// weights are normalised by a bound on the largest logit, so the distance,
// its reciprocal and the exponential of each heading are formed once and go
// straight into the softmax sum and the gradient's expectations. The
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

__device__ __forceinline__ float rcp_approx(float x)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// One pass over the headings of a step. The logit of heading k relative to
// the observed heading, beta w2 (d_o - d_k), is formed as a difference of
// squares, delta_k = d_o - d_k = 2 s (e_o - e_k).p / (d_o + d_k) with
// p = z - g and s = v dt, which keeps its relative precision however close
// the two headings are. Its largest value over k is bounded without looking
// at the headings: every d_k lies between ||p| - s| and |p| + s (triangle
// inequality), so with c the lower bound when beta w2 >= 0 and the upper one
// otherwise (sg = +1 / -1),
//   max_k beta w2 (d_o - d_k) <= beta w2 (d_o - c) = |beta w2| t_o,
//   t_o = 2 s (|p| + sg e_o.p) / (c + d_o) >= 0.
// The weights w_k = 2^(beta w2 log2(e) delta_k - B), B = |beta w2| log2(e) t_o,
// are then all at most 1 (up to rounding), log pi(obs) = -(B + log2 sum w) ln 2,
// and the softmax sum and every expectation of the gradient are formed in
// the same pass while d_k and 1/d_k are in registers. Where the bound is
// loose (sum w < 2^-8: the largest weight lies more than 8 binades below it,
// which needs beta w2 s (1 - cos(pi/K)) of several units), the rounding of
// the offset would show, and the step takes a second pass normalised by the
// largest logit instead.
struct StepGeo {
    float px, py, D, ro, d_o, bl2, B;
};

__device__ __forceinline__ StepGeo step_geo(const AdjointArgs &a, float px, float py, float ex, float ey, float bw)
{
    StepGeo g;
    g.px = px;
    g.py = py;
    const float P = fmaf(px, px, py * py);
    g.D = P + a.s2;
    const float pn = sqrtf(P);
    const float sg = bw >= 0.0f ? 1.0f : -1.0f;
    const float c = fabsf(pn - sg * a.s);
    const float po = fmaf(ex, px, ey * py);
    const float xo = fmaxf(fmaf(a.two_s, po, g.D), 0.0f);
    g.ro = rsqrtf(fmaxf(xo, 1e-30f));
    g.d_o = xo * g.ro;
    g.bl2 = bw * kLog2e;
    g.B = fabsf(g.bl2) * (a.two_s * fmaxf(fmaf(sg, po, pn), 0.0f) / fmaxf(c + g.d_o, 1e-30f));
    return g;
}

// The gradient terms from the weighted sums (S, sum w r, sum w r ux,
// sum w r uy, sum w r e.p, sum w delta) and the offset of the weights.
__device__ __forceinline__ StepGrad step_finish(const AdjointArgs &a, const StepGeo &g, float ex, float ey, float beta,
                                                float bw, float off, float S, float R, float RX, float RY, float RP,
                                                float DL, bool grad)
{
    StepGrad r;
    r.logpi = -(off + log2f(S)) * kLn2;
    if (!grad) return r;
    const float inv = 1.0f / S;
    // sum pi u_k with u_k = (p + s e_k) / d_k; sum pi e_k.u_k = sum pi (e_k.p + s) / d_k
    const float sux = fmaf(g.px, R, a.s * RX) * inv, suy = fmaf(g.py, R, a.s * RY) * inv;
    const float seu = fmaf(a.s, R, RP) * inv;
    const float uox = fmaf(a.s, ex, g.px) * g.ro, uoy = fmaf(a.s, ey, g.py) * g.ro;
    r.gx = bw * (uox - sux);
    r.gy = bw * (uoy - suy);
    r.gv = bw * a.dt * (seu - fmaf(ex, uox, ey * uoy));
    r.gw1 = 0.0f; // dQ/dw1 = -v dt for every heading: its expectation cancels
    r.gw2 = -beta * DL * inv; // sum pi d_k - d_o = -sum pi delta_k
    return r;
}

// log pi_j(theta_obs | z) and its derivatives for one observed step, over
// runtime K and enabled mask (scalar form).
template <int KT>
__device__ __forceinline__ StepGrad step_terms(const AdjointArgs &a, float zx, float zy, float ex, float ey,
                                               float gx, float gy, float beta, bool grad)
{
    const float bw = beta * a.w2;
    const StepGeo g = step_geo(a, zx - gx, zy - gy, ex, ey, bw);
    // delta_k = d_o - d_k of heading k, with 1/d_k and e_k.p
    auto delta = [&](int k, float &rk, float &pu) {
        pu = fmaf(a.ux[k], g.px, a.uy[k] * g.py);
        const float xk = fmaxf(fmaf(a.two_s, pu, g.D), 0.0f);
        rk = rsqrtf(fmaxf(xk, 1e-30f));
        const float num = a.two_s * fmaf(ex - a.ux[k], g.px, (ey - a.uy[k]) * g.py);
        return num * rcp_approx(fmaxf(fmaf(xk, rk, g.d_o), 1e-30f));
    };
    auto sums = [&](float off, float &S, float &R, float &RX, float &RY, float &RP, float &DL) {
        S = R = RX = RY = RP = DL = 0.0f;
#pragma unroll
        for (int k = 0; k < KT; ++k) {
            if (k >= a.K || !((a.enabled >> k) & 1ull)) continue;
            float rk, pu;
            const float dl = delta(k, rk, pu);
            const float w = ex2_approx(fmaf(g.bl2, dl, -off));
            const float wr = w * rk;
            S += w;
            R += wr;
            RX = fmaf(wr, a.ux[k], RX);
            RY = fmaf(wr, a.uy[k], RY);
            RP = fmaf(wr, pu, RP);
            DL = fmaf(w, dl, DL);
        }
    };
    float off = g.B, S, R, RX, RY, RP, DL;
    sums(off, S, R, RX, RY, RP, DL);
    if (!(S >= 0x1p-8f)) { // the bound is loose: normalise by the largest logit
        off = -INFINITY;
#pragma unroll 1
        for (int k = 0; k < KT; ++k) {
            if (k >= a.K || !((a.enabled >> k) & 1ull)) continue;
            float rk, pu;
            off = fmaxf(off, g.bl2 * delta(k, rk, pu));
        }
        sums(off, S, R, RX, RY, RP, DL);
    }
    return step_finish(a, g, ex, ey, beta, bw, off, S, R, RX, RY, RP, DL, grad);
}

// The same pass for KT (even) headings that are all enabled, on packed FP32
// pairs of consecutive headings (the same operations per element as
// step_terms, in half the issue slots; only the order of the sums differs:
// two interleaved partial sums). A step whose bound is loose is handed to
// step_terms, which takes the second pass.
template <int KT>
__device__ __forceinline__ StepGrad step_terms_full(const AdjointArgs &a, float zx, float zy, float ex, float ey,
                                                    float gx, float gy, float beta, bool grad)
{
    static_assert(KT % 2 == 0, "pairs of headings");
    const float bw = beta * a.w2;
    const StepGeo g = step_geo(a, zx - gx, zy - gy, ex, ey, bw);
    const f32x2 *UX = reinterpret_cast<const f32x2 *>(a.ux);
    const f32x2 *UY = reinterpret_cast<const f32x2 *>(a.uy);
    const f32x2 PX = f2_pack(g.px, g.px), PY = f2_pack(g.py, g.py), DD = f2_pack(g.D, g.D);
    const f32x2 EX = f2_pack(ex, ex), EY = f2_pack(ey, ey), DO = f2_pack(g.d_o, g.d_o);
    const f32x2 TS = f2_pack(a.two_s, a.two_s), BL = f2_pack(g.bl2, g.bl2), NB = f2_pack(-g.B, -g.B);
    const f32x2 Z = f2_pack(0.0f, 0.0f);
    f32x2 S2 = Z, R2 = Z, RX2 = Z, RY2 = Z, RP2 = Z, DL2 = Z;
#pragma unroll
    for (int k2 = 0; k2 < KT / 2; ++k2) {
        const f32x2 PU = f2_fma(UX[k2], PX, f2_mul(UY[k2], PY));
        float x0, x1;
        f2_unpack(f2_fma(TS, PU, DD), x0, x1);
        x0 = fmaxf(x0, 0.0f);
        x1 = fmaxf(x1, 0.0f);
        const f32x2 RK = f2_pack(rsqrtf(fmaxf(x0, 1e-30f)), rsqrtf(fmaxf(x1, 1e-30f)));
        float q0, q1;
        f2_unpack(f2_fma(f2_pack(x0, x1), RK, DO), q0, q1);
        const f32x2 NUM = f2_mul(TS, f2_fma(f2_sub(EX, UX[k2]), PX, f2_mul(f2_sub(EY, UY[k2]), PY)));
        const f32x2 DL = f2_mul(NUM, f2_pack(rcp_approx(fmaxf(q0, 1e-30f)), rcp_approx(fmaxf(q1, 1e-30f))));
        float e0, e1;
        f2_unpack(f2_fma(BL, DL, NB), e0, e1);
        const f32x2 W = f2_pack(ex2_approx(e0), ex2_approx(e1));
        const f32x2 WR = f2_mul(W, RK);
        S2 = f2_add(S2, W);
        R2 = f2_add(R2, WR);
        RX2 = f2_fma(WR, UX[k2], RX2);
        RY2 = f2_fma(WR, UY[k2], RY2);
        RP2 = f2_fma(WR, PU, RP2);
        DL2 = f2_fma(W, DL, DL2);
    }
    auto fold = [](f32x2 v) {
        float lo, hi;
        f2_unpack(v, lo, hi);
        return lo + hi;
    };
    const float S = fold(S2);
    if (!(S >= 0x1p-8f)) return step_terms<KT>(a, zx, zy, ex, ey, gx, gy, beta, grad);
    return step_finish(a, g, ex, ey, beta, bw, g.B, S, fold(R2), fold(RX2), fold(RY2), fold(RP2), fold(DL2), grad);
}

// Several speeds (control u = speed q x heading k moving sl_q = v m_q dt):
// Q_u = -w1 v m_q dt - w2 d_u, so
//   dQ_u/dg = w2 u_u, dQ_u/dv = -m_q dt (w1 + w2 e_k.u_u), dQ_u/dw1 = -v m_q dt,
//   dQ_u/dw2 = -d_u,
// and the observed control is the observed direction at the enabled speed
// nearest to the step's length. The logit relative to the observed control
// is beta (w1 (s_o - sl_q) + w2 delta_u) with the difference of squares
//   delta_u = d_o - d_u = ((s_o - sl)(s_o + sl) + 2 (s_o e_o - sl e_k).p) / (d_o + d_u),
// and each speed bounds its logits as in the one-speed pass, with its own
// c_q (from sl_q) and
//   d_o - c_q = ((s_o - sl_q)(s_o + sl_q) + 2 s_o e_o.p + 2 sg sl_q |p|) / (d_o + c_q);
// the weights are taken relative to the largest of these bounds in one pass
// over the controls, which keeps per speed the sums of the one-speed pass and
// combines them with the speed's constants.
__device__ __forceinline__ StepGrad step_terms_ms(const AdjointArgs &a, int K, float zx, float zy, float ex, float ey,
                                                  float len, float gx, float gy, float beta, bool grad)
{
    int q0 = 0;
    float best = INFINITY;
    const float rl = len / a.s;
    for (int q = 0; q < a.sp.S; ++q) {
        const float d = fabsf(a.sp.mult[q] - rl);
        if (((a.sp.speed_on >> q) & 1u) && d < best) {
            best = d;
            q0 = q;
        }
    }
    const float so = a.sp.sl[q0], mo = a.sp.mult[q0];
    const float px = zx - gx, py = zy - gy;
    const float P = fmaf(px, px, py * py);
    const float pn = sqrtf(P);
    const float po = fmaf(ex, px, ey * py);
    const float xo = fmaxf(fmaf(2.0f * so, po, fmaf(so, so, P)), 0.0f);
    const float ro = rsqrtf(fmaxf(xo, 1e-30f));
    const float d_o = xo * ro;
    const float bw2 = beta * a.w2;
    const float sg = bw2 >= 0.0f ? 1.0f : -1.0f;
    // logits in base 2 (exponentials on the SFU)
    const float bl1 = beta * a.sp.w1 * kLog2e, bl2 = bw2 * kLog2e;
    float B = -INFINITY;
    for (int q = 0; q < a.sp.S; ++q) {
        if (!((a.sp.speed_on >> q) & 1u)) continue;
        const float sl = a.sp.sl[q];
        const float c = fabsf(pn - sg * sl);
        const float tq = fmaf(so - sl, so + sl, 2.0f * fmaf(so, po, sg * sl * pn)) / fmaxf(d_o + c, 1e-30f);
        B = fmaxf(B, fmaf(bl1, so - sl, bl2 * tq));
    }
    float S, SUX, SUY, SMEU, SM, SDL, E;
    // one pass over the enabled controls with weights 2^(logit - off); E is
    // the largest logit seen
    auto sums = [&](float off) {
        S = SUX = SUY = SMEU = SM = SDL = 0.0f;
        E = -INFINITY;
        for (int q = 0; q < a.sp.S; ++q) {
            if (!((a.sp.speed_on >> q) & 1u)) continue;
            const float sl = a.sp.sl[q], mq = a.sp.mult[q];
            const float ts = 2.0f * sl, D = fmaf(sl, sl, P), dsq = (so - sl) * (so + sl);
            const float lq = fmaf(bl1, so - sl, -off), sox = so * ex, soy = so * ey;
            float Sq = 0.f, Rq = 0.f, RXq = 0.f, RYq = 0.f, RPq = 0.f, DLq = 0.f;
#pragma unroll 4
            for (int k = 0; k < K; ++k) {
                const float ux = a.ux[k], uy = a.uy[k];
                const float pu = fmaf(ux, px, uy * py);
                const float xk = fmaxf(fmaf(ts, pu, D), 0.0f);
                const float rk = rsqrtf(fmaxf(xk, 1e-30f));
                const float num = fmaf(2.0f, fmaf(fmaf(-sl, ux, sox), px, fmaf(-sl, uy, soy) * py), dsq);
                const float dl = num * rcp_approx(fmaxf(fmaf(xk, rk, d_o), 1e-30f));
                const float e = fmaf(bl2, dl, lq);
                E = fmaxf(E, e);
                const float w = ex2_approx(e);
                const float wr = w * rk;
                Sq += w;
                Rq += wr;
                RXq = fmaf(wr, ux, RXq);
                RYq = fmaf(wr, uy, RYq);
                RPq = fmaf(wr, pu, RPq);
                DLq = fmaf(w, dl, DLq);
            }
            S += Sq;
            SUX += fmaf(px, Rq, sl * RXq);              // sum w (p + sl e_k)_x / d_u
            SUY += fmaf(py, Rq, sl * RYq);
            SMEU = fmaf(mq, fmaf(sl, Rq, RPq), SMEU);   // sum w m_q e_k.u_u
            SM = fmaf(mq, Sq, SM);
            SDL += DLq;
        }
    };
    float off = B;
    sums(off);
    if (!(S >= 0x1p-8f)) { // the bounds are loose: normalise by the largest logit
        off += E;
        sums(off);
    }
    StepGrad res;
    res.logpi = -(off + log2f(S)) * kLn2;
    if (!grad) return res;
    const float inv = 1.0f / S;
    const float sux = SUX * inv, suy = SUY * inv, smeu = SMEU * inv, sm = SM * inv;
    const float uox = fmaf(so, ex, px) * ro, uoy = fmaf(so, ey, py) * ro;
    res.gx = bw2 * (uox - sux);
    res.gy = bw2 * (uoy - suy);
    res.gv = beta * a.dt * fmaf(a.sp.w1, sm - mo, a.w2 * (smeu - mo * fmaf(ex, uox, ey * uoy)));
    res.gw1 = beta * a.v * a.dt * (sm - mo);
    res.gw2 = -beta * SDL * inv; // sum pi d_u - d_o = -sum pi delta_u
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
            if constexpr (MS) s = step_terms_ms(a, a.K, zx, zy, ex, ey, len, gx, gy, beta, grad);
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
