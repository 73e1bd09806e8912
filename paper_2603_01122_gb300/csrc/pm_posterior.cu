// pm_posterior.cu -- Bayesian update of the joint belief over (beta, g),
// Eq. 3 evaluated in log space as Eq. 7.
//
// The per-step log-likelihood of component j = (g, b) is
//   l_t(j) = beta Q(z_t, theta_obs; g) - LSE_k beta Q(z_t, theta_k; g)
//          = -m_t(j) - log S_t(j),   S_t(j) = sum_k exp(a_k - m_t(j)),
// with a_k = beta w2 (d_obs - d_k), d the distance from the next state to the
// goal and m_t(j) = max_k a_k. The differences are formed without
// cancellation: d_obs - d_k = 2 s (e_obs - e_k).(z - g) / (d_obs + d_k).
// With several speeds (controls u = speed q x heading k, Sec. IV-B) the
// observed step is read as its direction at the enabled speed nearest to its
// length, and the logits run over all S*K controls (lanes over the controls,
// up to eight per lane); the speed term w1 (so - sl_q) joins the distance term.
//
// Layout: the observed steps are split into chunks, one CTA per chunk (and
// per human in the batched form); a warp handles one component at a time with
// its lanes over the headings (warp-shuffle max and sum). The per-step terms
// are accumulated without any per-step logarithm: sum_t m_t in double-float
// and prod_t S_t as a double-float mantissa with an integer power-of-two
// exponent, so the FP32 rounding of log(S_t) (2.4e-7 at S_t ~ 64, and
// correlated over steps) never enters. The last CTA of a human to finish
// (ticket counter, no waiting) folds the chunks in order, takes one logarithm
// per component, adds the prior and applies the LogSumExp normalisation once
// -- Eq. 7 telescoped over the steps, since its per-step normalisers are
// common to every component -- and resets the ticket for the next call.
#include <cuda_runtime.h>

#include "pm_kernels.cuh"

namespace pm {
namespace {

// ln 2 split so that a product with a small integer keeps its error term
constexpr float kLn2Hi = 0.693147182464599609375f;   // nearest float to ln 2
constexpr float kLn2Lo = -1.904654323148236e-09f;    // ln 2 - kLn2Hi

__device__ __forceinline__ float warp_max(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

__device__ __forceinline__ float warp_sum(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Double-float accumulators of one component over a run of steps.
struct Acc {
    float mh, ml; // sum of m_t (hi + lo)
    float ph, pl; // product of S_t, mantissa in [1, 2) (hi + lo)
    int e;        // product exponent
};

__device__ __forceinline__ void acc_init(Acc &a)
{
    a.mh = a.ml = 0.0f;
    a.ph = 1.0f;
    a.pl = 0.0f;
    a.e = 0;
}

__device__ __forceinline__ void acc_add(Acc &a, float m)
{
    const float s = a.mh + m;
    const float bb = s - a.mh;
    const float err = (a.mh - (s - bb)) + (m - bb);
    a.mh = s;
    a.ml += err;
}

// (ph, pl) *= (qh, ql), then scale the mantissa back into [1, 2).
__device__ __forceinline__ void acc_mul(Acc &a, float qh, float ql, int qe)
{
    const float p = a.ph * qh;
    const float err = fmaf(a.ph, qh, -p);
    const float q = fmaf(a.ph, ql, fmaf(a.pl, qh, err));
    float h = p + q;
    float l = q - (h - p);
    const int ex = ((__float_as_int(h) >> 23) & 0xFF) - 127; // h in [1, 2^8) here
    const float sc = __int_as_float((127 - ex) << 23);      // 2^-ex, exact
    a.ph = h * sc;
    a.pl = l * sc;
    a.e += ex + qe;
}

__device__ __forceinline__ void acc_merge(Acc &a, const Acc &b)
{
    acc_add(a, b.mh);
    acc_add(a, b.ml);
    acc_mul(a, b.ph, b.pl, b.e);
}

__device__ __forceinline__ Acc shfl_acc(const Acc &a, int o)
{
    Acc r;
    r.mh = __shfl_xor_sync(0xffffffffu, a.mh, o);
    r.ml = __shfl_xor_sync(0xffffffffu, a.ml, o);
    r.ph = __shfl_xor_sync(0xffffffffu, a.ph, o);
    r.pl = __shfl_xor_sync(0xffffffffu, a.pl, o);
    r.e = __shfl_xor_sync(0xffffffffu, a.e, o);
    return r;
}

// Logit of heading k relative to the observed heading, beta w2 (d_obs - d_k).
__device__ __forceinline__ float rel_logit(float bw, float two_s, float D, float px, float py,
                                           float ex, float ey, float d_o, float ux, float uy)
{
    const float dk = sqrtf(fmaxf(D + two_s * fmaf(ux, px, uy * py), 0.0f));
    const float num = two_s * fmaf(ex - ux, px, (ey - uy) * py);
    return bw * (num / fmaxf(d_o + dk, 1e-30f));
}

// Controls per lane of the several-speed form: S*K <= 256 over 32 lanes.
constexpr int kMsPerLane = 8;

// The enabled speed multiplier nearest to r (ties: the lower index).
__device__ __forceinline__ int snap_speed(const SpeedSet &sp, uint32_t speed_on, float r)
{
    int q0 = 0;
    float best = INFINITY;
    for (int q = 0; q < sp.S; ++q) {
        const float d = fabsf(sp.mult[q] - r);
        if (((speed_on >> q) & 1u) && d < best) {
            best = d;
            q0 = q;
        }
    }
    return q0;
}

// Several speeds: the logit of control u = (speed q, heading k) relative to
// the observed control (snapped speed length so, observed direction e),
//   beta (Q_u - Q_obs) = beta w1 (so - sl_q) + beta w2 (d_obs - d_u),
//   d_obs - d_u = ((so - sl)(so + sl) + 2 (so e - sl e_k).(z - g)) / (d_obs + d_u),
// again without cancellation. cu[u] = (cos, sin of theta_k, sl_q, enabled).
__device__ __forceinline__ void step_loglik_ms(const SpeedSet &sp, const float4 *cu, int U, float bw1, float bw2,
                                               float px, float py, float ex, float ey, float so, int lane, float &m,
                                               float &S)
{
    const float P = fmaf(px, px, py * py);
    const float d_o = sqrtf(fmaxf(fmaf(so, so, P) + 2.0f * so * fmaf(ex, px, ey * py), 0.0f));
    float lg[kMsPerLane];
    float mx = -INFINITY;
#pragma unroll
    for (int i = 0; i < kMsPerLane; ++i) {
        const int u = lane + 32 * i;
        lg[i] = -INFINITY;
        if (u < U) {
            const float4 c = cu[u];
            if (c.w != 0.0f) {
                const float du = sqrtf(fmaxf(fmaf(c.z, c.z, P) + 2.0f * c.z * fmaf(c.x, px, c.y * py), 0.0f));
                const float num = fmaf(so - c.z, so + c.z,
                                       2.0f * fmaf(fmaf(so, ex, -c.z * c.x), px, fmaf(so, ey, -c.z * c.y) * py));
                lg[i] = fmaf(bw1, so - c.z, bw2 * (num / fmaxf(d_o + du, 1e-30f)));
            }
        }
        mx = fmaxf(mx, lg[i]);
    }
    m = warp_max(mx);
    float sum = 0.0f;
#pragma unroll
    for (int i = 0; i < kMsPerLane; ++i) sum += (lg[i] == -INFINITY) ? 0.0f : expf(lg[i] - m);
    S = warp_sum(sum);
}

// One chunk of one human's observed steps; the last chunk of the human to
// finish folds all chunks and writes the posterior. MS: several speeds.
template <bool MS>
__device__ __forceinline__ void posterior_chunk(const PosteriorArgs &a, const PostHuman &h, int chunk, int nchunk)
{
    __shared__ int last;
    __shared__ float2 su[kMaxK]; // unit heading vectors
    __shared__ float4 cu[MS ? kMsPerLane * 32 : 1]; // several speeds: (e_k, sl_q, enabled) of control u
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    const int J = h.G * h.B;
    const int t0 = chunk * h.steps_per_chunk;
    const int t1 = min(h.n_obs, t0 + h.steps_per_chunk);
    // the table goes through shared memory once per CTA: lanes reading
    // different entries of the kernel parameters would be served one address
    // at a time by the constant cache
    __syncthreads(); // the previous chunk of this CTA (batched form) is done with su
    for (int k = threadIdx.x; k < kMaxK; k += blockDim.x) su[k] = make_float2(a.ux[k], a.uy[k]);
    const int U = MS ? a.sp.S * a.K : 0;
    if constexpr (MS) {
        for (int u = threadIdx.x; u < U; u += blockDim.x) {
            const int q = u / a.K, k = u - q * a.K;
            cu[u] = make_float4(a.ux[k], a.uy[k], a.sp.sl[q], ((h.speed_on >> q) & 1u) ? 1.0f : 0.0f);
        }
    }
    __syncthreads();
    const int k0 = lane, k1 = lane + 32;
    const bool on0 = k0 < a.K && ((a.enabled >> k0) & 1ull);
    const bool on1 = k1 < a.K && ((a.enabled >> k1) & 1ull);
    const float ux0 = on0 ? su[k0].x : 0.0f, uy0 = on0 ? su[k0].y : 0.0f;
    const float ux1 = on1 ? su[k1].x : 0.0f, uy1 = on1 ? su[k1].y : 0.0f;

    for (int j = warp; j < J; j += nwarp) {
        const int g = j / h.B, b = j - g * h.B;
        const float bw = h.beta[b] * a.w2;
        const float gx = h.goals[2 * g], gy = h.goals[2 * g + 1];
        Acc acc;
        acc_init(acc);
        for (int t = t0; t < t1; ++t) {
            const float zx = h.obs[2 * t], zy = h.obs[2 * t + 1];
            const float dx = h.obs[2 * t + 2] - zx, dy = h.obs[2 * t + 3] - zy;
            const float len = sqrtf(fmaf(dx, dx, dy * dy));
            if (!isfinite(len)) { // unusable observation: skipped and reported
                if (lane == 0) flag_status(a.status, kStatusObs);
                continue;
            }
            if (!(len >= 1e-6f)) continue; // stationary: the belief is unchanged
            float ex = dx / len, ey = dy / len;
            if (a.snap) { // the discrete control nearest to the observed heading
                const float2 e = nearest_heading(a.ux, a.uy, a.enabled, a.K, dx, dy);
                ex = e.x;
                ey = e.y;
            }
            const float px = zx - gx, py = zy - gy;
            if constexpr (MS) {
                const float so = a.sp.sl[snap_speed(a.sp, h.speed_on, len / a.s)];
                float m, S;
                step_loglik_ms(a.sp, cu, U, h.beta[b] * a.sp.w1, bw, px, py, ex, ey, so, lane, m, S);
                acc_add(acc, m);
                acc_mul(acc, S, 0.0f, 0);
                continue;
            }
            const float D = fmaf(px, px, fmaf(py, py, a.s2));
            const float d_o = sqrtf(fmaxf(D + a.two_s * fmaf(ex, px, ey * py), 0.0f));
            const float l0 = on0 ? rel_logit(bw, a.two_s, D, px, py, ex, ey, d_o, ux0, uy0) : -INFINITY;
            const float l1 = on1 ? rel_logit(bw, a.two_s, D, px, py, ex, ey, d_o, ux1, uy1) : -INFINITY;
            const float m = warp_max(fmaxf(l0, l1));
            const float S = warp_sum((on0 ? expf(l0 - m) : 0.0f) + (on1 ? expf(l1 - m) : 0.0f));
            acc_add(acc, m);
            acc_mul(acc, S, 0.0f, 0);
        }
        if (lane == 0) {
            float *p = h.part + 5 * ((size_t)chunk * J + j);
            p[0] = acc.mh;
            p[1] = acc.ml;
            p[2] = acc.ph;
            p[3] = acc.pl;
            p[4] = __int_as_float(acc.e);
            __threadfence(); // the partials are visible before this CTA takes its ticket
        }
    }

    // the last chunk to finish combines and normalises
    __syncthreads();
    if (threadIdx.x == 0) last = (atomicAdd(h.ticket, 1u) == (unsigned)(nchunk - 1));
    __syncthreads();
    if (!last) return;
    __threadfence();

    // L_j = log b_j + sum_t l_t(j) as a double-float pair (hi, lo) in shared
    // memory; the fold and the normalisation stay in FP32 arithmetic (this
    // GPU's FP64 unit retires about two lanes per clock per SM)
    __shared__ float2 L[kMaxJ];
    // whether any observed step moved the belief: when every step was
    // skipped (stationary or unusable), the update is the identity and the
    // prior is returned verbatim, not renormalised in FP32 (which would move
    // its last bits on every call)
    __shared__ int moved;
    if (threadIdx.x == 0) moved = 0;
    __syncthreads();
    for (int j = warp; j < J; j += nwarp) {
        Acc acc;
        acc_init(acc);
        for (int c = lane; c < nchunk; c += 32) {
            const volatile float *p = h.part + 5 * ((size_t)c * J + j);
            Acc q;
            q.mh = p[0];
            q.ml = p[1];
            q.ph = p[2];
            q.pl = p[3];
            q.e = __float_as_int(p[4]);
            acc_merge(acc, q);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const Acc q = shfl_acc(acc, o);
            acc_merge(acc, q);
        }
        if (lane == 0) {
            if (acc.mh != 0.0f || acc.ml != 0.0f || acc.ph != 1.0f || acc.pl != 0.0f || acc.e != 0) moved = 1;
            const float lb = h.log_prior[j];
            if (isnan(lb) || lb == INFINITY) flag_status(a.status, kStatusBelief);
            if (lb == -INFINITY) {
                L[j] = make_float2(-INFINITY, 0.0f);
            } else {
                // sum_t l_t(j) = -(sum_t m_t) - log(prod_t S_t),
                // log(prod_t S_t) = e ln2 + log1p(ph - 1) + pl / ph
                const float ef = (float)acc.e;
                const float p = ef * kLn2Hi;
                const float perr = fmaf(ef, kLn2Hi, -p) + ef * kLn2Lo; // e ln2 = p + perr
                Acc r;
                r.mh = lb;
                r.ml = 0.0f;
                acc_add(r, -acc.mh);
                acc_add(r, -acc.ml);
                acc_add(r, -p);
                acc_add(r, -(perr + log1pf(acc.ph - 1.0f) + acc.pl / acc.ph));
                L[j] = make_float2(r.mh, r.ml);
            }
        }
    }
    __syncthreads();
    if (warp == 0 && !moved) {
        for (int j = lane; j < J; j += 32) h.log_b[j] = h.log_prior[j];
        if (lane == 0) *h.ticket = 0u;
    } else if (warp == 0) {
        float mx = -INFINITY;
        for (int j = lane; j < J; j += 32) mx = fmaxf(mx, L[j].x);
        mx = warp_max(mx);
        float se = 0.0f;
        for (int j = lane; j < J; j += 32)
            if (L[j].x != -INFINITY) se += expf((L[j].x - mx) + L[j].y);
        se = warp_sum(se);
        const float lse = logf(se); // se in [1, J]
        for (int j = lane; j < J; j += 32)
            h.log_b[j] = (L[j].x == -INFINITY || mx == -INFINITY) ? -INFINITY : ((L[j].x - mx) + L[j].y) - lse;
        if (lane == 0) *h.ticket = 0u;
    }
}

// MS: several speeds. A template parameter rather than a branch, so that a
// launch carries only its own form's code (the kernel runs once per call on
// a cold instruction cache).
template <bool MS>
__global__ void __launch_bounds__(1024) posterior_kernel(const __grid_constant__ PosteriorArgs a)
{
    PostHuman h;
    h.goals = a.goals;
    h.beta = a.beta;
    h.G = a.G;
    h.B = a.B;
    h.obs = a.obs;
    h.n_obs = a.n_obs;
    h.steps_per_chunk = a.steps_per_chunk;
    h.log_prior = a.log_prior;
    h.log_b = a.log_b;
    h.part = a.part;
    h.ticket = a.ticket;
    h.speed_on = a.sp.speed_on;
    posterior_chunk<MS>(a, h, blockIdx.x, gridDim.x);
}

// Batched form: blockIdx.y is the human; the CTAs of a row stride over its
// chunks, so any number of observed steps fits a fixed grid (as a captured
// CUDA graph requires); humans with no observed steps leave their row idle.
template <bool MS>
__global__ void __launch_bounds__(1024) posterior_batch_kernel(const __grid_constant__ PosteriorArgs a,
                                                               const PostHuman *humans, const int *n_humans)
{
    if ((int)blockIdx.y >= *n_humans) return;
    const PostHuman h = humans[blockIdx.y];
    if (h.n_obs <= 0 || h.log_b == nullptr || h.log_prior == nullptr) return;
    const int nchunk = (h.n_obs + h.steps_per_chunk - 1) / h.steps_per_chunk;
    for (int ch = blockIdx.x; ch < nchunk; ch += gridDim.x) {
        posterior_chunk<MS>(a, h, ch, nchunk);
    }
}

} // namespace

size_t posterior_scratch_bytes(int n_chunks, int J)
{
    return (5 * (size_t)n_chunks * J) * sizeof(float);
}

int posterior_chunks(int n_obs, int *steps_per_chunk)
{
    const int spc = (n_obs + 63) / 64;
    *steps_per_chunk = spc < 1 ? 1 : spc;
    return (n_obs + *steps_per_chunk - 1) / *steps_per_chunk;
}

cudaError_t launch_posterior_batch(const PosteriorArgs &a, const PostHuman *humans, const int *n_humans,
                                   int max_rows, int max_chunks, int max_J, cudaStream_t s)
{
    int threads = 32 * max_J;
    if (threads > 1024) threads = 1024;
    if (max_rows <= 0) return cudaSuccess;
    const dim3 grid(max_chunks > 0 ? max_chunks : 1, max_rows);
    if (a.sp.S > 0) posterior_batch_kernel<true><<<grid, threads, 0, s>>>(a, humans, n_humans);
    else posterior_batch_kernel<false><<<grid, threads, 0, s>>>(a, humans, n_humans);
    return cudaGetLastError();
}

cudaError_t launch_posterior(const PosteriorArgs &a, int n_chunks, cudaStream_t s)
{
    const int J = a.G * a.B;
    int threads = 32 * J;
    if (threads > 1024) threads = 1024;
    if (a.sp.S > 0) posterior_kernel<true><<<n_chunks, threads, 0, s>>>(a);
    else posterior_kernel<false><<<n_chunks, threads, 0, s>>>(a);
    return cudaGetLastError();
}

} // namespace pm
