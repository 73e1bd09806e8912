// pm_posterior.cu -- Bayesian update of the joint belief over (beta, g),
// Eq. 3 evaluated in log space as Eq. 7.
//
// The per-step log-likelihood of component j = (g, b) is
//   l_t(j) = beta Q(z_t, theta_obs; g) - LSE_k beta Q(z_t, theta_k; g)
//          = -LSE_k beta w2 (d_obs - d_k),
// with d the distance from the next state to the goal. The differences are
// formed without cancellation: d_obs - d_k = 2 s (e_obs - e_k).(z - g) /
// (d_obs + d_k). One warp handles one component at a time with its lanes
// over the headings (warp-shuffle max and sum); the log-likelihoods are
// accumulated over the observed steps in FP64, and the LogSumExp
// normalisation over (beta, g) is applied once in FP64 at the end, which is
// the sequential Eq. 7 telescoped (the per-step normalisers are common to
// every component and cancel).
#include <cuda_runtime.h>

#include "pm_internal.cuh"

namespace pm {
namespace {

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

__device__ __forceinline__ double warp_max_d(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

__device__ __forceinline__ double warp_sum_d(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Logit of heading k relative to the observed heading, beta w2 (d_obs - d_k).
__device__ __forceinline__ float rel_logit(float bw, float two_s, float D, float px, float py,
                                           float ex, float ey, float d_o, float ux, float uy)
{
    const float dk = sqrtf(fmaxf(D + two_s * fmaf(ux, px, uy * py), 0.0f));
    const float num = two_s * fmaf(ex - ux, px, (ey - uy) * py);
    return bw * (num / fmaxf(d_o + dk, 1e-30f));
}

__global__ void __launch_bounds__(1024) posterior_kernel(const __grid_constant__ PosteriorArgs a)
{
    __shared__ double acc[kMaxJ];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    const int J = a.G * a.B;
    const int k0 = lane, k1 = lane + 32;
    const bool on0 = k0 < a.K && ((a.enabled >> k0) & 1ull);
    const bool on1 = k1 < a.K && ((a.enabled >> k1) & 1ull);
    const float ux0 = on0 ? a.ux[k0] : 0.0f, uy0 = on0 ? a.uy[k0] : 0.0f;
    const float ux1 = on1 ? a.ux[k1] : 0.0f, uy1 = on1 ? a.uy[k1] : 0.0f;

    for (int j = warp; j < J; j += nwarp) {
        const int g = j / a.B, b = j - g * a.B;
        const float bw = a.beta[b] * a.w2;
        const float gx = a.goals[2 * g], gy = a.goals[2 * g + 1];
        double sum = 0.0;
        for (int t = 0; t < a.n_obs; ++t) {
            const float zx = a.obs[2 * t], zy = a.obs[2 * t + 1];
            const float dx = a.obs[2 * t + 2] - zx, dy = a.obs[2 * t + 3] - zy;
            const float len = sqrtf(fmaf(dx, dx, dy * dy));
            if (!(len >= 1e-6f)) continue; // stationary: the belief is unchanged
            const float ex = dx / len, ey = dy / len;
            const float px = zx - gx, py = zy - gy;
            const float D = fmaf(px, px, fmaf(py, py, a.s2));
            const float d_o = sqrtf(fmaxf(D + a.two_s * fmaf(ex, px, ey * py), 0.0f));
            const float l0 = on0 ? rel_logit(bw, a.two_s, D, px, py, ex, ey, d_o, ux0, uy0) : -INFINITY;
            const float l1 = on1 ? rel_logit(bw, a.two_s, D, px, py, ex, ey, d_o, ux1, uy1) : -INFINITY;
            const float m = warp_max(fmaxf(l0, l1));
            const float se = warp_sum((on0 ? expf(l0 - m) : 0.0f) + (on1 ? expf(l1 - m) : 0.0f));
            sum -= (double)m + (double)logf(se);
        }
        if (lane == 0) acc[j] = sum;
    }
    __syncthreads();
    if (warp == 0) {
        double L[kMaxJ / 32];
        double mx = -INFINITY;
#pragma unroll
        for (int q = 0; q < kMaxJ / 32; ++q) {
            const int j = lane + 32 * q;
            L[q] = (j < J) ? (double)a.log_b[j] + acc[j] : -INFINITY;
            mx = fmax(mx, L[q]);
        }
        mx = warp_max_d(mx);
        double se = 0.0;
#pragma unroll
        for (int q = 0; q < kMaxJ / 32; ++q)
            if (L[q] != -INFINITY) se += exp(L[q] - mx);
        se = warp_sum_d(se);
        const double lse = mx + log(se);
#pragma unroll
        for (int q = 0; q < kMaxJ / 32; ++q) {
            const int j = lane + 32 * q;
            if (j < J) a.log_b[j] = (float)(L[q] - lse);
        }
    }
}

} // namespace

cudaError_t launch_posterior(const PosteriorArgs &a, cudaStream_t s)
{
    const int J = a.G * a.B;
    int threads = 32 * J;
    if (threads > 1024) threads = 1024;
    posterior_kernel<<<1, threads, 0, s>>>(a);
    return cudaGetLastError();
}

} // namespace pm
