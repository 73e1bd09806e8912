// pm_mppi.cu -- the local planner of Sec. III-C on the predicted occupancy:
// model predictive path integral control for the robot of Eq. 8.
//
// mppi_rollout_kernel: one thread per sample. It applies u_ref[t] +
// delta[t][i] for t = 0..T-1 with explicit Euler steps of the unicycle with
// acceleration (x += v cos(th) dt, y += v sin(th) dt, v += a dt, th += w dt),
// charges after every step the quadratic state and control costs, a
// per-step cost, and the collision cost when the predicted occupancy at the
// robot's cell (prediction step (t+1)*pred_stride - 1) reaches the
// threshold, then adds the terminal cost and turns the running costs into the
// cost-to-go S_i(t) in place (suffix sums, from the last step back).
//
// mppi_update_kernel: one CTA per step t. The path-integral average of the
// perturbations, u*[t] = u_ref[t] + sum_i w_i delta[t][i] / sum_i w_i with
// w_i = exp(-(S_i(t) - min_i S_i(t)) / tau): a block minimum, then block sums
// in a fixed order (deterministic).
#include <cuda_runtime.h>

#include "pm_kernels.cuh"

namespace pm {
namespace {

constexpr int kMppiThreads = 256;

__global__ void __launch_bounds__(kMppiThreads) mppi_rollout_kernel(const __grid_constant__ MppiArgs a)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.N) return;
    float x = a.z0[0], y = a.z0[1], v = a.z0[2], th = a.z0[3];
    const float dt = a.dt;
    for (int t = 0; t < a.T; ++t) {
        const float2 d = reinterpret_cast<const float2 *>(a.delta)[(size_t)t * a.N + i];
        const float ua = a.u_ref[2 * t] + d.x, uw = a.u_ref[2 * t + 1] + d.y;
        float sn, cs;
        sincosf(th, &sn, &cs);
        const float x1 = x + v * cs * dt, y1 = y + v * sn * dt;
        const float v1 = v + ua * dt, th1 = th + uw * dt;
        const float ex = x1 - a.goal[0], ey = y1 - a.goal[1], ev = v1 - a.goal[2], et = th1 - a.goal[3];
        float c = a.q[0] * ex * ex + a.q[1] * ey * ey + a.q[2] * ev * ev + a.q[3] * et * et + a.r[0] * ua * ua +
                  a.r[1] * uw * uw + a.step_cost;
        const int k = (t + 1) * a.pred_stride - 1;
        if (a.prob && k < a.prob_T) {
            const float vx = __fmul_rn(__fsub_rn(x1, a.gx0), a.inv_res);
            const float vy = __fmul_rn(__fsub_rn(y1, a.gy0), a.inv_res);
            const float fx = floorf(vx), fy = floorf(vy);
            if (fx >= 0.0f && fx < (float)a.W && fy >= 0.0f && fy < (float)a.H) {
                const float p = a.prob[((size_t)k * a.H + (int)fy) * a.W + (int)fx];
                if (p >= a.coll_threshold) c += a.coll_cost;
            }
        }
        a.ctg[(size_t)t * a.N + i] = c; // running cost for now
        x = x1;
        y = y1;
        v = v1;
        th = th1;
    }
    const float ex = x - a.goal[0], ey = y - a.goal[1], ev = v - a.goal[2], et = th - a.goal[3];
    float acc = a.q_final[0] * ex * ex + a.q_final[1] * ey * ey + a.q_final[2] * ev * ev + a.q_final[3] * et * et;
    for (int t = a.T - 1; t >= 0; --t) {
        acc += a.ctg[(size_t)t * a.N + i];
        a.ctg[(size_t)t * a.N + i] = acc;
    }
}

__device__ __forceinline__ float block_reduce(float v, float *sh, bool is_min)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float u = __shfl_xor_sync(0xffffffffu, v, o);
        v = is_min ? fminf(v, u) : v + u;
    }
    __syncthreads(); // sh is free
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    v = (lane < nw) ? sh[lane] : (is_min ? INFINITY : 0.0f);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float u = __shfl_xor_sync(0xffffffffu, v, o);
        v = is_min ? fminf(v, u) : v + u;
    }
    return v; // every thread holds the result
}

__global__ void __launch_bounds__(kMppiThreads) mppi_update_kernel(const __grid_constant__ MppiArgs a)
{
    __shared__ float sh[32];
    const int t = blockIdx.x;
    const float *S = a.ctg + (size_t)t * a.N;
    const float2 *D = reinterpret_cast<const float2 *>(a.delta) + (size_t)t * a.N;
    float mn = INFINITY;
    for (int i = threadIdx.x; i < a.N; i += blockDim.x) mn = fminf(mn, S[i]);
    mn = block_reduce(mn, sh, true);
    const float inv_tau = 1.0f / a.temperature;
    float sw = 0.0f, sa = 0.0f, so = 0.0f;
    for (int i = threadIdx.x; i < a.N; i += blockDim.x) {
        const float w = expf(-(S[i] - mn) * inv_tau);
        const float2 d = D[i];
        sw += w;
        sa = fmaf(w, d.x, sa);
        so = fmaf(w, d.y, so);
    }
    sw = block_reduce(sw, sh, false);
    sa = block_reduce(sa, sh, false);
    so = block_reduce(so, sh, false);
    if (threadIdx.x == 0) {
        a.u_opt[2 * t] = a.u_ref[2 * t] + sa / sw;
        a.u_opt[2 * t + 1] = a.u_ref[2 * t + 1] + so / sw;
    }
}

} // namespace

cudaError_t launch_mppi(const MppiArgs &a, cudaStream_t s)
{
    if (a.N <= 0 || a.T <= 0) return cudaSuccess;
    mppi_rollout_kernel<<<(a.N + kMppiThreads - 1) / kMppiThreads, kMppiThreads, 0, s>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    mppi_update_kernel<<<a.T, kMppiThreads, 0, s>>>(a);
    return cudaGetLastError();
}

} // namespace pm
