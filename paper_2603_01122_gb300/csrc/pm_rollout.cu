// pm_rollout.cu -- Algorithm 1 (hardware-accelerated human prediction) with the
// bootstrapped belief of Sec. III-B and the per-step emplacement onto an
// occupancy grid, as one fused kernel: one lane per particle, persistent
// warps.
//
// Per particle and step (the hot loop), for every heading k:
//   distance from the next state to the goal, d_k = sqrt(D + 2 s e_k.(z - g))
//   with D = ||z - g||^2 + s^2, taken from the approximate square root plus
//   one Newton correction from its residual, so that beta*w2*(d_j - d_k)
//   keeps FP32 relative precision even when ||z - g|| >> s (a plain FP32
//   distance of a 5 m vector carries 5e-7 m of rounding, i.e. 5e-5 of logit at
//   beta = 100); logits beta*Q_k up to a common shift are -beta*w2*d_k (w1
//   cancels, Eq. 2), shifted by a bound of the extreme distance (or the exact
//   extreme) so that every exponent is <= 0, then ex2.approx on the SFU;
//   weights are rounded to 23-bit fixed point so that the running sums C_k of
//   the inverse CDF are exact integers (the sampling decision then depends
//   only on the rounded weights, not on summation order).
// The drawn heading moves the FP32 state by one Euler step (Eq. 1); the state
// is binned with FP32 operations (x - x0) * inv_res and the lanes of the warp
// that land in the same cell are combined (match.any) into one global
// reduction per cell and step.
// rollout_multi_kernel<KT> is the same kernel for a control set of several
// speeds (controls = speeds x headings, Sec. IV-B): the fused per-speed draw
// for K = KT, the general one for any K (KT = 0).
#include <cuda_runtime.h>

#include "pm_internal.cuh"
#include "pm_rollout_dev.cuh"

namespace pm {
namespace {


constexpr int kWarpCtaThreads = 128; // 4 warps: one per SM sub-partition
constexpr int kWarpCtaMinBlocks = 6;

// Every warp leaves the chunk loop once, after its last (failed) grab; the
// last one to leave resets the counter head[0] and its own count head[2], so
// each launch finds both at zero without a memset before it (the counters
// are zeroed when the context allocates them).
__device__ __forceinline__ void release_counter(unsigned *head, int lane)
{
    if (lane != 0) return;
    const unsigned warps = gridDim.x * (blockDim.x >> 5);
    if (atomicAdd(head + 2, 1u) == warps - 1u) {
        atomicExch(head, 0u);
        atomicExch(head + 2, 0u);
    }
}

// Persistent warps over one human: the CTA loads the component table, the
// belief CDF and the Euler steps into shared memory once, then each warp
// takes chunks of 32 particles (one per lane) from a global counter until the
// particles are exhausted, so the work spreads evenly over the schedulers and
// SMs whatever the particle count.
template <int KT, bool FULL>
__global__ void __launch_bounds__(kWarpCtaThreads, kWarpCtaMinBlocks)
    rollout_warp_kernel(const __grid_constant__ RolloutArgs a, unsigned *head)
{
    __shared__ float4 comp[kMaxJ];
    __shared__ uint32_t cdf[kMaxJ];
    __shared__ float2 step[kMaxK];
    const int tid = threadIdx.x, lane = tid & 31;
    const int J = a.G * a.B;
    for (int j = tid; j < J; j += blockDim.x) {
        const int g = j / a.B, b = j - g * a.B;
        const float cbj = a.beta[b] * a.w2_log2e;
        comp[j] = make_float4(cbj, a.goals[2 * g], a.goals[2 * g + 1], lb_flag(a.tab, cbj));
        if (bad_component(cbj, comp[j].y, comp[j].z)) flag_status(a.status, kStatusModel);
    }
    for (int k = tid; k < KT; k += blockDim.x) step[k] = make_float2(a.tab.sx[k], a.tab.sy[k]);
    if (tid < 32 && belief_cdf(a.log_b, J, cdf, tid) && tid == 0) flag_status(a.status, kStatusBelief);
    __syncthreads();

    TileCtx c;
    c.z0x = a.z0x;
    c.z0y = a.z0y;
    c.T = a.T;
    c.N = a.N;
    c.n_trace = a.n_trace;
    c.seed = a.seed;
    c.human = a.human;
    c.J = J;
    c.hist = a.counts != nullptr;
    c.gx0 = a.gx0;
    c.gy0 = a.gy0;
    c.inv_res = a.inv_res;
    c.W = a.W;
    c.H = a.H;
    c.cx_off = 0;
    c.cy_off = 0;
    c.counts = a.counts;
    c.oob = a.oob;
    c.win_x0 = c.win_y0 = c.ww = c.wh = 0;
    c.tr_states = a.tr_states;
    c.tr_head = a.tr_head;
    c.tr_comp = a.tr_comp;
    c.flags = nullptr;
    c.fbx = c.fplane = 0;
    for (;;) {
        unsigned item = 0;
        if (lane == 0) item = atomicAdd(head, 1u);
        item = __shfl_sync(0xffffffffu, item, 0);
        const int64_t i0 = (int64_t)item * 32;
        if (i0 >= a.N) break;
        c.i = i0 + lane;
        rollout_lane<KT, FULL>(a.tab, a.enabled, a.s2, c, comp, cdf, step);
    }
    release_counter(head, lane);
}

// The same persistent warps for a control set of several speeds: KT > 0 is
// the heading count of the fused draw (K == KT), KT = 0 the general draw.
template <int KT>
__global__ void __launch_bounds__(kWarpCtaThreads, kWarpCtaMinBlocks)
    rollout_multi_kernel(const __grid_constant__ RolloutArgs a, unsigned *head)
{
    __shared__ float4 comp[kMaxJ];
    __shared__ float betas[kMaxJ];
    __shared__ uint32_t cdf[kMaxJ];
    __shared__ float2 step[PM_MAX_SPEEDS * kMaxK];
    const int tid = threadIdx.x, lane = tid & 31;
    const int J = a.G * a.B;
    for (int j = tid; j < J; j += blockDim.x) {
        const int g = j / a.B, b = j - g * a.B;
        const float cbj = a.beta[b] * a.w2_log2e;
        comp[j] = make_float4(cbj, a.goals[2 * g], a.goals[2 * g + 1], lb_flag(a.tab, cbj));
        if (bad_component(cbj, comp[j].y, comp[j].z)) flag_status(a.status, kStatusModel);
        betas[j] = a.beta[b];
    }
    for (int u = tid; u < a.tab.S * a.K; u += blockDim.x)
        step[u] = make_float2(a.tab.msx[u / a.K][u % a.K], a.tab.msy[u / a.K][u % a.K]);
    if (tid < 32 && belief_cdf(a.log_b, J, cdf, tid) && tid == 0) flag_status(a.status, kStatusBelief);
    __syncthreads();

    TileCtx c;
    c.z0x = a.z0x;
    c.z0y = a.z0y;
    c.T = a.T;
    c.N = a.N;
    c.n_trace = a.n_trace;
    c.seed = a.seed;
    c.human = a.human;
    c.J = J;
    c.hist = a.counts != nullptr;
    c.gx0 = a.gx0;
    c.gy0 = a.gy0;
    c.inv_res = a.inv_res;
    c.W = a.W;
    c.H = a.H;
    c.cx_off = 0;
    c.cy_off = 0;
    c.counts = a.counts;
    c.oob = a.oob;
    c.win_x0 = c.win_y0 = c.ww = c.wh = 0;
    c.tr_states = a.tr_states;
    c.tr_head = a.tr_head;
    c.tr_comp = a.tr_comp;
    c.flags = nullptr;
    c.fbx = c.fplane = 0;
    for (;;) {
        unsigned item = 0;
        if (lane == 0) item = atomicAdd(head, 1u);
        item = __shfl_sync(0xffffffffu, item, 0);
        const int64_t i0 = (int64_t)item * 32;
        if (i0 >= a.N) break;
        c.i = i0 + lane;
        rollout_lane<KT, false, true>(a.tab, a.enabled, a.s2, c, comp, cdf, step, betas, a.K, a.tab.speed_on);
    }
    release_counter(head, lane);
}

template <int KT>
cudaError_t launch_multi(const RolloutArgs &a, unsigned *head, int sm_count, cudaStream_t s, int *occ)
{
    int n = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, rollout_multi_kernel<KT>, kWarpCtaThreads, 0);
    if (e != cudaSuccess) return e;
    if (occ) {
        *occ = n;
        return cudaSuccess;
    }
    const int64_t chunks = ((int64_t)a.N + 31) / 32;
    const int64_t need = (chunks + kWarpCtaThreads / 32 - 1) / (kWarpCtaThreads / 32);
    int64_t blocks = (int64_t)sm_count * (n > 0 ? n : 1);
    if (need < blocks) blocks = need;
    cudaGetLastError();
    rollout_multi_kernel<KT><<<(unsigned)blocks, kWarpCtaThreads, 0, s>>>(a, head);
    return cudaGetLastError();
}

template <int KT>
cudaError_t launch_kt(const RolloutArgs &a, unsigned *head, int sm_count, cudaStream_t s, int *occ)
{
    const uint64_t all = (KT >= 64) ? ~0ull : ((1ull << KT) - 1ull);
    const bool full = (a.K == KT) && ((a.enabled & all) == all);
    auto k = full ? rollout_warp_kernel<KT, true> : rollout_warp_kernel<KT, false>;
    int n = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, kWarpCtaThreads, 0);
    if (e != cudaSuccess) return e;
    if (occ) {
        *occ = n;
        return cudaSuccess;
    }
    const int64_t chunks = ((int64_t)a.N + 31) / 32;
    const int64_t need = (chunks + kWarpCtaThreads / 32 - 1) / (kWarpCtaThreads / 32);
    int64_t blocks = (int64_t)sm_count * (n > 0 ? n : 1);
    if (need < blocks) blocks = need;
    cudaGetLastError(); // clear errors of earlier calls whose failure was handled
    k<<<(unsigned)blocks, kWarpCtaThreads, 0, s>>>(a, head);
    return cudaGetLastError();
}

cudaError_t dispatch(const RolloutArgs &a, unsigned *head, int sm_count, cudaStream_t s, int *occ)
{
    if (a.tab.S > 0) { // several speeds (all K headings enabled, K % 4 == 0)
        switch (a.K) {
        case 16: return launch_multi<16>(a, head, sm_count, s, occ);
        case 32: return launch_multi<32>(a, head, sm_count, s, occ);
        case 36: return launch_multi<36>(a, head, sm_count, s, occ);
        default: return launch_multi<0>(a, head, sm_count, s, occ);
        }
    }
    switch (rollout_kt_for(a.K)) {
    case 8: return launch_kt<8>(a, head, sm_count, s, occ);
    case 16: return launch_kt<16>(a, head, sm_count, s, occ);
    case 36: return launch_kt<36>(a, head, sm_count, s, occ);
    default: return launch_kt<64>(a, head, sm_count, s, occ);
    }
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

cudaError_t launch_rollout(const RolloutArgs &a, unsigned *head, int sm_count, cudaStream_t s)
{
    return dispatch(a, head, sm_count, s, nullptr);
}

} // namespace pm
