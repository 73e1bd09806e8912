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
#include "pm_rollout_dev.cuh"

namespace pm {
namespace {

constexpr int kRolloutThreads = 256;

// Resident CTAs per SM the compiler is asked to fit: the warp-histogram forms
// use almost no shared memory, so registers decide their occupancy.
template <int PPT, bool WARP_HIST>
constexpr int rollout_min_blocks()
{
    return WARP_HIST ? (PPT == 1 ? 3 : 2) : 3;
}

template <int KT, bool FULL, int PPT, bool WARP_HIST>
__global__ void __launch_bounds__(kRolloutThreads, (rollout_min_blocks<PPT, WARP_HIST>()))
    rollout_kernel(const __grid_constant__ RolloutArgs a)
{
    __shared__ RolloutShared sh;
    extern __shared__ __align__(16) uint32_t dyn[];
    const int tid = threadIdx.x;
    const int nthr = blockDim.x;
    const int J = a.G * a.B;
    const bool hist = a.counts != nullptr;
    const int ww = a.win_side & 0xFFFF, wh = a.win_side >> 16; // window width/height (cells)

    for (int j = tid; j < J; j += nthr) {
        const int g = j / a.B, b = j - g * a.B;
        sh.comp[j] = make_float4(a.beta[b] * a.w2_log2e, a.goals[2 * g], a.goals[2 * g + 1], 0.0f);
    }
    for (int k = tid; k < KT; k += nthr) sh.step[k] = make_float2(a.tab.sx[k], a.tab.sy[k]);
    if (hist && !WARP_HIST) {
        const int win_words = 2 * window_stride_words(ww, wh); // both windows
        for (int w = tid; w < win_words; w += nthr) dyn[w] = 0u;
    }
    if (tid < 3) sh.list_n[tid] = 0u;
    if (tid < 2) sh.oob_n[tid] = 0u;
    if (tid < 32) belief_cdf(a.log_b, J, sh.cdf, tid);
    __syncthreads();

    TileCtx c;
    c.z0x = a.z0x;
    c.z0y = a.z0y;
    c.T = a.T;
    c.i = (int64_t)blockIdx.x * nthr * PPT + tid;
    c.N = a.N;
    c.n_trace = a.n_trace;
    c.seed = a.seed;
    c.human = a.human;
    c.J = J;
    c.hist = hist;
    c.gx0 = a.gx0;
    c.gy0 = a.gy0;
    c.inv_res = a.inv_res;
    c.W = a.W;
    c.H = a.H;
    c.cx_off = 0;
    c.cy_off = 0;
    c.counts = a.counts;
    c.oob = a.oob;
    c.win_x0 = a.win_x0;
    c.win_y0 = a.win_y0;
    c.ww = ww;
    c.wh = wh;
    c.tr_states = a.tr_states;
    c.tr_head = a.tr_head;
    c.tr_comp = a.tr_comp;
    rollout_tile<KT, FULL, PPT, WARP_HIST>(a.tab, a.enabled, a.s2, c, sh, dyn);
}

template <int KT, bool FULL, int PPT, bool WH>
cudaError_t launch_one(const RolloutArgs &a, int threads, size_t dyn_smem, cudaStream_t s, int *occ)
{
    auto k = rollout_kernel<KT, FULL, PPT, WH>;
    if (dyn_smem > 0) { // static + dynamic may pass the 48 KiB default
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn_smem);
        if (e != cudaSuccess) return e;
    }
    if (occ) return cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, k, threads, dyn_smem);
    const unsigned blocks = (unsigned)((a.N + (int64_t)threads * PPT - 1) / ((int64_t)threads * PPT));
    cudaGetLastError(); // clear errors of earlier calls whose failure was handled
    k<<<blocks, threads, dyn_smem, s>>>(a);
    return cudaGetLastError();
}

template <int KT, bool FULL>
cudaError_t launch_shape(const RolloutArgs &a, const RolloutShape &sh, size_t dyn, cudaStream_t s, int *occ)
{
    if (sh.warp_hist) {
        if (sh.ppt == 2) return launch_one<KT, FULL, 2, true>(a, sh.threads, dyn, s, occ);
        return launch_one<KT, FULL, 1, true>(a, sh.threads, dyn, s, occ);
    }
    return launch_one<KT, FULL, 1, false>(a, sh.threads, dyn, s, occ);
}

template <int KT>
cudaError_t launch_kt(const RolloutArgs &a, const RolloutShape &sh, size_t dyn, cudaStream_t s, int *occ)
{
    const uint64_t all = (KT >= 64) ? ~0ull : ((1ull << KT) - 1ull);
    const bool full = (a.K == KT) && ((a.enabled & all) == all);
    if (full) return launch_shape<KT, true>(a, sh, dyn, s, occ);
    return launch_shape<KT, false>(a, sh, dyn, s, occ);
}

cudaError_t dispatch(const RolloutArgs &a, const RolloutShape &sh, size_t dyn, cudaStream_t s, int *occ)
{
    switch (rollout_kt_for(a.K)) {
    case 8: return launch_kt<8>(a, sh, dyn, s, occ);
    case 16: return launch_kt<16>(a, sh, dyn, s, occ);
    case 36: return launch_kt<36>(a, sh, dyn, s, occ);
    default: return launch_kt<64>(a, sh, dyn, s, occ);
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

int rollout_occupancy(const RolloutArgs &a, const RolloutShape &shape, size_t dyn_smem)
{
    int n = 0;
    if (dispatch(a, shape, dyn_smem, nullptr, &n) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

cudaError_t launch_rollout(const RolloutArgs &a, const RolloutShape &shape, size_t dyn_smem, cudaStream_t s)
{
    return dispatch(a, shape, dyn_smem, s, nullptr);
}

} // namespace pm
