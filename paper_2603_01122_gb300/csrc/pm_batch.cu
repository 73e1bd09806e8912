// pm_batch.cu -- many humans in one persistent launch.
//
// The work list holds tiles (human, first particle), sorted on the host by
// horizon (longest first). A grid of SMs x CTAs-per-SM persistent CTAs (or
// warps) takes tiles from a global counter (one atomicAdd per tile, no
// waiting), loads the human's component table and belief CDF into shared
// memory when the human changes and runs Algorithm 1 for the tile with the
// same device code as the single-human kernel, so each human's histogram is
// bit-identical alone and in the mix (its random numbers are keyed on
// (seed, human_id, particle) only and the counts are integer sums).
// Every human of a batch shares K, v, dt, w, the speeds and the disabled
// headings (the heading tables live in the kernel parameters); goals, beta
// grid, belief, start, particles, horizon, output and the speeds masked for
// the human differ per human.
//
// Two forms: batch_warp_kernel (persistent warps take 32-particle tiles and
// emplace with warp-combined global reductions; optionally also mark the
// occupied 16 x 16-cell blocks for the union epilogue) and
// batch_rollout_kernel (CTAs take tiles of blockDim particles and count each
// step in a shared-memory window around the human's start cell). The
// autotuner times both.
#include <algorithm>
#include <climits>

#include <cuda_runtime.h>

#include "pm_kernels.cuh"
#include "pm_rollout_dev.cuh"

namespace pm {
namespace {

constexpr int kBatchMaxThreads = 256;

// Window form: a CTA takes a tile of blockDim particles and counts each step
// in its shared-memory window (rollout_tile), one particle per thread.
template <int KT, bool FULL>
__global__ void __launch_bounds__(kBatchMaxThreads, 3) batch_rollout_kernel(const __grid_constant__ BatchArgs a)
{
    __shared__ RolloutShared sh;
    __shared__ int s_item;
    __shared__ int s_geom[6]; // cx_off, cy_off, win_x0, win_y0, ww, wh
    __shared__ float s_z0[2];
    extern __shared__ __align__(16) uint32_t dyn[];
    const int tid = threadIdx.x, nthr = blockDim.x;
    for (int k = tid; k < KT; k += nthr) sh.step[k] = make_float2(a.tab.sx[k], a.tab.sy[k]);
    const int n_items = *a.n_items;
    int cur = -1;
    for (;;) {
        __syncthreads(); // the previous tile is done with shared memory
        if (tid == 0) s_item = (int)atomicAdd(a.head, 1u);
        __syncthreads();
        const int it = s_item;
        if (it >= n_items) break;
        const int2 item = a.items[it]; // (human, first particle)
        const BatchHuman *h = a.humans + item.x;
        const int J = h->G * h->B;
        if (item.x != cur) {
            for (int j = tid; j < J; j += nthr) {
                const int g = j / h->B, b = j - g * h->B;
                const float cbj = h->beta[b] * a.w2_log2e;
                sh.comp[j] = make_float4(cbj, h->goals[2 * g], h->goals[2 * g + 1], lb_flag(a.tab, cbj));
                if (bad_component(cbj, sh.comp[j].y, sh.comp[j].z)) flag_status(a.status, kStatusModel);
            }
            if (tid < 32 && belief_cdf(h->log_b, J, sh.cdf, tid) && tid == 0) flag_status(a.status, kStatusBelief);
            cur = item.x;
        }
        if (tid == 0) {
            const float zx = h->z0[0], zy = h->z0[1];
            // start cell on the binning grid, with the same FP32 rule as the states
            const int gcx = __float2int_rd(__fmul_rn(__fsub_rn(zx, h->gx0), h->inv_res));
            const int gcy = __float2int_rd(__fmul_rn(__fsub_rn(zy, h->gy0), h->inv_res));
            int cx_off = h->cx_off, cy_off = h->cy_off;
            if (h->center) {
                cx_off = gcx - (h->W - 1) / 2;
                cy_off = gcy - (h->H - 1) / 2;
            }
            const int cxo = gcx - cx_off, cyo = gcy - cy_off;
            int r = min(h->reach_cells, a.win_radius_cap);
            int x_lo = max(cxo - r, 0), x_hi = min(cxo + r, h->W - 1);
            int y_lo = max(cyo - r, 0), y_hi = min(cyo + r, h->H - 1);
            int ww = x_hi - x_lo + 1, wh = y_hi - y_lo + 1;
            if (ww <= 0 || wh <= 0) ww = wh = 0, x_lo = y_lo = 0;
            s_geom[0] = cx_off;
            s_geom[1] = cy_off;
            s_geom[2] = x_lo;
            s_geom[3] = y_lo;
            s_geom[4] = ww;
            s_geom[5] = wh;
            s_z0[0] = zx;
            s_z0[1] = zy;
        }
        if (tid < 3) sh.list_n[tid] = 0u;
        if (tid < 2) sh.oob_n[tid] = 0u;
        __syncthreads();
        {
            const int words = 2 * window_stride_words(s_geom[4], s_geom[5]);
            for (int w = tid; w < words; w += nthr) dyn[w] = 0u;
        }
        __syncthreads();
        TileCtx c;
        c.z0x = s_z0[0];
        c.z0y = s_z0[1];
        c.T = h->T;
        c.i = (int64_t)item.y + tid;
        c.N = h->N;
        c.n_trace = 0;
        c.seed = h->seed;
        c.human = h->human;
        c.J = J;
        c.hist = true;
        c.gx0 = h->gx0;
        c.gy0 = h->gy0;
        c.inv_res = h->inv_res;
        c.W = h->W;
        c.H = h->H;
        c.cx_off = s_geom[0];
        c.cy_off = s_geom[1];
        c.counts = h->counts;
        c.oob = h->oob;
        c.win_x0 = s_geom[2];
        c.win_y0 = s_geom[3];
        c.ww = s_geom[4];
        c.wh = s_geom[5];
        c.tr_states = nullptr;
        c.tr_head = nullptr;
        c.tr_comp = nullptr;
        c.flags = nullptr; // the window form writes no block flags
        c.fbx = c.fplane = 0;
        rollout_tile<KT, FULL, 1, false>(a.tab, a.enabled, a.s2, c, sh, dyn);
    }
}

// Bytes of one warp's tables in dynamic shared memory: comp[kMaxJ] (16 B
// each) then cdf[kMaxJ] (4 B each). Sized for the library's largest G*B, not
// for the current batch, so that a CUDA graph captured on one batch stays
// valid when humans with more components join later.
constexpr size_t kWarpTableBytes = (size_t)kMaxJ * 20;
// Several speeds: also the components' beta[kMaxJ] (4 B each) after cdf.
constexpr size_t kWarpTableBytesMS = (size_t)kMaxJ * 24;

// Persistent warps over all humans: each warp takes a 32-particle tile
// (human, first particle) from the global counter, loads that human's
// component table and belief CDF into its own slice of shared memory when
// the human changes, and runs the tile with the warp-combined emplacement.
// No block barrier after the start, so tiles of different humans and
// horizons mix freely on every scheduler.
// MS: the control set of several speeds (draw_multi).
// MARKS: also write the block occupancy flags (a separate instantiation, so
// the kernel without marks carries none of their code).
template <int KT, bool FULL, bool MS = false, bool MARKS = false>
__device__ __forceinline__ void batch_warp_body(const BatchArgs &a)
{
    __shared__ float2 step[MS ? PM_MAX_SPEEDS * kMaxK : kMaxK];
    extern __shared__ __align__(16) uint32_t dyn[];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if constexpr (MS) {
        for (int u = tid; u < a.tab.S * a.K; u += blockDim.x)
            step[u] = make_float2(a.tab.msx[u / a.K][u % a.K], a.tab.msy[u / a.K][u % a.K]);
    } else {
        for (int k = tid; k < KT; k += blockDim.x) step[k] = make_float2(a.tab.sx[k], a.tab.sy[k]);
    }
    __syncthreads();
    char *slab = reinterpret_cast<char *>(dyn) + (size_t)warp * (MS ? kWarpTableBytesMS : kWarpTableBytes);
    float4 *comp = reinterpret_cast<float4 *>(slab);
    uint32_t *cdf = reinterpret_cast<uint32_t *>(slab + (size_t)kMaxJ * 16);
    float *betas = reinterpret_cast<float *>(slab + (size_t)kMaxJ * 20); // MS only
    const int n_items = *a.n_items;
    int cur = -1;
    for (;;) {
        unsigned it = 0;
        if (lane == 0) it = atomicAdd(a.head, 1u);
        it = __shfl_sync(0xffffffffu, it, 0);
        if ((int)it >= n_items) break;
        const int2 item = a.items[it]; // (human, first particle)
        const BatchHuman *h = a.humans + item.x;
        const int J = min(h->G * h->B, kMaxJ); // the host rejects larger models
        if (item.x != cur) {
            __syncwarp();
            bool bad = false;
            for (int j = lane; j < J; j += 32) {
                const int g = j / h->B, b = j - g * h->B;
                const float cbj = h->beta[b] * a.w2_log2e;
                const float gx = h->goals[2 * g], gy = h->goals[2 * g + 1];
                comp[j] = make_float4(cbj, gx, gy, lb_flag(a.tab, cbj));
                bad = bad || bad_component(cbj, gx, gy);
                if constexpr (MS) betas[j] = h->beta[b];
            }
            // one latch per warp and human for unusable inputs
            const unsigned bits = belief_cdf(h->log_b, J, cdf, lane) | (__any_sync(0xffffffffu, bad) ? kStatusModel : 0u);
            if (lane == 0 && bits) flag_status(a.status, bits);
            __syncwarp();
            cur = item.x;
        }
        const float zx = h->z0[0], zy = h->z0[1];
        int cx_off = h->cx_off, cy_off = h->cy_off;
        if (h->center) {
            // the output window is centred on the start cell (same FP32 rule as the states)
            cx_off = __float2int_rd(__fmul_rn(__fsub_rn(zx, h->gx0), h->inv_res)) - (h->W - 1) / 2;
            cy_off = __float2int_rd(__fmul_rn(__fsub_rn(zy, h->gy0), h->inv_res)) - (h->H - 1) / 2;
        }
        TileCtx c;
        c.z0x = zx;
        c.z0y = zy;
        c.T = h->T;
        c.i = (int64_t)item.y + lane;
        c.N = h->N;
        c.n_trace = 0;
        c.seed = h->seed;
        c.human = h->human;
        c.J = J;
        c.hist = true;
        c.gx0 = h->gx0;
        c.gy0 = h->gy0;
        c.inv_res = h->inv_res;
        c.W = h->W;
        c.H = h->H;
        c.cx_off = cx_off;
        c.cy_off = cy_off;
        c.counts = h->counts;
        c.oob = h->oob;
        c.win_x0 = c.win_y0 = c.ww = c.wh = 0;
        c.tr_states = nullptr;
        c.tr_head = nullptr;
        c.tr_comp = nullptr;
        c.flags = MARKS ? h->flags : nullptr;
        c.fbx = h->fbx;
        c.fplane = h->fbx * h->fby;
        if constexpr (MS)
            rollout_lane<KT, false, true>(a.tab, a.enabled, a.s2, c, comp, cdf, step, betas, a.K, h->speed_on);
        else rollout_lane<KT, FULL>(a.tab, a.enabled, a.s2, c, comp, cdf, step);
    }
}

// Two register budgets of the same body: 80 registers (6 CTAs of 128 threads
// per SM), and 72 (7 CTAs) for the one-speed instantiations with K <= 36,
// which do not spill there (24 bytes with marks); the 64-human served frame
// is 0.6 % faster with 7. K = 64 and several speeds spill at 72 and keep 80.
template <int KT, bool FULL, bool MS = false, bool MARKS = false>
__global__ void __launch_bounds__(kBatchMaxThreads, 3) batch_warp_kernel(const __grid_constant__ BatchArgs a)
{
    batch_warp_body<KT, FULL, MS, MARKS>(a);
}

template <int KT, bool FULL, bool MARKS = false>
__global__ void __maxnreg__(72) batch_warp_kernel72(const __grid_constant__ BatchArgs a)
{
    batch_warp_body<KT, FULL, false, MARKS>(a);
}

// Output cells [x0, x1] x [y0, y1] that a particle started at z can occupy
// after t steps of at most smax each: the start cell (by the rollout's own
// FP32 rule) widened by ceil(R / res) + 3 cells, R = t smax plus a bound on
// the rounding the t FP32 position additions can accumulate; the extra cells
// cover the rounding of the binning. Empty when x0 > x1 or y0 > y1.
struct ReachBox {
    int x0, x1, y0, y1;
};

__device__ __forceinline__ ReachBox reach_box(const BatchHuman &h, float zx, float zy, int t, float smax)
{
    const int gcx = __float2int_rd(__fmul_rn(__fsub_rn(zx, h.gx0), h.inv_res));
    const int gcy = __float2int_rd(__fmul_rn(__fsub_rn(zy, h.gy0), h.inv_res));
    int cx_off = h.cx_off, cy_off = h.cy_off;
    if (h.center) {
        cx_off = gcx - (h.W - 1) / 2;
        cy_off = gcy - (h.H - 1) / 2;
    }
    const float R = (float)t * smax;
    const float err = (float)t * (fabsf(zx) + fabsf(zy) + R) * 0x1p-22f;
    const int rc = (int)fminf(ceilf((R + err) * h.inv_res), 4194304.0f) + 3;
    ReachBox r;
    r.x0 = max(gcx - cx_off - rc, 0);
    r.x1 = min(gcx - cx_off + rc, h.W - 1);
    r.y0 = max(gcy - cy_off - rc, 0);
    r.y1 = min(gcy - cy_off + rc, h.H - 1);
    return r;
}

// Zero every human's counts [T][H][W], oob [T] and block flags: blockIdx.y
// strides over humans, the x dimension over 16-byte words of the counts
// (scalar head and tail).
__global__ void batch_zero_kernel(const BatchHuman *humans, const int *n_dev)
{
    const int n = *n_dev;
    for (int hh = blockIdx.y; hh < n; hh += gridDim.y) {
        const BatchHuman &h = humans[hh];
        const size_t words = (size_t)h.T * h.H * h.W;
        uint32_t *p = h.counts;
        const size_t head = ((16 - ((uintptr_t)p & 15)) & 15) / 4;
        const size_t lead = head < words ? head : words;
        const size_t nvec = (words - lead) / 4;
        const size_t tail0 = lead + nvec * 4;
        const size_t stride = (size_t)gridDim.x * blockDim.x;
        const size_t t0 = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
        uint4 *v = reinterpret_cast<uint4 *>(p + lead);
        for (size_t q = t0; q < nvec; q += stride) v[q] = make_uint4(0u, 0u, 0u, 0u);
        if (t0 < lead) p[t0] = 0u;
        if (t0 < words - tail0) p[tail0 + t0] = 0u;
        for (size_t q = t0; q < (size_t)h.T; q += stride) h.oob[q] = 0u;
        if (h.flags) {
            const size_t nf = (size_t)h.T * h.fbx * h.fby;
            for (size_t q = t0; q < nf; q += stride) h.flags[q] = 0u;
        }
    }
}

// The reachable-cells form. A warp per (human, step t, part g of
// kReachGroups): it zeroes oob[t] and the step's block flags (g = 0) and
// part g of one contiguous span of step t's counts: from the first to the
// last cell of the smallest rectangle holding
//  - the two boxes a particle can reach from this prediction's start z0 and
//    from the previous prediction's start into the same buffers (prev), or
//  - the whole plane, when the human has no recorded previous start (NaN) or
//    a non-finite start.
// The span's cells outside the boxes are zero already, so zeroing them again
// is harmless, and a contiguous span is written with 16-byte stores. Where
// the rectangle is more than kSpanSlack words narrower than the plane (the
// span would zero that much more per row than the rectangle), the warp
// zeroes the rectangle's rows r = g mod kReachGroups instead: the served
// 121-cell windows take the span, full 400-cell grids the rows. Every cell
// outside what is zeroed still holds the zero of an earlier pass, because no
// particle leaves its box. The last CTA to finish records each human's z0 in
// prev (ticket, no waiting; every CTA has read prev before it takes its
// ticket).
constexpr int kReachGroups = 4;
constexpr int kSpanSlack = 128; // extra words per row a span may zero before the rows are cheaper

// Zero n consecutive words at p with the lanes of a warp: 16-byte stores for
// the aligned body, single words for the head and the tail.
__device__ __forceinline__ void zero_span(uint32_t *p, long n, int lane)
{
    if (n <= 0) return;
    const int head = (int)min((long)((4u - (((uintptr_t)p >> 2) & 3u)) & 3u), n);
    const long body = (n - head) >> 2;
    const int tail = (int)((n - head) & 3);
    if (lane < head) p[lane] = 0u;
    uint4 *v = reinterpret_cast<uint4 *>(p + head);
    for (long i = lane; i < body; i += 32) v[i] = make_uint4(0u, 0u, 0u, 0u);
    if (lane < tail) p[head + 4 * body + lane] = 0u;
}

__global__ void batch_zero_reach_kernel(const BatchHuman *humans, const int *n_dev, float2 *prev, unsigned *ticket,
                                        float smax)
{
    const int n = n_dev[0], t_max = max(n_dev[1], 1); // humans and their longest horizon
    const int lane = threadIdx.x & 31;
    const long nwarp = ((long)gridDim.x * blockDim.x) >> 5;
    const long items = (long)n * t_max * kReachGroups;
    for (long it = ((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; it < items; it += nwarp) {
        const int g = (int)(it % kReachGroups);
        const int t = (int)((it / kReachGroups) % t_max);
        const int hh = (int)(it / ((long)kReachGroups * t_max));
        const BatchHuman &h = humans[hh];
        if (t >= h.T) continue;
        if (g == 0) {
            if (lane == 0) h.oob[t] = 0u;
            if (h.flags) {
                const int nf = h.fbx * h.fby;
                for (int q = lane; q < nf; q += 32) h.flags[(size_t)t * nf + q] = 0u;
            }
        }
        const float zx = h.z0[0], zy = h.z0[1];
        const float2 zp = prev[hh];
        long lo = 0, hi = (long)h.W * h.H; // the span [lo, hi) of the step's plane
        if (isfinite(zp.x) && isfinite(zp.y) && isfinite(zx) && isfinite(zy)) {
            const ReachBox a = reach_box(h, zx, zy, t + 1, smax);
            const ReachBox b = reach_box(h, zp.x, zp.y, t + 1, smax);
            const bool ea = a.x0 <= a.x1 && a.y0 <= a.y1, eb = b.x0 <= b.x1 && b.y0 <= b.y1;
            if (!ea && !eb) continue;
            const int x0 = min(ea ? a.x0 : INT_MAX, eb ? b.x0 : INT_MAX), x1 = max(ea ? a.x1 : -1, eb ? b.x1 : -1);
            const int y0 = min(ea ? a.y0 : INT_MAX, eb ? b.y0 : INT_MAX), y1 = max(ea ? a.y1 : -1, eb ? b.y1 : -1);
            lo = (long)y0 * h.W + x0;
            hi = (long)y1 * h.W + x1 + 1;
            if (h.W - (x1 - x0 + 1) > kSpanSlack) { // a rectangle much narrower than the plane: its rows
                uint32_t *stepp = h.counts + (size_t)t * h.W * h.H;
                for (int row = y0 + ((g - y0 % kReachGroups) + kReachGroups) % kReachGroups; row <= y1;
                     row += kReachGroups)
                    zero_span(stepp + (size_t)row * h.W + x0, x1 - x0 + 1, lane);
                continue;
            }
        }
        const long len = hi - lo, p0 = lo + len * g / kReachGroups, p1 = lo + len * (g + 1) / kReachGroups;
        zero_span(h.counts + (size_t)t * h.W * h.H + p0, p1 - p0, lane);
    }
    __shared__ bool last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(ticket, 1u) == gridDim.x - 1u;
    }
    __syncthreads();
    if (!last) return;
    for (int hh = threadIdx.x; hh < n; hh += blockDim.x) prev[hh] = make_float2(humans[hh].z0[0], humans[hh].z0[1]);
    if (threadIdx.x == 0) *ticket = 0u;
}

// The single-human form of the above: the counts in 16-byte words (scalar
// head and tail), oob and the chunk counter, so one launch replaces three
// memsets before the rollout.
__global__ void zero_outputs_kernel(uint32_t *counts, size_t words, uint32_t *oob, int T, unsigned *head)
{
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    const size_t t0 = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (counts) {
        const size_t lead0 = ((16 - ((uintptr_t)counts & 15)) & 15) / 4;
        const size_t lead = lead0 < words ? lead0 : words;
        const size_t nvec = (words - lead) / 4;
        const size_t tail0 = lead + nvec * 4;
        uint4 *v = reinterpret_cast<uint4 *>(counts + lead);
        for (size_t q = t0; q < nvec; q += stride) v[q] = make_uint4(0u, 0u, 0u, 0u);
        if (t0 < lead) counts[t0] = 0u;
        if (t0 < words - tail0) counts[tail0 + t0] = 0u;
    }
    if (oob)
        for (size_t q = t0; q < (size_t)T; q += stride) oob[q] = 0u;
    if (head && t0 == 0) *head = 0u;
}

template <typename Kern>
cudaError_t launch_or_query(Kern k, const BatchArgs &a, int blocks, int threads, size_t dyn, cudaStream_t s, int *occ)
{
    if (dyn > 0) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
        if (e != cudaSuccess) return e;
    }
    if (occ) return cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, k, threads, dyn);
    cudaGetLastError();
    k<<<blocks, threads, dyn, s>>>(a);
    return cudaGetLastError();
}

template <int KT, bool FULL>
cudaError_t batch_shape(const BatchArgs &a, const RolloutShape &sh, int blocks, size_t dyn, cudaStream_t s, int *occ)
{
    if (sh.warp_hist) {
        if constexpr (KT <= 36) {
            if (a.marks) return launch_or_query(batch_warp_kernel72<KT, FULL, true>, a, blocks, sh.threads, dyn, s, occ);
            return launch_or_query(batch_warp_kernel72<KT, FULL>, a, blocks, sh.threads, dyn, s, occ);
        } else {
            if (a.marks)
                return launch_or_query(batch_warp_kernel<KT, FULL, false, true>, a, blocks, sh.threads, dyn, s, occ);
            return launch_or_query(batch_warp_kernel<KT, FULL>, a, blocks, sh.threads, dyn, s, occ);
        }
    }
    return launch_or_query(batch_rollout_kernel<KT, FULL>, a, blocks, sh.threads, dyn, s, occ);
}

cudaError_t batch_dispatch(const BatchArgs &a, const RolloutShape &sh, int blocks, size_t dyn, cudaStream_t s, int *occ)
{
    if (a.tab.S > 0) { // several speeds: warp-combined emplacement only
        switch (a.K) {
        case 16:
            return a.marks ? launch_or_query(batch_warp_kernel<16, false, true, true>, a, blocks, sh.threads, dyn, s, occ)
                           : launch_or_query(batch_warp_kernel<16, false, true>, a, blocks, sh.threads, dyn, s, occ);
        case 32:
            return a.marks ? launch_or_query(batch_warp_kernel<32, false, true, true>, a, blocks, sh.threads, dyn, s, occ)
                           : launch_or_query(batch_warp_kernel<32, false, true>, a, blocks, sh.threads, dyn, s, occ);
        case 36:
            return a.marks ? launch_or_query(batch_warp_kernel<36, false, true, true>, a, blocks, sh.threads, dyn, s, occ)
                           : launch_or_query(batch_warp_kernel<36, false, true>, a, blocks, sh.threads, dyn, s, occ);
        default:
            return a.marks ? launch_or_query(batch_warp_kernel<0, false, true, true>, a, blocks, sh.threads, dyn, s, occ)
                           : launch_or_query(batch_warp_kernel<0, false, true>, a, blocks, sh.threads, dyn, s, occ);
        }
    }
    const int KT = rollout_kt_for(a.K);
    const uint64_t all = (KT >= 64) ? ~0ull : ((1ull << KT) - 1ull);
    const bool full = (a.K == KT) && ((a.enabled & all) == all);
    switch (KT) {
    case 8: return full ? batch_shape<8, true>(a, sh, blocks, dyn, s, occ) : batch_shape<8, false>(a, sh, blocks, dyn, s, occ);
    case 16: return full ? batch_shape<16, true>(a, sh, blocks, dyn, s, occ) : batch_shape<16, false>(a, sh, blocks, dyn, s, occ);
    case 36: return full ? batch_shape<36, true>(a, sh, blocks, dyn, s, occ) : batch_shape<36, false>(a, sh, blocks, dyn, s, occ);
    default: return full ? batch_shape<64, true>(a, sh, blocks, dyn, s, occ) : batch_shape<64, false>(a, sh, blocks, dyn, s, occ);
    }
}

} // namespace

size_t batch_warp_tables_bytes(int threads, bool multi_speed)
{
    return (size_t)(threads / 32) * (multi_speed ? kWarpTableBytesMS : kWarpTableBytes);
}

int batch_rollout_occupancy(int K, uint64_t enabled, int S, bool marks, const RolloutShape &shape, size_t dyn)
{
    BatchArgs a;
    a.K = K;
    a.enabled = enabled;
    a.tab.S = S;
    a.marks = marks ? 1 : 0;
    int n = 0;
    if (batch_dispatch(a, shape, 0, dyn, nullptr, &n) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

cudaError_t launch_batch_rollout(const BatchArgs &a, const RolloutShape &shape, int blocks, size_t dyn, cudaStream_t s)
{
    return batch_dispatch(a, shape, blocks, dyn, s, nullptr);
}

cudaError_t launch_zero_outputs(uint32_t *counts, size_t words, uint32_t *oob, int T, unsigned *head, int sm_count,
                                cudaStream_t s)
{
    // enough threads for a few 16-byte stores each at paper-scale sizes,
    // never more than the work
    const size_t nvec = words / 4 + 1;
    size_t blocks = (nvec + 255) / 256;
    const size_t cap = (size_t)(sm_count > 0 ? sm_count : 1) * 4;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    zero_outputs_kernel<<<(unsigned)blocks, 256, 0, s>>>(counts, words, oob, T, head);
    return cudaGetLastError();
}

cudaError_t launch_batch_zero(const BatchHuman *humans, const int *n_dev, int max_rows, int sm_count, int t_max,
                              float2 *prev, unsigned *ticket, float smax, cudaStream_t s)
{
    if (max_rows <= 0) return cudaSuccess;
    if (prev) {
        // a warp per (human, step, row group), 8 warps per CTA; the kernel
        // reads the live counts and strides over what this grid does not cover
        const long warps = (long)max_rows * t_max * kReachGroups;
        const long ctas = std::min<long>((warps + 7) / 8, (long)sm_count * 64);
        batch_zero_reach_kernel<<<(unsigned)std::max<long>(ctas, 1), 256, 0, s>>>(humans, n_dev, prev, ticket, smax);
        return cudaGetLastError();
    }
    dim3 grid((unsigned)(sm_count * 2), (unsigned)(max_rows < 64 ? max_rows : 64));
    batch_zero_kernel<<<grid, 256, 0, s>>>(humans, n_dev);
    return cudaGetLastError();
}

} // namespace pm
