// pm_grid.cu -- the grid epilogue after emplacement:
//   * the Gaussian convolution of Sec. III-B, as a blur of each step's
//     normalised occupancy (counts / N) by the truncated, normalised,
//     separable Gaussian (zero padding: mass blurred off the grid is dropped);
//   * the multi-human prediction of Sec. IV-B: every human's blurred window
//     placed at its cell offset on one shared grid, which takes the pointwise
//     maximum over humans.
//
// A first kernel reduces each human of a batch to a compact source record
// (counts, 1/N, horizon, window size and cell offset; a centred window's
// offset from the human's start cell, by the rollout's own formula). The
// union kernel then produces a 64 x 32 tile of the shared grid at one step
// per CTA: it loads the source records into shared memory, and for the
// sources whose window (widened by the blur radius R) meets the tile it
// stages the counts of the tile plus an R-cell halo in shared memory, two
// sources at a time (coalesced rows; both sources' loads in flight before
// either is stored), blurs along x into a third buffer with each thread
// sliding a register window over four outputs, blurs along y the same way,
// and folds the result into the running maximum; the tile is written once.
// The work streams over the count planes: HBM-bound when the windows cover
// the grid, shared-memory-bound for small windows. A region with no particle
// adds nothing (the blur of zeros is zero and the running maximum is >= 0):
// the batched rollout marks the 16 x 16-cell blocks it emplaces into, the
// union reads every source's marks for its tile in one pass and stages only
// the sources with a particle nearby, and a staged region that turns out
// empty skips both blur passes. The HBM traffic follows the occupied blocks.
#include <utility>

#include <cuda_runtime.h>

#include "pm_kernels.cuh"

namespace pm {
namespace {

constexpr int kTileX = 64, kTileY = 32, kGridThreads = 256;
constexpr int kRowsPerThread = kTileX * kTileY / kGridThreads; // 8 (vertical pass)
constexpr int kSrcChunk = 128; // source records staged in shared memory at a time

__global__ void union_sources_kernel(const BatchHuman *humans, const int *n_humans, SmoothSrc *srcs)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= *n_humans) return;
    const BatchHuman h = humans[i];
    SmoothSrc s;
    s.counts = h.counts;
    s.inv_n = 1.0f / (float)h.N;
    s.small = h.N < (1 << 23);
    s.T = h.T;
    s.W = h.W;
    s.H = h.H;
    s.flags = h.flags;
    s.fbx = h.fbx;
    s.fby = h.fby;
    if (h.center) {
        s.ox = __float2int_rd(__fmul_rn(__fsub_rn(h.z0[0], h.gx0), h.inv_res)) - (h.W - 1) / 2;
        s.oy = __float2int_rd(__fmul_rn(__fsub_rn(h.z0[1], h.gy0), h.inv_res)) - (h.H - 1) / 2;
    } else {
        s.ox = h.cx_off;
        s.oy = h.cy_off;
    }
    srcs[i] = s;
}

// Shared-memory layout of smooth_union_kernel<RB> (dynamic: the two staging
// buffers exceed the 48 KiB of static shared memory at larger R).
template <int RB>
struct UnionSmem {
    static constexpr int AW = kTileX + 2 * RB, AH = kTileY + 2 * RB;
    static constexpr int NW = 2 * RB + 4; // window of four outputs
    // row stride: a multiple of 4 floats (16-byte vector loads) covering the
    // last vector load of the widest window, columns up to 60 + 4 ceil(NW/4) - 1
    static constexpr int AS = 60 + 4 * ((NW + 3) / 4);
    static_assert(AS >= AW && AS % 4 == 0, "row stride");
    float A[2][AH][AS];     // counts of two sources' widened tiles
    float Bx[AH][kTileX];   // after the horizontal pass
    SmoothSrc S[kSrcChunk]; // source records
    unsigned live[kSrcChunk / 32];
    int list[kSrcChunk];    // the live sources, in order
    int n_live;
    int4 cand[kSrcChunk];   // sources whose widened window meets the tile: (index, bx0, by0, nbx | nby << 16)
    int n_cand;
};

template <int RB>
size_t union_smem_bytes() { return sizeof(UnionSmem<RB>); }

// RB: the blur radius R as a compile-time constant, so that the sliding
// windows of both passes live in registers and every tap is one FMA. Up to
// R = 8 the kernel fits 80 registers without spills and runs 3 CTAs per SM;
// larger R keeps 2 CTAs (128 registers, no spills).
//
// The live sources of a tile are staged two at a time: the loads of both
// regions are issued before either is stored, so a tile with several
// occupied sources pays one load latency per pair.
template <int RB>
__global__ void __launch_bounds__(kGridThreads, (RB >= 1 && RB <= 8) ? 3 : 2)
    smooth_union_kernel(const __grid_constant__ SmoothArgs a)
{
    using L = UnionSmem<RB>;
    constexpr int AW = L::AW, AH = L::AH, NW = L::NW;
    extern __shared__ __align__(16) unsigned char union_smem_raw[];
    L &sm = *reinterpret_cast<L *>(union_smem_raw);
    // flag blocks that can meet the widened tile, per source
    constexpr int BX = (AW + kFlagBlock - 1) / kFlagBlock + 1, BY = (AH + kFlagBlock - 1) / kFlagBlock + 1;
    const int tid = threadIdx.x;
    const int X0 = blockIdx.x * kTileX, Y0 = blockIdx.y * kTileY, t = blockIdx.z;
    // horizontal pass: thread -> (row hy0 + 16 j, columns 4 hx .. 4 hx + 3)
    const int hx = tid & 15, hy0 = tid >> 4;
    // vertical pass and output: thread -> (column vx, rows 8 vg .. 8 vg + 7)
    const int vx = tid & 63, vg = tid >> 6;
    constexpr int RT = kRowsPerThread, NV = 2 * RB + RT;
    constexpr int kStageIters = (AW * AH + kGridThreads - 1) / kGridThreads;
    float w[2 * RB + 1];
#pragma unroll
    for (int k = 0; k <= 2 * RB; ++k) w[k] = a.w[k];
    float acc[RT];
#pragma unroll
    for (int j = 0; j < RT; ++j) acc[j] = 0.0f;

    // this thread's elements e = tid + i * kGridThreads of a source's widened tile
    auto load = [&](const SmoothSrc &s, uint32_t (&c)[kStageIters]) {
        const uint32_t *plane = s.counts + (size_t)t * s.W * s.H;
        const int wx0 = X0 - RB - s.ox, wy0 = Y0 - RB - s.oy; // window cell of A[.][0][0]
#pragma unroll
        for (int i = 0; i < kStageIters; ++i) {
            const int e = tid + i * kGridThreads;
            const int ry = e / AW, rx = e - ry * AW;
            const int wy = wy0 + ry, wx = wx0 + rx;
            const bool in = e < AW * AH && wy >= 0 && wy < s.H && wx >= 0 && wx < s.W;
            c[i] = in ? plane[(size_t)wy * s.W + wx] : 0u;
        }
    };
    // counts stay raw until here (exact in FP32 below 2^23, converted on the
    // FP32 pipe); the 1/N scale is applied once per output at the end
    auto store = [&](const uint32_t (&c)[kStageIters], float (*A)[L::AS]) {
        uint32_t nz = 0u;
#pragma unroll
        for (int i = 0; i < kStageIters; ++i) {
            const int e = tid + i * kGridThreads;
            const int ry = e / AW, rx = e - ry * AW;
            nz |= c[i];
            if (e < AW * AH)
                A[ry][rx] = c[i] < 0x800000u ? __int_as_float((int)(c[i] | 0x4B000000u)) - 8388608.0f : (float)c[i];
        }
        return nz;
    };
    auto blur = [&](float (*A)[L::AS], float inv_n) {
        if constexpr (RB == 0) {
#pragma unroll
            for (int j = 0; j < RT; ++j) acc[j] = fmaxf(acc[j], A[RT * vg + j][vx] * inv_n);
        } else {
            for (int y = hy0; y < AH; y += kGridThreads / 16) {
                float v[NW];
#pragma unroll
                for (int k = 0; k < NW; k += 4) {
                    // 16-byte load; the last one may read the row's padding (never used)
                    const float4 q = *reinterpret_cast<const float4 *>(&A[y][4 * hx + k]);
                    v[k] = q.x;
                    if (k + 1 < NW) v[k + 1] = q.y;
                    if (k + 2 < NW) v[k + 2] = q.z;
                    if (k + 3 < NW) v[k + 3] = q.w;
                }
                float o[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
                for (int j = 0; j < 4; ++j)
#pragma unroll
                    for (int k = 0; k <= 2 * RB; ++k) o[j] = fmaf(w[k], v[j + k], o[j]);
                *reinterpret_cast<float4 *>(&sm.Bx[y][4 * hx]) = make_float4(o[0], o[1], o[2], o[3]);
            }
            __syncthreads();
            float v[NV];
#pragma unroll
            for (int k = 0; k < NV; ++k) v[k] = sm.Bx[RT * vg + k][vx];
#pragma unroll
            for (int j = 0; j < RT; ++j) {
                float o = 0.0f;
#pragma unroll
                for (int k = 0; k <= 2 * RB; ++k) o = fmaf(w[k], v[j + k], o);
                acc[j] = fmaxf(acc[j], o * inv_n);
            }
            __syncthreads(); // Bx is refilled by the next blur
        }
    };

    const int n = a.srcs ? *a.n_srcs : 1;
    for (int c0 = 0; c0 < n; c0 += kSrcChunk) {
        const int nc = min(kSrcChunk, n - c0);
        __syncthreads(); // the previous chunk's records and buffers are no longer read
        if (tid < kSrcChunk / 32) sm.live[tid] = 0u;
        if (tid == 0) sm.n_cand = 0;
        __syncthreads();
        // Which sources reach the tile: the widened window must meet it (one
        // thread per source), and where the source carries block flags one of
        // the blocks under the widened tile must hold a particle at step t.
        // All candidates' flags are read in one pass, so a tile costs one
        // round trip, not one per source.
        if (tid < nc) {
            const SmoothSrc q = a.srcs ? a.srcs[c0 + tid] : a.single;
            sm.S[tid] = q;
            const int wx0 = X0 - RB - q.ox, wy0 = Y0 - RB - q.oy;
            const int xlo = max(wx0, 0), xhi = min(wx0 + AW, q.W), ylo = max(wy0, 0), yhi = min(wy0 + AH, q.H);
            if (t < q.T && xlo < xhi && ylo < yhi) {
                const int bx0 = xlo >> kFlagShift, by0 = ylo >> kFlagShift;
                const int nbx = ((xhi - 1) >> kFlagShift) - bx0 + 1, nby = ((yhi - 1) >> kFlagShift) - by0 + 1;
                sm.cand[atomicAdd(&sm.n_cand, 1)] = make_int4(tid, bx0, by0, nbx | (nby << 16));
            }
        }
        __syncthreads();
        const int ncand = sm.n_cand;
        for (int p = tid; p < ncand * BX * BY; p += kGridThreads) {
            const int ci = p / (BX * BY), b = p - ci * (BX * BY);
            const int4 cd = sm.cand[ci];
            const SmoothSrc &q = sm.S[cd.x];
            bool hit;
            if (!q.flags) {
                hit = b == 0;
            } else {
                const int bxr = b % BX, byr = b / BX;
                hit = bxr < (cd.w & 0xFFFF) && byr < (cd.w >> 16) &&
                      q.flags[((size_t)t * q.fby + cd.z + byr) * q.fbx + cd.y + bxr] != 0u;
            }
            if (hit) atomicOr(&sm.live[cd.x >> 5], 1u << (cd.x & 31));
        }
        __syncthreads();
        if (tid == 0) { // the live sources in order
            int m = 0;
            for (int wd = 0; wd < (nc + 31) / 32; ++wd)
                for (unsigned bits = sm.live[wd]; bits; bits &= bits - 1u) sm.list[m++] = wd * 32 + __ffs((int)bits) - 1;
            sm.n_live = m;
        }
        __syncthreads();
        const int nl = sm.n_live;
        for (int i = 0; i < nl; i += 2) {
            const bool two = i + 1 < nl;
            const SmoothSrc s0 = sm.S[sm.list[i]];
            const SmoothSrc s1 = sm.S[sm.list[two ? i + 1 : i]];
            uint32_t c[2][kStageIters];
            load(s0, c[0]);
            if (two) load(s1, c[1]); // both sources' loads in flight before any store
            const uint32_t nz0 = store(c[0], sm.A[0]);
            const uint32_t nz1 = two ? store(c[1], sm.A[1]) : 0u;
            // counts and taps are >= 0, so a region without particles blurs to 0
            // and leaves the running maximum (>= 0) unchanged: skip its passes
            const bool b0 = __syncthreads_or(nz0 != 0u), b1 = __syncthreads_or(nz1 != 0u);
            if (b0) blur(sm.A[0], s0.inv_n);
            if (b1) blur(sm.A[1], s1.inv_n);
            __syncthreads(); // the buffers are refilled for the next pair
        }
    }
    const int X = X0 + vx;
#pragma unroll
    for (int j = 0; j < RT; ++j) {
        const int Y = Y0 + RT * vg + j;
        if (X < a.W && Y < a.H) a.out[((size_t)t * a.H + Y) * a.W + X] = acc[j];
    }
}

template <int RB>
void launch_rb(const SmoothArgs &a, dim3 grid, cudaStream_t s)
{
    const size_t bytes = union_smem_bytes<RB>();
    cudaFuncSetAttribute(smooth_union_kernel<RB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    smooth_union_kernel<RB><<<grid, kGridThreads, bytes, s>>>(a);
}

template <int... Rs>
bool dispatch_rb(int R, const SmoothArgs &a, dim3 grid, cudaStream_t s, std::integer_sequence<int, Rs...>)
{
    bool done = false;
    ((R == Rs ? (launch_rb<Rs>(a, grid, s), done = true) : false), ...);
    return done;
}

} // namespace

cudaError_t launch_union_sources(const BatchHuman *humans, const int *n_humans, int max_humans, SmoothSrc *srcs,
                                 cudaStream_t s)
{
    if (max_humans <= 0) return cudaSuccess;
    union_sources_kernel<<<(max_humans + 127) / 128, 128, 0, s>>>(humans, n_humans, srcs);
    return cudaGetLastError();
}

cudaError_t launch_smooth_union(const SmoothArgs &a, cudaStream_t s)
{
    if (a.T <= 0 || a.W <= 0 || a.H <= 0) return cudaSuccess;
    const dim3 grid((a.W + kTileX - 1) / kTileX, (a.H + kTileY - 1) / kTileY, a.T);
    if (!dispatch_rb(a.R, a, grid, s, std::make_integer_sequence<int, kMaxSmoothR + 1>{}))
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

} // namespace pm
