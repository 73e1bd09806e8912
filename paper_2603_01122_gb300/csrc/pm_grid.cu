// pm_grid.cu -- the grid epilogue after emplacement:
//   * the Gaussian convolution of Sec. III-B, as a blur of each step's
//     normalised occupancy (counts / N) by the truncated, normalised,
//     separable Gaussian (zero padding: mass blurred off the grid is dropped);
//   * the multi-human prediction of Sec. IV-B: every human's blurred window
//     placed at its cell offset on one shared grid, which takes the pointwise
//     maximum over humans.
//
// One CTA produces a 64 x 16 tile of the shared grid at one step. For each
// human whose window (widened by the blur radius R) meets the tile, it stages
// the human's counts over the tile plus an R-cell halo in shared memory
// (coalesced rows, scaled by 1/N), blurs along x into a second buffer, blurs
// along y into registers and folds the result into the running maximum; the
// tile is written once. The work is a stream over the count planes: bound by
// HBM bandwidth (each count read once, plus halo re-reads that L2 absorbs).
#include <cuda_runtime.h>

#include "pm_internal.cuh"

namespace pm {
namespace {

constexpr int kTileX = 64, kTileY = 16, kGridThreads = 256;
constexpr int kCellsPerThread = kTileX * kTileY / kGridThreads; // 4

// Window offset of human h on the shared grid (the rollout's own formula for
// a centred window).
__device__ __forceinline__ void window_offset(const BatchHuman &h, int &ox, int &oy)
{
    if (h.center) {
        const int gcx = __float2int_rd(__fmul_rn(__fsub_rn(h.z0[0], h.gx0), h.inv_res));
        const int gcy = __float2int_rd(__fmul_rn(__fsub_rn(h.z0[1], h.gy0), h.inv_res));
        ox = gcx - (h.W - 1) / 2;
        oy = gcy - (h.H - 1) / 2;
    } else {
        ox = h.cx_off;
        oy = h.cy_off;
    }
}

__global__ void __launch_bounds__(kGridThreads) smooth_union_kernel(const __grid_constant__ SmoothArgs a)
{
    __shared__ float A[kTileY + 2 * kMaxSmoothR][kTileX + 2 * kMaxSmoothR];
    __shared__ float Bx[kTileY + 2 * kMaxSmoothR][kTileX];
    const int tid = threadIdx.x;
    const int R = a.R;
    if (R < 0 || R > kMaxSmoothR) return; // the host validates R; never index past the tiles
    const int X0 = blockIdx.x * kTileX, Y0 = blockIdx.y * kTileY, t = blockIdx.z;
    const int AW = kTileX + 2 * R, AH = kTileY + 2 * R;
    float acc[kCellsPerThread];
#pragma unroll
    for (int q = 0; q < kCellsPerThread; ++q) acc[q] = 0.0f;

    const int n = a.humans ? *a.n_humans : 1;
    for (int hi = 0; hi < n; ++hi) {
        const uint32_t *counts;
        float inv_n;
        int Th, Wh, Hh, ox, oy;
        if (a.humans) {
            const BatchHuman &h = a.humans[hi];
            counts = h.counts;
            inv_n = 1.0f / (float)h.N;
            Th = h.T;
            Wh = h.W;
            Hh = h.H;
            window_offset(h, ox, oy);
        } else {
            counts = a.single.counts;
            inv_n = a.single.inv_n;
            Th = a.single.T;
            Wh = a.single.W;
            Hh = a.single.H;
            ox = a.single.ox;
            oy = a.single.oy;
        }
        // the human reaches this tile only if its widened window meets it
        if (t >= Th || ox - R >= X0 + kTileX || ox + Wh + R <= X0 || oy - R >= Y0 + kTileY || oy + Hh + R <= Y0)
            continue;
        const uint32_t *plane = counts + (size_t)t * Wh * Hh;
        for (int e = tid; e < AW * AH; e += kGridThreads) {
            const int ry = e / AW, rx = e - ry * AW;
            const int wx = X0 - R + rx - ox, wy = Y0 - R + ry - oy; // window cell
            float v = 0.0f;
            if (wx >= 0 && wx < Wh && wy >= 0 && wy < Hh) v = (float)plane[(size_t)wy * Wh + wx] * inv_n;
            A[ry][rx] = v;
        }
        __syncthreads();
        if (R == 0) {
#pragma unroll
            for (int q = 0; q < kCellsPerThread; ++q) {
                const int c = tid + q * kGridThreads, y = c / kTileX, x = c - y * kTileX;
                acc[q] = fmaxf(acc[q], A[y][x]);
            }
        } else {
            for (int e = tid; e < AH * kTileX; e += kGridThreads) {
                const int y = e / kTileX, x = e - y * kTileX;
                float s = 0.0f;
                for (int k = 0; k <= 2 * R; ++k) s = fmaf(a.w[k], A[y][x + k], s);
                Bx[y][x] = s;
            }
            __syncthreads();
#pragma unroll
            for (int q = 0; q < kCellsPerThread; ++q) {
                const int c = tid + q * kGridThreads, y = c / kTileX, x = c - y * kTileX;
                float s = 0.0f;
                for (int k = 0; k <= 2 * R; ++k) s = fmaf(a.w[k], Bx[y + k][x], s);
                acc[q] = fmaxf(acc[q], s);
            }
        }
        __syncthreads(); // A and Bx are refilled for the next human
    }
#pragma unroll
    for (int q = 0; q < kCellsPerThread; ++q) {
        const int c = tid + q * kGridThreads, y = c / kTileX, x = c - y * kTileX;
        const int X = X0 + x, Y = Y0 + y;
        if (X < a.W && Y < a.H) a.out[((size_t)t * a.H + Y) * a.W + X] = acc[q];
    }
}

} // namespace

cudaError_t launch_smooth_union(const SmoothArgs &a, cudaStream_t s)
{
    if (a.T <= 0 || a.W <= 0 || a.H <= 0) return cudaSuccess;
    const dim3 grid((a.W + kTileX - 1) / kTileX, (a.H + kTileY - 1) / kTileY, a.T);
    smooth_union_kernel<<<grid, kGridThreads, 0, s>>>(a);
    return cudaGetLastError();
}

} // namespace pm
