// pm_misc.cu -- raw Philox blocks (for the bit-exact generator check) and the
// special-function-unit throughput probe used as the roofline denominator.
#include <cuda_runtime.h>

#include "pm_kernels.cuh"

namespace pm {
namespace {

__global__ void philox_blocks_kernel(uint64_t seed, uint32_t human, uint32_t purpose,
                                     uint64_t particle0, uint64_t block, int n, uint64_t *out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const U64x4 r = philox4x64_10(U64x4{particle0 + (uint64_t)i, block, (uint64_t)purpose, 0ull},
                                  seed, (uint64_t)human);
    out[4 * (size_t)i + 0] = r.a;
    out[4 * (size_t)i + 1] = r.b;
    out[4 * (size_t)i + 2] = r.c;
    out[4 * (size_t)i + 3] = r.d;
}

// Eight independent dependency chains per thread of one operation: the SFU
// (0 ex2, 1 sqrt, 2 rsqrt), the FP32 pipe (3 scalar FMA, 4 packed FMA on
// pairs) or the integer pipe (5 add; chains in dependent pairs).
template <int OP>
__global__ void sfu_probe_kernel(int iters, float *sink)
{
    float v[8];
    f32x2 p[8];
    uint32_t u[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        v[c] = 0.5f + 0.01f * (float)(threadIdx.x & 7) + 0.001f * (float)c;
        p[c] = f2_pack(v[c], v[c] + 0.25f);
        u[c] = threadIdx.x * 8u + (uint32_t)c;
    }
    const f32x2 M = f2_pack(0.999f, 0.998f), A = f2_pack(0.001f, 0.002f);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            if (OP == 0) v[c] = ex2_approx(-v[c]);
            else if (OP == 1) v[c] = sqrt_approx(v[c]);
            else if (OP == 2) v[c] = rsqrt_approx(v[c]);
            else if (OP == 3) v[c] = fmaf(v[c], 0.999f, 0.001f);
            else if (OP == 4) p[c] = f2_fma(p[c], M, A);
            else u[c] += u[c ^ 1]; // four chains of dependent pairs (no closed form)
        }
    }
    float s = 0.0f;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        float lo, hi;
        f2_unpack(p[c], lo, hi);
        s += v[c] + lo + hi + (float)u[c];
    }
    sink[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

} // namespace

cudaError_t launch_philox_blocks(uint64_t seed, uint32_t human, uint32_t purpose, uint64_t particle0,
                                 uint64_t block, int n, uint64_t *out, cudaStream_t s)
{
    philox_blocks_kernel<<<(n + 255) / 256, 256, 0, s>>>(seed, human, purpose, particle0, block, n, out);
    return cudaGetLastError();
}

cudaError_t launch_sfu_probe(int op, int blocks, int threads, int iters, float *sink, cudaStream_t s)
{
    switch (op) {
    case 0: sfu_probe_kernel<0><<<blocks, threads, 0, s>>>(iters, sink); break;
    case 1: sfu_probe_kernel<1><<<blocks, threads, 0, s>>>(iters, sink); break;
    case 2: sfu_probe_kernel<2><<<blocks, threads, 0, s>>>(iters, sink); break;
    case 3: sfu_probe_kernel<3><<<blocks, threads, 0, s>>>(iters, sink); break;
    case 4: sfu_probe_kernel<4><<<blocks, threads, 0, s>>>(iters, sink); break;
    default: sfu_probe_kernel<5><<<blocks, threads, 0, s>>>(iters, sink); break;
    }
    return cudaGetLastError();
}

} // namespace pm
