// pm_misc.cu -- raw Philox blocks (for the bit-exact generator check) and the
// special-function-unit throughput probe used as the roofline denominator.
#include <cuda_runtime.h>

#include "pm_internal.cuh"

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

// Eight independent dependency chains per thread of one SFU operation.
template <int OP>
__global__ void sfu_probe_kernel(int iters, float *sink)
{
    float v[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) v[c] = 0.5f + 0.01f * (float)(threadIdx.x & 7) + 0.001f * (float)c;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            if (OP == 0) v[c] = ex2_approx(-v[c]);
            else if (OP == 1) v[c] = sqrt_approx(v[c]);
            else v[c] = rsqrt_approx(v[c]);
        }
    }
    float s = 0.0f;
#pragma unroll
    for (int c = 0; c < 8; ++c) s += v[c];
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
    if (op == 0) sfu_probe_kernel<0><<<blocks, threads, 0, s>>>(iters, sink);
    else if (op == 1) sfu_probe_kernel<1><<<blocks, threads, 0, s>>>(iters, sink);
    else sfu_probe_kernel<2><<<blocks, threads, 0, s>>>(iters, sink);
    return cudaGetLastError();
}

} // namespace pm
