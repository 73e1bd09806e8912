// pm_noalloc.cu -- the belief update for callers that cannot allocate device
// memory: a real-time control loop that forbids allocation once it runs, code
// enqueued while a stream is being captured into a CUDA graph in a mode that
// rejects cudaMalloc, or an application whose device memory is owned by its
// own pool. Its scratch is this file's static device array instead of the
// context's allocated buffers, so the call allocates nothing and needs no
// context.
#include <cstring>
#include <mutex>

#include <cuda_runtime.h>

#include "pm.h"
#include "pm_kernels.cuh"

pm_status pm_internal_posterior_on_scratch(const pm_model *model, const float *obs_xy, int32_t n_obs,
                                           float *log_belief, float *part, unsigned *ticket, size_t part_bytes,
                                           int max_chunks, void *stream);
pm_status pm_internal_error(pm_status st, const char *msg);

namespace {

constexpr int kNoAllocChunks = 32;              // CTAs of one call at most
constexpr size_t kTicketBytes = 256;            // one zero word, padded
// five FP32 partial sums per (chunk, component), the belief kernel's layout
constexpr size_t kPartBytes = 5 * kNoAllocChunks * PM_MAX_COMPONENTS * sizeof(float);
constexpr size_t kScratchBytes = kTicketBytes + kPartBytes;
static_assert(kScratchBytes == 164096, "the size stated in pm.h");

// Shared by every call on a device; it keeps the last call's contents.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_addr[kMaxDevices] = {};

// Device address of g_scratch on the current device (the host-side symbol is
// only a stand-in). It is looked up again on every call made outside a stream
// capture, so a device reset (which reloads the module at another address)
// leaves no stale pointer behind; inside a capture the address of the last
// lookup on this device is used, since a capture may forbid the lookup (the
// first call on a device loads the module, which allocates).
pm_status scratch_address(int device, cudaStream_t stream, unsigned char **out)
{
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(stream, &cap);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return PM_ECUDA;
    }
    std::lock_guard<std::mutex> lock(g_mu);
    if (cap == cudaStreamCaptureStatusNone || !g_addr[device]) {
        if (cap != cudaStreamCaptureStatusNone) return PM_EINVAL; // first call inside a capture
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return PM_ECUDA;
        }
        g_addr[device] = p;
    }
    *out = static_cast<unsigned char *>(g_addr[device]);
    return PM_OK;
}

} // namespace

extern "C" pm_status pm_update_posterior_noalloc(const pm_model *model, const float *obs_xy, int32_t n_obs,
                                                 float *log_belief, void *stream)
{
    int device = -1;
    cudaError_t e = cudaGetDevice(&device);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return pm_internal_error(PM_ECUDA, "pm_update_posterior_noalloc: cudaGetDevice failed");
    }
    if (device < 0 || device >= kMaxDevices)
        return pm_internal_error(PM_EINVAL, "pm_update_posterior_noalloc: device ordinal beyond 63");
    unsigned char *base = nullptr;
    const pm_status st = scratch_address(device, (cudaStream_t)stream, &base);
    if (st == PM_EINVAL)
        return pm_internal_error(PM_EINVAL, "pm_update_posterior_noalloc: the first call on a device must come "
                                            "before any stream capture");
    if (st != PM_OK)
        return pm_internal_error(PM_ECUDA, "pm_update_posterior_noalloc: cudaGetSymbolAddress of the scratch failed");
    unsigned *ticket = reinterpret_cast<unsigned *>(base);
    float *part = reinterpret_cast<float *>(base + kTicketBytes);
    return pm_internal_posterior_on_scratch(model, obs_xy, n_obs, log_belief, part, ticket, kPartBytes,
                                            kNoAllocChunks, stream);
}
