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
constexpr size_t kPartBytes = 5 * kNoAllocChunks * PM_MAX_COMPONENTS * sizeof(float) +
                              PM_MAX_COMPONENTS * sizeof(double);
constexpr size_t kScratchBytes = kTicketBytes + kPartBytes; // 165,888 bytes

// Shared by every call on a device; it keeps the last call's contents.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_addr[kMaxDevices] = {};

// Device address of g_scratch on the current device (the host-side symbol is
// only a stand-in); looked up once per device.
pm_status scratch_address(int device, unsigned char **out)
{
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[device]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
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
    if (scratch_address(device, &base) != PM_OK)
        return pm_internal_error(PM_ECUDA, "pm_update_posterior_noalloc: cudaGetSymbolAddress of the scratch failed");
    unsigned *ticket = reinterpret_cast<unsigned *>(base);
    float *part = reinterpret_cast<float *>(base + kTicketBytes);
    return pm_internal_posterior_on_scratch(model, obs_xy, n_obs, log_belief, part, ticket, kPartBytes,
                                            kNoAllocChunks, stream);
}
