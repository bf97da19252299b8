// noalloc.cu -- sp2_density for callers that must not allocate device memory.
//
// Some callers cannot call cudaMalloc once they are running: an MD engine whose
// device memory is already reserved by its own pool or by another framework's
// caching allocator (a fresh allocation can fail or fragment that pool), or a
// time-critical step loop that cannot afford an allocation's latency.  For them
// this file keeps the whole workspace of one solve in a statically allocated
// device array, sized for N <= SP2_NOALLOC_MAX_N, and runs the ordinary
// sp2_density kernels on it.
//
// The array is held by every GPU on which the library's device code has been
// loaded, for the life of the process.  With lazy module loading (the CUDA
// default) that happens at first use on a device -- this entry point's first
// call there -- and not when the library is loaded, so that first call should
// come before the caller reserves the rest of the device's memory.  Host code
// may not use the array's name as a device address: the address is obtained
// once per device with cudaGetSymbolAddress, with that device current.
#include <mutex>

#include <cuda_runtime.h>

#include "host_link.h"
#include "sp2.h"

namespace {

constexpr size_t kScratchBytes = (size_t)6 << 20;  // 6 MiB: the workspace of one N <= 512 solve

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
void *g_scratch_addr[kMaxDevices] = {};

}  // namespace

extern "C" sp2_status sp2_density_noalloc(const double *H, int N, double n_occ, double tol, float *D,
                                          sp2_stats *st, const sp2_opts *o, void *stream) {
    if (N < 1 || N > SP2_NOALLOC_MAX_N) return SP2_ERR_ARG;
    if (!H || !D || !sp2i::is_device_ptr(H) || !sp2i::is_device_ptr(D)) return SP2_ERR_ARG;  // staging host data would allocate
    if (o && o->profile) return SP2_ERR_ARG;                              // timing events are not allowed here
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return SP2_ERR_CUDA;
    void *scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_mutex);
        if (!g_scratch_addr[dev]) {
            // First call on this device: resolve the device address of the array
            // (with this device current).
            // With lazy loading this is where the module (and the array) is
            // loaded on the device, so it can fail for lack of device memory.
            void *p = nullptr;
            const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess || !p) {
                cudaGetLastError();
                return e == cudaErrorMemoryAllocation ? SP2_ERR_NOMEM : SP2_ERR_CUDA;
            }
            g_scratch_addr[dev] = p;
        }
        scratch = g_scratch_addr[dev];
    }
    if (sp2_density_workspace_bytes(N, o) > kScratchBytes) return SP2_ERR_ARG;
    // sp2_density clears every word of its workspace that must start at zero
    // (barrier counter, error word, control blocks) and writes every partial
    // and matrix before reading it, so stale contents of the shared array from
    // an earlier call do not leak into this one.
    return sp2_density(H, N, n_occ, tol, D, st, o, scratch, kScratchBytes, stream);
}
