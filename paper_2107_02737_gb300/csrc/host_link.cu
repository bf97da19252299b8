// host_link.cu -- residency of the caller's pointers, and staging a host-resident
// symmetric FP64 matrix from its lower triangle.
//
// A call with host-resident H is bound by the host link: this GB300's link moves
// ~210 GB/s host -> device, with the copy engines or with SM loads alike, so the
// 537 MB of an N = 8192 FP64 H take 2.5 ms against a 26 ms chain.  H is
// symmetric, so only n(n+1)/2 of its entries carry information.  The SMs read
// them directly from page-locked host memory (zero-copy, one 32 x 32 tile of
// the lower triangle per step, rows of 256 bytes) and write each tile and its
// transpose to the device copy, through shared memory so that both writes are
// coalesced rows.
#include "host_link.h"

namespace sp2i {

namespace {

constexpr int LINK_THREADS = 256;     // 32 tile columns x 8 row groups
constexpr int LINK_BLOCKS_PER_SM = 8; // 8.4 KB of shared memory per block

__global__ void __launch_bounds__(LINK_THREADS) k_stage_lower(const double *__restrict__ src,
                                                              double *__restrict__ dst, int n) {
    __shared__ double s[32][33];
    const int tc = threadIdx.x & 31, tr0 = threadIdx.x >> 5;
    const int nt = (n + 31) / 32;
    const long long ntiles = (long long)nt * (nt + 1) / 2;
    for (long long k = blockIdx.x; k < ntiles; k += gridDim.x) {
        // k -> (ti, tj), tj <= ti, row-major over the lower triangle of tiles:
        // an FP32 root corrected to the exact integer.
        int ti = (int)((sqrtf(8.0f * (float)k + 1.0f) - 1.0f) * 0.5f);
        while ((long long)(ti + 1) * (ti + 2) / 2 <= k) ++ti;
        while ((long long)ti * (ti + 1) / 2 > k) --ti;
        const int tj = (int)(k - (long long)ti * (ti + 1) / 2);
        const int i0 = ti * 32, j0 = tj * 32;
        double v[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {  // four loads in flight per thread before any use
            const int r = tr0 + 8 * q, i = i0 + r, j = j0 + tc;
            v[q] = (i < n && j < n && (ti > tj || r >= tc)) ? src[(size_t)i * n + j] : 0.0;
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) s[tr0 + 8 * q][tc] = v[q];
        __syncthreads();
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int r = tr0 + 8 * q;
            int i = i0 + r, j = j0 + tc;
            if (i < n && j < n) dst[(size_t)i * n + j] = (ti > tj || r >= tc) ? s[r][tc] : s[tc][r];
            i = j0 + r;
            j = i0 + tc;
            if (ti > tj && i < n && j < n) dst[(size_t)i * n + j] = s[tc][r];  // the mirror tile (tj, ti)
        }
        __syncthreads();
    }
}

}  // namespace

bool is_device_ptr(const void *p) {
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

const void *mapped_host_ptr(const void *p) {
    if (!p) return nullptr;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

cudaError_t launch_stage_lower(const double *src, double *dst, int n, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const long long nt = (n + 31) / 32, ntiles = nt * (nt + 1) / 2;
    const long long cap = (long long)sms * LINK_BLOCKS_PER_SM;
    const int grid = (int)(ntiles < cap ? ntiles : cap);
    k_stage_lower<<<grid, LINK_THREADS, 0, s>>>(src, dst, n);
    return cudaGetLastError();
}

}  // namespace sp2i
