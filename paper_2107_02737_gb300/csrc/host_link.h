// host_link.h -- where a caller's matrices live (device, page-locked or pageable
// host memory), and moving the symmetric inputs of a host-resident call across
// the host link.  H is the Kohn-Sham matrix in a real basis, hence symmetric
// (Section "The density matrix"), and the output kernel already reads only the
// lower triangles of X_L and H; what crosses the link can therefore be halved.
#pragma once
#include <cuda_runtime.h>

namespace sp2i {

// True when the kernels of this device can use p directly: device memory or
// managed memory.  Host memory (pageable or page-locked) and unknown pointers
// give false.
bool is_device_ptr(const void *p);

// Device address through which the SMs can read and write the page-locked host
// memory at p (mapped into this device's address space), or nullptr when p is
// pageable, device memory, or not mapped.
const void *mapped_host_ptr(const void *p);

// dst (device, n x n, row-major) = the symmetric matrix whose lower triangle,
// diagonal included, is that of src (mapped page-locked host memory, n x n,
// row-major).  Only src's lower triangle is read: n(n+1)/2 values cross the
// link.  The copy is bit-exact; for a bit-symmetric src, dst == src.
cudaError_t launch_stage_lower(const double *src, double *dst, int n, cudaStream_t s);

}  // namespace sp2i
