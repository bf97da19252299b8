// fp64_ext.cu -- the steps on either side of the chain that need FP64 matrices:
//
//  * refinement: a few further layers of the same network with X held in FP64
//    (section "Deep-neural network electronic structure solver", the refinement
//    step that purifies the eigenvalues closer to 0 and 1), each sign taken on
//    the device by the trace rule;
//  * the non-orthogonal route of section "The density matrix":
//    H_orth = Z^T H Z, D_orth = theta(mu I - H_orth), D = Z D_orth Z^T.
//
// The matrix products here are plain dense FP64 GEMMs and run in cuBLAS with
// FP64 emulated on the tensor cores (CUBLAS_COMPUTE_64F_EMULATED_FIXEDPOINT);
// everything else (conversions, FP64 traces, the sign decision, the layer
// update, Tr[DH]) is in the kernels below.
#include <cublas_v2.h>

#include <mutex>
#include <vector>

#include "device_common.cuh"
#include "host_link.h"

namespace {

using namespace sp2i;

constexpr int T64 = 256;
constexpr int RED_BLOCKS = 512;

__device__ __forceinline__ double warp_sum64(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// Block sums of two doubles in a fixed order; valid in thread 0.
__device__ __forceinline__ double2 block_sum2_64(double a, double b) {
    __shared__ double sa[T64 / 32], sb[T64 / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    a = warp_sum64(a);
    b = warp_sum64(b);
    if (lane == 0) {
        sa[w] = a;
        sb[w] = b;
    }
    __syncthreads();
    double2 r = make_double2(0.0, 0.0);
    if (threadIdx.x == 0)
        for (int k = 0; k < T64 / 32; ++k) {
            r.x += sa[k];
            r.y += sb[k];
        }
    __syncthreads();
    return r;
}

__global__ void k_f32_to_f64(const float *__restrict__ src, double *__restrict__ dst, size_t count) {
    for (size_t i = (size_t)blockIdx.x * T64 + threadIdx.x; i < count; i += (size_t)gridDim.x * T64)
        dst[i] = (double)src[i];
}

__global__ void k_f64_to_f32(const double *__restrict__ src, float *__restrict__ dst, size_t count) {
    for (size_t i = (size_t)blockIdx.x * T64 + threadIdx.x; i < count; i += (size_t)gridDim.x * T64)
        dst[i] = (float)src[i];
}

// Per-block FP64 partials of (Tr X, ||X||_F^2) for an n x n row-major X.
__global__ void __launch_bounds__(T64) k_stats64(const double *__restrict__ X, int n, double2 *part) {
    double t = 0.0, q = 0.0;
    for (int i = blockIdx.x; i < n; i += gridDim.x) {
        const double *row = X + (size_t)i * n;
        for (int j = threadIdx.x; j < n; j += T64) {
            const double x = row[j];
            q += x * x;
            if (i == j) t += x;
        }
    }
    const double2 s = block_sum2_64(t, q);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// One thread: sum the partials, record (Tr, ||.||^2, Tr - ||.||^2) of the current X in
// rec[0..2], and pick the next sign by the trace rule.
__global__ void k_decide64(const double2 *part, int nblocks, double n_occ, int *choice, double *rec) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double t = 0.0, q = 0.0;
    for (int k = 0; k < nblocks; ++k) {
        t += part[k].x;
        q += part[k].y;
    }
    rec[0] = t;
    rec[1] = q;
    rec[2] = t - q;
    rec[3] = 0.0;
    *choice = layer_rule(t, q, n_occ);
}

// X <- S (X^2 layer) or 2X - S (2X - X^2 layer), the sign read from the device.
__global__ void k_update64(double *__restrict__ X, const double *__restrict__ S, size_t count, const int *choice) {
    const bool flip = (*choice == SP2_CHOICE_FLIP);
    for (size_t i = (size_t)blockIdx.x * T64 + threadIdx.x; i < count; i += (size_t)gridDim.x * T64)
        X[i] = flip ? 2.0 * X[i] - S[i] : S[i];
}

// Per-block partials of Tr[D H] (symmetric: upper triangle, weight 2) and Tr D.
__global__ void __launch_bounds__(T64) k_energy64(const double *__restrict__ D, const double *__restrict__ H, int n,
                                                  double2 *part) {
    double e = 0.0, t = 0.0;
    for (int i = blockIdx.x; i < n; i += gridDim.x) {
        const size_t b = (size_t)i * n;
        for (int j = i + threadIdx.x; j < n; j += T64) {
            const double d = D[b + j];
            e += (j == i ? 1.0 : 2.0) * d * H[b + j];
            if (j == i) t += d;
        }
    }
    const double2 s = block_sum2_64(e, t);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}

__global__ void k_sum_parts(const double2 *part, int nblocks, double *out) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double a = 0.0, b = 0.0;
    for (int k = 0; k < nblocks; ++k) {
        a += part[k].x;
        b += part[k].y;
    }
    out[0] = a;
    out[1] = b;
}

// Symmetrise in place: X <- (X + X^T)/2 (the FP64 GEMM result of a symmetric
// product is symmetric only up to rounding).
__global__ void k_symmetrise64(double *X, int n) {
    for (int i = blockIdx.x; i < n; i += gridDim.x)
        for (int j = i + 1 + threadIdx.x; j < n; j += T64) {
            const double v = 0.5 * (X[(size_t)i * n + j] + X[(size_t)j * n + i]);
            X[(size_t)i * n + j] = v;
            X[(size_t)j * n + i] = v;
        }
}

int grid_for(size_t work) {
    size_t g = (work + T64 - 1) / T64;
    if (g > 4096) g = 4096;
    return g < 1 ? 1 : (int)g;
}

// cuBLAS handle per device, created once; calls through it are serialised.
struct Blas {
    cublasHandle_t h = nullptr;
    std::mutex mu;
};
Blas g_blas[64];

// Row-major C = op(A) op(B) for n x n FP64 matrices, FP64 emulated on the tensor cores.
cublasStatus_t rm_gemm(cublasHandle_t h, int n, bool ta, const double *A, bool tb, const double *B, double *C) {
    const double one = 1.0, zero = 0.0;
    // Column-major view of row-major memory is the transpose: C^T = op(B)^T op(A)^T.
    return cublasGemmEx(h, tb ? CUBLAS_OP_T : CUBLAS_OP_N, ta ? CUBLAS_OP_T : CUBLAS_OP_N, n, n, n, &one, B, CUDA_R_64F,
                        n, A, CUDA_R_64F, n, &zero, C, CUDA_R_64F, n, CUBLAS_COMPUTE_64F_EMULATED_FIXEDPOINT,
                        CUBLAS_GEMM_DEFAULT);
}

struct DevBuf {
    std::vector<void *> p;
    cudaStream_t s;
    explicit DevBuf(cudaStream_t st) : s(st) {}
    void *get(size_t bytes) {
        void *q = nullptr;
        if (cudaMallocAsync(&q, bytes ? bytes : 256, s) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        p.push_back(q);
        return q;
    }
    ~DevBuf() {
        for (void *q : p) cudaFreeAsync(q, s);
        cudaStreamSynchronize(s);
    }
};

#define CKS(x)                                 \
    do {                                       \
        cudaError_t e_ = (x);                  \
        if (e_ != cudaSuccess) {               \
            cudaGetLastError();                \
            return SP2_ERR_CUDA;               \
        }                                      \
    } while (0)
#define CKB(x)                                        \
    do {                                              \
        if ((x) != CUBLAS_STATUS_SUCCESS) return SP2_ERR_CUDA; \
    } while (0)

// The shared driver: optional congruence by Z, the split-precision chain through
// sp2_density, FP64 refinement layers, optional back-transformation, FP64 output.
sp2_status run_fp64(const double *H_in, const double *Z_in, int N, double n_occ, double tol, int refine_layers,
                    double *D_out, sp2_stats *st, const sp2_opts *o, void *stream) {
    if (N < 1 || N > 65536 || !H_in || !D_out || refine_layers < 0 || refine_layers > 8) return SP2_ERR_ARG;
    if (!(n_occ >= 0.0 && n_occ <= N && n_occ == (double)(long long)n_occ)) return SP2_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0;
    CKS(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return SP2_ERR_CUDA;
    const size_t nn = (size_t)N * N;
    DevBuf buf(s);
    // Inputs on the device: page-locked H from its lower triangle (as every entry
    // point reads it), pageable H and any Z (not symmetric) copied whole.
    const double *H = H_in;
    if (!is_device_ptr(H_in)) {
        double *t = (double *)buf.get(nn * 8);
        if (!t) return SP2_ERR_NOMEM;
        if (const void *m = mapped_host_ptr(H_in)) CKS(launch_stage_lower((const double *)m, t, N, s));
        else CKS(cudaMemcpyAsync(t, H_in, nn * 8, cudaMemcpyHostToDevice, s));
        H = t;
    }
    const double *Z = Z_in;
    if (Z_in && !is_device_ptr(Z_in)) {
        double *t = (double *)buf.get(nn * 8);
        if (!t) return SP2_ERR_NOMEM;
        CKS(cudaMemcpyAsync(t, Z_in, nn * 8, cudaMemcpyHostToDevice, s));
        Z = t;
    }
    double *X64 = (double *)buf.get(nn * 8);
    double *S64 = (double *)buf.get(nn * 8);
    float *D32 = (float *)buf.get(nn * 4);
    double2 *part = (double2 *)buf.get(sizeof(double2) * RED_BLOCKS);
    int *d_choice = (int *)buf.get(64);
    double *d_rec = (double *)buf.get(sizeof(double) * 4 * 16 + 64);
    if (!X64 || !S64 || !D32 || !part || !d_choice || !d_rec) return SP2_ERR_NOMEM;

    Blas &bl = g_blas[dev];
    std::lock_guard<std::mutex> lock(bl.mu);
    if (!bl.h) {
        if (cublasCreate(&bl.h) != CUBLAS_STATUS_SUCCESS) {
            bl.h = nullptr;
            return SP2_ERR_UNSUPPORTED;
        }
    }
    CKB(cublasSetStream(bl.h, s));
    CKB(cublasSetEmulationStrategy(bl.h, CUBLAS_EMULATION_STRATEGY_EAGER));

    // H_orth = Z^T H Z (symmetrised); the chain runs on it.
    const double *Hc = H;
    if (Z) {
        CKB(rm_gemm(bl.h, N, false, H, false, Z, S64));   // S64 = H Z
        CKB(rm_gemm(bl.h, N, true, Z, false, S64, X64));  // X64 = Z^T (H Z)
        k_symmetrise64<<<grid_for(N), T64, 0, s>>>(X64, N);
        CKS(cudaGetLastError());
        Hc = X64;
    }
    sp2_stats local;
    memset(&local, 0, sizeof(local));
    std::vector<sp2_layer_stat> lay(SP2_MAX_LAYERS_LIMIT + 16);
    local.layer = lay.data();
    local.layer_cap = (int)lay.size();
    sp2_status r = sp2_density(Hc, N, n_occ, tol, D32, &local, o, nullptr, 0, s);
    if (r != SP2_OK && r != SP2_ERR_NOT_CONVERGED) return r;
    const sp2_status chain_status = r;

    // Refinement layers in FP64 (X64 now holds D_orth).
    k_f32_to_f64<<<grid_for(nn), T64, 0, s>>>(D32, X64, nn);
    CKS(cudaGetLastError());
    const int rb = N < RED_BLOCKS ? N : RED_BLOCKS;
    for (int l = 0; l <= refine_layers; ++l) {
        k_stats64<<<rb, T64, 0, s>>>(X64, N, part);
        k_decide64<<<1, 32, 0, s>>>(part, rb, n_occ, d_choice, d_rec + 4 * l);
        CKS(cudaGetLastError());
        if (l == refine_layers) break;
        CKB(rm_gemm(bl.h, N, false, X64, false, X64, S64));  // S = X^2
        k_update64<<<grid_for(nn), T64, 0, s>>>(X64, S64, nn, d_choice);
        k_symmetrise64<<<grid_for(N), T64, 0, s>>>(X64, N);
        CKS(cudaGetLastError());
    }
    // Back-transformation D = Z D_orth Z^T.
    double *Dfin = X64;
    if (Z) {
        CKB(rm_gemm(bl.h, N, false, X64, true, Z, S64));  // S64 = D_orth Z^T
        CKB(rm_gemm(bl.h, N, false, Z, false, S64, X64)); // X64 = Z (D_orth Z^T)
        k_symmetrise64<<<grid_for(N), T64, 0, s>>>(X64, N);
        CKS(cudaGetLastError());
    }
    // FP64 Tr[D H] (original H) and Tr D.
    k_energy64<<<rb, T64, 0, s>>>(Dfin, H, N, part);
    k_sum_parts<<<1, 32, 0, s>>>(part, rb, d_rec + 4 * (refine_layers + 1));
    CKS(cudaGetLastError());
    if (is_device_ptr(D_out)) CKS(cudaMemcpyAsync(D_out, Dfin, nn * 8, cudaMemcpyDeviceToDevice, s));
    else CKS(cudaMemcpyAsync(D_out, Dfin, nn * 8, cudaMemcpyDeviceToHost, s));
    std::vector<double> rec(4 * (refine_layers + 2));
    CKS(cudaMemcpyAsync(rec.data(), d_rec, sizeof(double) * rec.size(), cudaMemcpyDeviceToHost, s));
    CKS(cudaStreamSynchronize(s));

    if (st) {
        sp2_layer_stat *user_layers = st->layer;
        const int cap = st->layer_cap;
        *st = local;
        st->layer = user_layers;
        st->layer_cap = cap;
        const int L = local.layers;
        // The chain's layers, then the refinement layers (the sign of layer l is
        // the decision taken on the statistics of layer l - 1).
        int k = 0;
        for (; k <= L && k < cap; ++k) st->layer[k] = lay[k];
        for (int l = 1; l <= refine_layers && L + l < cap; ++l) {
            sp2_layer_stat ls;
            ls.trace = rec[4 * l + 0];
            ls.trace_sq = rec[4 * l + 1];
            ls.idem = rec[4 * l + 2];
            ls.choice = layer_rule(rec[4 * (l - 1) + 0], rec[4 * (l - 1) + 1], n_occ);
            ls.reserved = 0;
            ls.alpha = 1.0;
            st->layer[L + l] = ls;
        }
        st->layers = L + refine_layers;
        st->band_energy = rec[4 * (refine_layers + 1) + 0];
        st->trace_D = rec[4 * (refine_layers + 1) + 1];
    }
    return chain_status;
}

}  // namespace

extern "C" sp2_status sp2_density_refined(const double *H, int N, double n_occ, double tol, int refine_layers,
                                          double *D, sp2_stats *st, const sp2_opts *o, void *stream) {
    return run_fp64(H, nullptr, N, n_occ, tol, refine_layers, D, st, o, stream);
}

extern "C" sp2_status sp2_density_nonorth(const double *H, const double *Z, int N, double n_occ, double tol,
                                          int refine_layers, double *D, sp2_stats *st, const sp2_opts *o,
                                          void *stream) {
    if (!Z) return SP2_ERR_ARG;
    return run_fp64(H, Z, N, n_occ, tol, refine_layers, D, st, o, stream);
}
