// fp64_ext.cu -- the steps on either side of the chain that need FP64 matrices:
//
//  * refinement: a few further layers of the same network with X held in
//    double precision (section "Deep-neural network electronic structure
//    solver", the refinement step that purifies the eigenvalues closer to 0
//    and 1), each sign taken on the device by the trace rule;
//  * the non-orthogonal route of section "The density matrix":
//    H_orth = Z^T H Z, D_orth = theta(mu I - H_orth), D = Z D_orth Z^T.
//
// Every matrix product here is an exact-slice product on the FP16 tensor cores
// (exact_kernel.cu): FP64-level accuracy from integer slices whose products are
// summed exactly in FP32 tensor memory.  The refinement layers carry
// Y = X - I/2 in 64-bit fixed point between layers.
#include <cmath>
#include <cstring>
#include <vector>

#include "device_common.cuh"
#include "exact.h"
#include "host_link.h"

namespace {

using namespace sp2i;

constexpr int T64 = 256;
constexpr int RED_BLOCKS = 512;
constexpr int DEFAULT_SLICES = 6;   // 11 + 5 b bits per row, b = 6 up to N = 8192 (about 2^-41 of the row norms)

// Slices per operand row from the options (0 = default), or 0 when out of range.
int slices_of(const sp2_opts &o) {
    if (o.exact_slices == 0) return DEFAULT_SLICES;
    return (o.exact_slices >= 4 && o.exact_slices <= XS_MAX_SLICES) ? o.exact_slices : 0;
}

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

int grid_for(size_t work) {
    size_t g = (work + T64 - 1) / T64;
    if (g > 4096) g = 4096;
    return g < 1 ? 1 : (int)g;
}

// Device allocations of one call, freed on every exit path; with `fail` set
// (sp2_opts.test_hook = 2) every allocation reports failure.
struct DevBuf {
    std::vector<void *> p;
    cudaStream_t s;
    bool fail = false;
    explicit DevBuf(cudaStream_t st) : s(st) {}
    void *get(size_t bytes) {
        if (fail) return nullptr;
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

#define CKS(x)                        \
    do {                              \
        cudaError_t e_ = (x);         \
        if (e_ != cudaSuccess) {      \
            cudaGetLastError();       \
            return SP2_ERR_CUDA;      \
        }                             \
    } while (0)

int sm_count_now() {
    int dev = 0, sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return sm;
}

// Slices of three n x n operands for the congruences, and the intermediate product.
struct CongruenceBufs {
    XsOperand m, z, w;   // slices of M, of Z or Z^T, of the intermediate's transpose
    double *inter = nullptr, *scratch = nullptr;
    long long *pscr = nullptr;   // product scratch of the kernel
};

bool alloc_operand(DevBuf &buf, XsOperand &op, int np, int slices) {
    op.base = (uint16_t *)buf.get((size_t)slices * np * np * 2);
    op.exps = (int *)buf.get((size_t)np * sizeof(int));
    return op.base && op.exps;
}

// out = Z^T M Z (side 0) or Z M Z^T (side 1) for symmetric M; out is exactly symmetric.
//   side 0: W = M Z (A = M, B = Z^T), out = Z^T W (A = Z^T, B = W^T);
//   side 1: V = M Z^T (A = M, B = Z), out = Z V (A = Z, B = V^T).
sp2_status congruence(const double *Z, const double *M, int n, int side, double *out, CongruenceBufs &cb, int *d_err,
                      int pairs, int slices, unsigned long long timeout_ns, cudaStream_t s) {
    const int np = round_up(n, XS_TILE_N);
    const int beta = xs_choose_beta(slices, np);
    CKS(xs_slice_rows(M, false, n, np, slices, beta, cb.m, cb.scratch, d_err, s));
    CKS(xs_slice_rows(Z, side == 0, n, np, slices, beta, cb.z, cb.scratch, d_err, s));
    XsProduct p;
    p.n = n;
    p.np = np;
    p.slices = slices;
    p.beta = beta;
    p.err = d_err;
    p.timeout_ns = timeout_ns;
    p.scratch = cb.pscr;
    p.mode = XS_GEN;
    p.a = cb.m;
    p.b = cb.z;
    p.c = cb.inter;
    CKS(xs_product(p, pairs, s));
    CKS(xs_slice_rows(cb.inter, true, n, np, slices, beta, cb.w, cb.scratch, d_err, s));
    p.mode = XS_GEN_SYM;
    p.a = cb.z;
    p.b = cb.w;
    p.c = out;
    CKS(xs_product(p, pairs, s));
    return SP2_OK;
}

// CUDA events of one call (sp2_opts.profile), destroyed on every exit path.
struct PhaseEvents {
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    bool on = false;
    explicit PhaseEvents(bool want) {
        if (!want) return;
        on = true;
        for (auto &e : ev)
            if (cudaEventCreate(&e) != cudaSuccess) {
                cudaGetLastError();
                on = false;
            }
    }
    void mark(int k, cudaStream_t s) {
        if (on) cudaEventRecord(ev[k], s);
    }
    // [0] congruence + chain, [1] refinement layers, [2] back-transformation + Tr[DH], [3] all.
    void fill(float *ms) {
        if (!on) return;
        const int from[4] = {0, 1, 2, 0}, to[4] = {1, 2, 3, 3};
        for (int k = 0; k < 4; ++k)
            if (cudaEventElapsedTime(&ms[k], ev[from[k]], ev[to[k]]) != cudaSuccess) {
                cudaGetLastError();
                ms[k] = 0.0f;
            }
    }
    ~PhaseEvents() {
        for (auto e : ev)
            if (e) cudaEventDestroy(e);
    }
};

sp2_status read_err(const int *d_err, cudaStream_t s) {
    int h = 0;
    CKS(cudaMemcpyAsync(&h, d_err, sizeof(int), cudaMemcpyDeviceToHost, s));
    CKS(cudaStreamSynchronize(s));
    return (sp2_status)h;
}

// The shared driver: optional congruence by Z, the split-precision chain through
// sp2_density, FP64 refinement layers, optional back-transformation, FP64 output.
sp2_status run_fp64(const double *H_in, const double *Z_in, int N, double n_occ, double tol, int refine_layers,
                    double *D_out, sp2_stats *st, const sp2_opts *o, void *stream) {
    if (N < 1 || N > 65536 || !H_in || !D_out || refine_layers < 0 || refine_layers > 8) return SP2_ERR_ARG;
    if (!(n_occ >= 0.0 && n_occ <= N && n_occ == (double)(long long)n_occ)) return SP2_ERR_ARG;
    sp2_opts opt;
    sp2_default_opts(&opt);
    if (o) opt = *o;
    cudaStream_t s = (cudaStream_t)stream;
    const int slices = slices_of(opt);
    if (!slices) return SP2_ERR_ARG;
    if (!xs_available()) return SP2_ERR_UNSUPPORTED;
    const int sm = sm_count_now();
    const int pairs = xs_resident_pairs(sm);
    if (pairs < 1) return SP2_ERR_UNSUPPORTED;
    const unsigned long long timeout_ns = (unsigned long long)(opt.timeout_ms * 1e6);
    const size_t nn = (size_t)N * N;
    const int np = round_up(N, XS_TILE_N);
    DevBuf buf(s);
    buf.fail = (opt.test_hook == 2);
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
    float *D32 = (float *)buf.get(nn * 4);
    double2 *part = (double2 *)buf.get(sizeof(double2) * RED_BLOCKS);
    int *d_choice = (int *)buf.get(64);
    int *d_err = (int *)buf.get(64);
    double *d_rec = (double *)buf.get(sizeof(double) * 4 * 16 + 64);
    if (!X64 || !D32 || !part || !d_choice || !d_err || !d_rec) return SP2_ERR_NOMEM;
    // The chain's workspace, with the call's other buffers (so that no allocation
    // falls inside the timed phases), 256-byte aligned as sp2_density requires.
    const size_t chain_bytes = sp2_density_workspace_bytes(N, &opt);
    uint8_t *chain_raw = (uint8_t *)buf.get(chain_bytes + 256);
    if (!chain_raw) return SP2_ERR_NOMEM;
    void *chain_ws = (void *)(((uintptr_t)chain_raw + 255) & ~(uintptr_t)255);
    CKS(cudaMemsetAsync(d_err, 0, sizeof(int), s));
    CongruenceBufs cb;
    if (Z) {
        if (!alloc_operand(buf, cb.m, np, slices) || !alloc_operand(buf, cb.z, np, slices) ||
            !alloc_operand(buf, cb.w, np, slices))
            return SP2_ERR_NOMEM;
        cb.inter = (double *)buf.get(nn * 8);
        cb.scratch = (double *)buf.get(nn * 8);
        cb.pscr = (long long *)buf.get(xs_scratch_bytes(pairs));
        if (!cb.inter || !cb.scratch || !cb.pscr) return SP2_ERR_NOMEM;
    }

    PhaseEvents pe(opt.profile != 0);
    pe.mark(0, s);
    // H_orth = Z^T H Z; the chain runs on it.
    const double *Hc = H;
    if (Z) {
        sp2_status r = congruence(Z, H, N, 0, X64, cb, d_err, pairs, slices, timeout_ns, s);
        if (r != SP2_OK) return r;
        r = read_err(d_err, s);
        if (r != SP2_OK) return r;
        Hc = X64;
    }
    sp2_stats local;
    memset(&local, 0, sizeof(local));
    std::vector<sp2_layer_stat> lay(SP2_MAX_LAYERS_LIMIT + 16);
    local.layer = lay.data();
    local.layer_cap = (int)lay.size();
    sp2_status r = sp2_density(Hc, N, n_occ, tol, D32, &local, &opt, chain_ws, chain_bytes, s);
    if (r != SP2_OK && r != SP2_ERR_NOT_CONVERGED) return r;
    const sp2_status chain_status = r;
    pe.mark(1, s);

    // Refinement layers on Y = X - I/2 in fixed point (X64 then holds D_orth).
    std::vector<double> rec(4 * (refine_layers + 2), 0.0);
    if (refine_layers > 0) {
        const int beta = xs_choose_beta(slices, np);
        long long *Y = (long long *)buf.get((size_t)np * np * 8);   // updated in place, layer by layer
        XsOperand sl[2];
        double2 *xpart = (double2 *)buf.get(xs_part_bytes(np));
        long long *pscr = (long long *)buf.get(xs_scratch_bytes(pairs));
        if (!pscr) return SP2_ERR_NOMEM;
        for (int k = 0; k < 2; ++k) {
            sl[k].base = (uint16_t *)buf.get((size_t)slices * np * np * 2);
            if (!sl[k].base) return SP2_ERR_NOMEM;
        }
        if (!Y) return SP2_ERR_NOMEM;
        if (!xpart) return SP2_ERR_NOMEM;
        int nparts = 0;
        CKS(xs_init_sp2(D32, N, np, slices, beta, Y, sl[0].base, xpart, &nparts, d_err, s));
        CKS(xs_decide(xpart, nparts, N, n_occ, d_choice, d_rec, s));
        XsProduct p;
        p.mode = XS_SP2;
        p.n = N;
        p.np = np;
        p.slices = slices;
        p.beta = beta;
        p.choice = d_choice;
        p.part = xpart;
        p.scratch = pscr;
        p.err = d_err;
        p.timeout_ns = timeout_ns;
        const int nt = xs_tile_count(np, XS_SP2);
        for (int l = 0; l < refine_layers; ++l) {
            p.a = p.b = sl[l & 1];
            p.y_in = Y;
            p.y_out = Y;
            p.next_slices = sl[(l + 1) & 1].base;
            CKS(xs_product(p, pairs, s));
            CKS(xs_decide(xpart, 2 * nt, N, n_occ, d_choice, d_rec + 4 * (l + 1), s));
        }
        CKS(xs_finish_sp2(Y, N, np, slices, beta, X64, s));
    } else {
        k_f32_to_f64<<<grid_for(nn), T64, 0, s>>>(D32, X64, nn);
        CKS(cudaGetLastError());
    }
    pe.mark(2, s);
    // Back-transformation D = Z D_orth Z^T.
    double *Dfin = X64;
    if (Z) {
        Dfin = (double *)buf.get(nn * 8);
        if (!Dfin) return SP2_ERR_NOMEM;
        sp2_status rc = congruence(Z, X64, N, 1, Dfin, cb, d_err, pairs, slices, timeout_ns, s);
        if (rc != SP2_OK) return rc;
    }
    // FP64 Tr[D H] (original H) and Tr D.
    const int rb = N < RED_BLOCKS ? N : RED_BLOCKS;
    k_energy64<<<rb, T64, 0, s>>>(Dfin, H, N, part);
    k_sum_parts<<<1, 32, 0, s>>>(part, rb, d_rec + 4 * (refine_layers + 1));
    CKS(cudaGetLastError());
    pe.mark(3, s);
    if (is_device_ptr(D_out)) CKS(cudaMemcpyAsync(D_out, Dfin, nn * 8, cudaMemcpyDeviceToDevice, s));
    else CKS(cudaMemcpyAsync(D_out, Dfin, nn * 8, cudaMemcpyDeviceToHost, s));
    CKS(cudaMemcpyAsync(rec.data(), d_rec, sizeof(double) * rec.size(), cudaMemcpyDeviceToHost, s));
    const sp2_status dev_status = read_err(d_err, s);
    if (dev_status != SP2_OK) return dev_status;

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
        for (; k <= L && k < cap && user_layers; ++k) st->layer[k] = lay[k];
        for (int l = 1; l <= refine_layers && L + l < cap && user_layers; ++l) {
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
        pe.fill(st->phase_ms);
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

extern "C" sp2_status sp2_congruence(const double *Z, const double *M, int N, int side, double *out,
                                     const sp2_opts *o, void *stream) {
    if (N < 1 || N > 65536 || !Z || !M || !out || (side != 0 && side != 1)) return SP2_ERR_ARG;
    if (!is_device_ptr(Z) || !is_device_ptr(M) || !is_device_ptr(out)) return SP2_ERR_ARG;
    sp2_opts opt;
    sp2_default_opts(&opt);
    if (o) opt = *o;
    const int slices = slices_of(opt);
    if (!slices) return SP2_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (!xs_available()) return SP2_ERR_UNSUPPORTED;
    const int pairs = xs_resident_pairs(sm_count_now());
    if (pairs < 1) return SP2_ERR_UNSUPPORTED;
    const int np = round_up(N, XS_TILE_N);
    const size_t nn = (size_t)N * N;
    DevBuf buf(s);
    buf.fail = (opt.test_hook == 2);
    CongruenceBufs cb;
    int *d_err = (int *)buf.get(64);
    if (!d_err || !alloc_operand(buf, cb.m, np, slices) || !alloc_operand(buf, cb.z, np, slices) ||
        !alloc_operand(buf, cb.w, np, slices))
        return SP2_ERR_NOMEM;
    cb.inter = (double *)buf.get(nn * 8);
    cb.scratch = (double *)buf.get(nn * 8);
    cb.pscr = (long long *)buf.get(xs_scratch_bytes(pairs));
    if (!cb.inter || !cb.scratch || !cb.pscr) return SP2_ERR_NOMEM;
    CKS(cudaMemsetAsync(d_err, 0, sizeof(int), s));
    sp2_status r =
        congruence(Z, M, N, side, out, cb, d_err, pairs, slices, (unsigned long long)(opt.timeout_ms * 1e6), s);
    if (r != SP2_OK) return r;
    return read_err(d_err, s);
}
