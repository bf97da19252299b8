// aux_kernels.cu -- the HBM-bound steps around the layer loop:
//   * Gershgorin spectral bounds of H in FP64 (one read pass over H),
//   * the input layer X_0 = (eps_max I - H)/(eps_max - eps_min) with its FP32
//     master, split operands and FP64 trace partials (one read of H, one write of X),
//   * the response / adjoint stream start Y_0 (scaled by a power of two),
//   * the output copy D = X_L with FP64 Tr[D H] and Tr D.
#include "device_common.cuh"

namespace sp2i {

namespace {

constexpr int AUX_THREADS = 256;

// ---------------------------------------------------------------------------
// FP64 -> FP32 pairs with 32-bit integer operations only.  GB300 runs FP64
// arithmetic and FP64 <-> FP32 conversions at a small fraction of its FP32 and
// integer rates, so the HBM-bound kernels that read FP64 matrices unpack them
// here.  split_f64(v, hi, lo24): hi = v with its mantissa truncated to 24
// bits, lo24 = 2^24 x (the next 24 bits, truncated), so that
// 0 <= |v| - (|hi| + 2^-24 |lo24|) < 2^-47 |v| for |v| >= 2^-98; below that
// lo24 is 0 and the cut is < 2^-121.  The 2^24 keeps lo24 a normal float.
// Values below 2^-126 give hi = 0; non-finite inputs and |v| >= 2^128 set `bad`.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void split_f64(double v, float &hi, float &lo24, int &bad) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    const unsigned int h32 = (unsigned int)(b >> 32), l32 = (unsigned int)b;
    const unsigned int sign = h32 & 0x80000000u;
    const int e = (int)((h32 >> 20) & 0x7FFu);
    if (e == 0x7FF) bad = 1;
    const int e32 = e - 1023 + 127;
    if (e == 0 || e32 <= 0 || e32 >= 255) {
        hi = 0.0f;
        lo24 = 0.0f;
        if (e32 >= 255 && e != 0x7FF) bad = 1;
        return;
    }
    // 52-bit mantissa m = [h32 & 0xFFFFF : l32]; hi keeps its top 23 bits.
    const unsigned int mhi = ((h32 & 0xFFFFFu) << 3) | (l32 >> 29);
    hi = __uint_as_float(sign | ((unsigned int)e32 << 23) | mhi);
    // The remaining 29 bits (l32 & 0x1FFFFFFF) weigh 2^(e - 1023 - 52); times
    // 2^24 that is the float exponent field e32 - 28.
    const unsigned int rem = l32 & 0x1FFFFFFFu;
    const float r = __uint2float_rz(rem) * __uint_as_float((unsigned int)(e32 > 28 ? e32 - 28 : 1) << 23);
    lo24 = (e32 > 28) ? (sign ? -r : r) : 0.0f;
}

__device__ __forceinline__ double warp_sum_d(double v) {
    // Fixed shuffle-down tree: lane 0 holds the sum, in the same order every run.
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// Block-wide deterministic sum of three doubles; result valid in thread 0.
__device__ __forceinline__ double3 block_sum3(double a, double b, double c) {
    __shared__ double sa[AUX_THREADS / 32], sb[AUX_THREADS / 32], sc[AUX_THREADS / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    a = warp_sum_d(a);
    b = warp_sum_d(b);
    c = warp_sum_d(c);
    if (lane == 0) {
        sa[w] = a;
        sb[w] = b;
        sc[w] = c;
    }
    __syncthreads();
    double3 r = make_double3(0.0, 0.0, 0.0);
    if (threadIdx.x == 0) {
        for (int k = 0; k < AUX_THREADS / 32; ++k) {
            r.x += sa[k];
            r.y += sb[k];
            r.z += sc[k];
        }
    }
    __syncthreads();
    return r;
}

// Block-wide deterministic sum of two doubles; result valid in thread 0.
__device__ __forceinline__ double2 block_sum2(double a, double b) {
    __shared__ double sa[AUX_THREADS / 32], sb[AUX_THREADS / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    a = warp_sum_d(a);
    b = warp_sum_d(b);
    if (lane == 0) {
        sa[w] = a;
        sb[w] = b;
    }
    __syncthreads();
    double2 r = make_double2(0.0, 0.0);
    if (threadIdx.x == 0) {
        for (int k = 0; k < AUX_THREADS / 32; ++k) {
            r.x += sa[k];
            r.y += sb[k];
        }
    }
    __syncthreads();
    return r;
}

// Gershgorin discs: one warp per row.  Each off-diagonal |H_ij| is unpacked
// with integer operations into |hi| + 2^-24 |lo24|, which falls short of it by
// less than 2^-47 relative (2^-121 absolute for tiny entries); the |hi| are
// summed in compensated FP32 pairs and the |lo24| in FP32.  The radius is then
// widened to r (1 + 2^-36) + 2^-50 |d| + N 2^-120, which covers the cut, the
// sums and the rounding of d -/+ r, so the bounds contain every exact disc and
// exceed it by about 2^-36 relative.  Centres and bounds are FP64.
__global__ void __launch_bounds__(AUX_THREADS) k_gershgorin(InstDesc *inst) {
    const InstDesc &d = inst[blockIdx.y];
    const int n = d.n;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    double lo = INFINITY, hi = -INFINITY;
    int bad = 0;
    for (int row = blockIdx.x * (AUX_THREADS / 32) + w; row < n; row += gridDim.x * (AUX_THREADS / 32)) {
        const double *__restrict__ h = d.H + (size_t)row * n;
        FF acc[2] = {{0.f, 0.f}, {0.f, 0.f}};
        float acc_lo = 0.0f;  // sum of the 2^24-scaled low parts
        for (int j0 = lane; j0 < n; j0 += 32 * 8) {
            double v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int j = j0 + 32 * u;
                v[u] = (j < n) ? h[j] : 0.0;
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int j = j0 + 32 * u;
                float a, b;
                split_f64(v[u], a, b, bad);
                if (j != row) {
                    ff_add(acc[u & 1], fabsf(a));
                    acc_lo += fabsf(b);
                }
            }
        }
        double rs = warp_sum_d(ff_value(acc[0]) + ff_value(acc[1]) + (double)acc_lo * 0x1p-24);
        rs = __shfl_sync(0xffffffffu, rs, 0);
        const double dv = h[row];
        if (!isfinite(dv)) bad = 1;
        rs = rs * (1.0 + 0x1p-36) + fabs(dv) * 0x1p-50 + (double)n * 0x1p-120;
        lo = fmin(lo, dv - rs);
        hi = fmax(hi, dv + rs);
    }
    bad = __any_sync(0xffffffffu, bad);
    if (lane == 0) {
        if (lo <= hi) {
            atomicMin(&d.ctl->emin_key, dkey(lo));
            atomicMax(&d.ctl->emax_key, dkey(hi));
        }
        if (bad) atomicOr(&d.ctl->nonfinite, 1);
    }
}

// max |M_ij| over an n x n FP64 matrix (H1 or G), for the power-of-two scale of Y.
__global__ void __launch_bounds__(AUX_THREADS) k_maxabs(InstDesc *inst) {
    const InstDesc &d = inst[blockIdx.y];
    const size_t total = (size_t)d.n * d.n;
    double m = 0.0;
    int bad = 0;
    float mf = 0.0f;
    for (size_t e = (size_t)blockIdx.x * AUX_THREADS + threadIdx.x; e < total; e += (size_t)gridDim.x * AUX_THREADS) {
        float a, b;
        split_f64(d.H1[e], a, b, bad);
        mf = fmaxf(mf, fabsf(a) + fabsf(b) * 0x1p-24f);
    }
    m = (double)mf;
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_down_sync(0xffffffffu, m, o));
    bad = __any_sync(0xffffffffu, bad);
    if ((threadIdx.x & 31) == 0) {
        atomicMax(&d.ctl->ymax_key, dkey(m));
        if (bad) atomicOr(&d.ctl->nonfinite, 1);
    }
}

__device__ __forceinline__ void resolve_bounds(const InstDesc &d, bool user_bounds, double &emin, double &emax) {
    if (user_bounds) {
        emin = d.ctl->eps_min;
        emax = d.ctl->eps_max;
    } else {
        emin = dkey_value(d.ctl->emin_key);
        emax = dkey_value(d.ctl->emax_key);
    }
}

// X_0 over the padded np x np matrix; four consecutive columns per thread.
template <int PATH, int PREC>
__global__ void __launch_bounds__(AUX_THREADS) k_init_x(InstDesc *inst, int user_bounds) {
    const InstDesc &d = inst[blockIdx.y];
    const int n = d.n, np = d.np;
    double emin, emax;
    resolve_bounds(d, user_bounds != 0, emin, emax);
    const double delta = emax - emin;
    const bool degenerate = !(delta > 0.0) || !isfinite(delta) || d.ctl->nonfinite;
    const double inv = degenerate ? 0.0 : 1.0 / delta;
    const float inv_hi = (float)inv;                 // 1/delta as a float pair
    const float inv_lo = (float)(inv - (double)inv_hi);
    const float inv_lo24 = inv_hi * 0x1p-24f;       // weight of the 2^24-scaled low part
    int bad_unused = 0;
    float *__restrict__ xf = xmaster(d, 0, false);
    uint16_t *__restrict__ op1 = d.xop;                    // hi
    uint16_t *__restrict__ op2 = d.xop + (size_t)np * np;  // lo
    // ft: Tr X_0; fq: ||X_0||_F^2; fw (tensor-core path): ||Y_0||_F^2 - ||X_0||_F^2,
    // which only the diagonal (y = x - 1/2 there) contributes.
    FF ft = {0.f, 0.f}, fq = {0.f, 0.f}, fw = {0.f, 0.f};
    // Rows are strided over blocks, four consecutive columns per thread: no
    // index divisions on the hot loop; restrict-qualified so that the loads of
    // the next columns can be issued ahead of this group's stores.
    for (int i = blockIdx.x; i < np; i += gridDim.x) {
        const double *__restrict__ hrow = d.H + (size_t)(i < n ? i : 0) * n;
        // The row's diagonal entry in FP64, once per row (FP64 is slow on this part),
        // and its terms of the diagonal sums in the thread that stores it.
        const float xdiag = (i < n) ? (float)((emax - hrow[i]) * inv) : 0.0f;
        if (i < n && (int)threadIdx.x == (i % (AUX_THREADS * 4)) / 4) {
            ff_add(ft, xdiag);
            if (PATH == PATH_TC) {
                ff_add_sq(fw, xdiag - 0.5f, 1.0f);
                ff_add_sq(fw, xdiag, -1.0f);
            }
        }
#pragma unroll 2
        for (int j0 = threadIdx.x * 4; j0 < np; j0 += AUX_THREADS * 4) {
            const size_t idx = (size_t)i * np + j0;
            float x[4], y[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int j = j0 + q;
                float v = 0.0f;
                if (i < n && j < n) {
                    float a, b;  // -h / (eps_max - eps_min): one rounding of a sum of small terms
                    split_f64(hrow[j], a, b, bad_unused);
                    v = (i == j) ? xdiag : -fmaf(a, inv_hi, fmaf(a, inv_lo, b * inv_lo24));
                }
                x[q] = v;
                y[q] = (i == j && i < n) ? v - 0.5f : v;
                ff_add_sq(fq, v, 1.0f);
            }
            if (PATH == PATH_SIMT || j0 + 3 <= i) {
                *(float4 *)(xf + idx) = make_float4(x[0], x[1], x[2], x[3]);
            } else if (j0 <= i) {
                // The tensor-core layers and the output read the master's lower
                // triangle and diagonal only.
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    if (j0 + q <= i) xf[idx + q] = x[q];
            }
            if (PATH == PATH_TC) {
                // operands of the first square: the split of Y_0 = X_0 - I/2
                uint16_t b[4], c[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) split2<PREC, X_SHIFT>(y[q], b[q], c[q]);
                *(ushort4 *)(op1 + idx) = make_ushort4(b[0], b[1], b[2], b[3]);
                *(ushort4 *)(op2 + idx) = make_ushort4(c[0], c[1], c[2], c[3]);
            }
        }
    }
    if (PATH == PATH_TC) ff_add_ff(fw, fq);   // ||Y_0||_F^2
    double3 s = block_sum3(ff_value(ft), ff_value(fq), ff_value(fw));
    if (threadIdx.x == 0) {
        Part pr;
        pr.t = s.x;
        pr.q = s.y;
        pr.w = s.z;
        pr.p = 0.0;
        d.part[0][blockIdx.x] = pr;
        if (blockIdx.x == 0) {
            d.ctl->init_parts = gridDim.x;
            d.ctl->eps_min = emin;
            d.ctl->eps_max = emax;
            if (d.ctl->nonfinite) d.ctl->status = SP2_ERR_NONFINITE;
            else if (degenerate) d.ctl->degenerate = 1;
        }
    }
}

// X_0 given directly (FP32, n x n), for the layer-application entry point.
template <int PATH, int PREC>
__global__ void __launch_bounds__(AUX_THREADS) k_init_x_from(InstDesc *inst, const float *X0) {
    const InstDesc &d = inst[0];
    const int n = d.n, np = d.np;
    float *xf = d.xf[0];
    uint16_t *op1 = d.xop, *op2 = d.xop + (size_t)np * np;
    FF ft = {0.f, 0.f}, fq = {0.f, 0.f}, fw = {0.f, 0.f};
    for (int i = blockIdx.x; i < np; i += gridDim.x) {
        for (int j = threadIdx.x; j < np; j += AUX_THREADS) {
            const size_t idx = (size_t)i * np + j;
            const float v = (i < n && j < n) ? X0[(size_t)i * n + j] : 0.0f;
            xf[idx] = v;
            if (i == j) ff_add(ft, v);
            ff_add_sq(fq, v, 1.0f);
            if (PATH == PATH_TC) {
                const float y = (i == j && i < n) ? v - 0.5f : v;
                ff_add_sq(fw, y, 1.0f);
                uint16_t b, c;
                split2<PREC, X_SHIFT>(y, b, c);
                op1[idx] = b;
                op2[idx] = c;
            }
        }
    }
    double3 s = block_sum3(ff_value(ft), ff_value(fq), ff_value(fw));
    if (threadIdx.x == 0) {
        Part pr;
        pr.t = s.x;
        pr.q = s.y;
        pr.w = s.z;
        pr.p = 0.0;
        d.part[0][blockIdx.x] = pr;
        if (blockIdx.x == 0) d.ctl->init_parts = gridDim.x;
    }
}

// Y_0 = coef * y_scale * (M + M^T)/2 over the padded matrix.  coef is
// -1/(eps_max - eps_min) for the response (X1_0 = -H1/(eps_max - eps_min)) and 1
// for the adjoint (G_L = sym(G)); y_scale is the power of two that brings
// max |Y_0| into (1/2, 1] so that the 16-bit split operands stay in range.
template <int PREC>
__global__ void __launch_bounds__(AUX_THREADS) k_init_y(InstDesc *inst, int mode) {
    const InstDesc &d = inst[0];
    const int n = d.n, np = d.np;
    const double emin = d.ctl->eps_min, emax = d.ctl->eps_max;
    const double coef = (mode == MODE_RESPONSE) ? -1.0 / (emax - emin) : 1.0;
    const double mabs = dkey_value(d.ctl->ymax_key) * fabs(coef);
    int ex = 0;
    if (mabs > 0.0 && isfinite(mabs)) frexp(mabs, &ex);  // mabs in [2^(ex-1), 2^ex)
    const double yscale = ldexp(1.0, -ex);
    const double c = coef * yscale;
    uint16_t *op1 = d.yop, *op2 = d.yop + (size_t)np * np;
    for (int i = blockIdx.x; i < np; i += gridDim.x)
        for (int j = threadIdx.x; j < np; j += AUX_THREADS) {
        const size_t idx = (size_t)i * np + j;
        double a = 0.0, b = 0.0;
        if (i < n && j < n) {
            a = d.H1[(size_t)i * n + j];
            b = d.H1[(size_t)j * n + i];
        }
        const float y = (float)(0.5 * (a + b) * c);
        d.yf[0][idx] = y;
        uint16_t o1, o2;
        split2<PREC, Y_SHIFT>(y, o1, o2);
        op1[idx] = o1;
        op2[idx] = o2;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) d.ctl->y_scale = yscale;
}

// D = X_L (un-padded copy, diagonal offset added), FP64 partials of Tr[D H] and
// Tr D per block; the response / adjoint output is the Y stream with its scale
// removed.  The layer kernels keep only the lower triangle and the diagonal of
// the FP32 masters current (the next layer reads nothing else), so the output
// is assembled from 32 x 32 lower-triangle tiles (ti >= tj) staged in shared
// memory: each tile is written to (ti, tj) and, transposed, to (tj, ti), both
// with coalesced rows.  H is symmetric, so Tr[D H] is summed over the lower
// triangle with off-diagonal weight 2.
// Eight blocks per SM (32 registers per thread at most): the 1024 blocks then run as one wave.
__global__ void __launch_bounds__(AUX_THREADS, 8) k_finalize(InstDesc *inst, int mode) {
    __shared__ float sx[32][33], sy[32][33];
    const InstDesc &d = inst[blockIdx.y];
    if (blockIdx.x >= d.fin_blocks) return;
    const int n = d.n, np = d.np;
    const InstCtl *ctl = d.ctl;
    const float *__restrict__ X = d.ckpt_s > 0 ? xmaster(d, ctl->layers, false) : d.xf[ctl->final_x & 1];
    const float *__restrict__ Y = d.yf[ctl->final_y & 1];
    const double *__restrict__ H = d.H;
    float *__restrict__ out = d.out;
    float *__restrict__ out1 = d.out1;
    const float xoff = (float)ctl->x_offset;
    const bool second = (mode == MODE_RESPONSE || mode == MODE_ADJOINT);
    float ys = 0.0f;
    if (mode == MODE_RESPONSE) ys = (float)(1.0 / ctl->y_scale);
    if (mode == MODE_ADJOINT) ys = (float)(-1.0 / (ctl->y_scale * (ctl->eps_max - ctl->eps_min)));
    // Tr[D H]: each H_ij unpacked to an FP32 pair (h1 + 2^-24 h2), x * h1 split exactly
    // into product and error (FMA), all summed in a compensated FP32 pair.
    FF fe = {0.f, 0.f}, ftr = {0.f, 0.f};   // compensated FP32 pairs (FP64 is slow on this part)
    int bad_unused = 0;
    const int tc = threadIdx.x & 31, tr0 = threadIdx.x >> 5;   // tile column, first tile row
    const int nt = (n + 31) / 32;
    const long long ntiles = (long long)nt * (nt + 1) / 2;
    for (long long k = blockIdx.x; k < ntiles; k += d.fin_blocks) {
        // k -> (ti, tj) with tj <= ti, row-major over the lower triangle of tiles: an FP32
        // root (FP64 is slow on this GPU) corrected to the exact integer below
        int ti = (int)((sqrtf(8.0f * (float)k + 1.0f) - 1.0f) * 0.5f);
        while ((long long)(ti + 1) * (ti + 2) / 2 <= k) ++ti;
        while ((long long)ti * (ti + 1) / 2 > k) --ti;
        const int tj = (int)(k - (long long)ti * (ti + 1) / 2);
        const int i0 = ti * 32, j0 = tj * 32;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int r = tr0 + 8 * q, i = i0 + r, j = j0 + tc;
            float x = 0.0f, yv = 0.0f;
            if (i < n && j < n && (ti > tj || r >= tc)) {
                x = X[(size_t)i * np + j];
                if (i == j) {
                    x += xoff;  // true X_L = stored X_L + c_L I
                    ff_add(ftr, x);
                }
                if (H) {
                    float h1, h2;
                    split_f64(H[(size_t)i * n + j], h1, h2, bad_unused);
                    const float wgt = (j == i) ? 1.0f : 2.0f;
                    const float p = __fmul_rn(x, h1);
                    const float perr = __fmaf_rn(x, h1, -p);
                    ff_add(fe, __fmul_rn(wgt, p));
                    fe.c = __fadd_rn(fe.c, __fmul_rn(wgt, __fmaf_rn(x, h2 * 0x1p-24f, perr)));
                }
                if (second) yv = Y[(size_t)i * np + j] * ys;
            }
            sx[r][tc] = x;
            sy[r][tc] = yv;
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int r = tr0 + 8 * q;
            const bool low = (ti > tj || r >= tc);   // the diagonal tile's upper half comes transposed
            int i = i0 + r, j = j0 + tc;
            if (i < n && j < n) {
                if (out) out[(size_t)i * n + j] = low ? sx[r][tc] : sx[tc][r];
                if (second) out1[(size_t)i * n + j] = low ? sy[r][tc] : sy[tc][r];
            }
            i = j0 + r;
            j = i0 + tc;
            if (ti > tj && i < n && j < n) {        // the mirror tile (tj, ti)
                if (out) out[(size_t)i * n + j] = sx[tc][r];
                if (second) out1[(size_t)i * n + j] = sy[tc][r];
            }
        }
        __syncthreads();
    }
    double2 s = block_sum2(ff_value(fe), ff_value(ftr));
    if (threadIdx.x == 0) d.fin_part[blockIdx.x] = s;
}

// One block per instance: fixed-stride partial sums, then the fixed block tree.
__global__ void __launch_bounds__(AUX_THREADS) k_finalize_reduce(InstDesc *inst) {
    const InstDesc &d = inst[blockIdx.x];
    double e = 0.0, tr = 0.0;
    for (int k = threadIdx.x; k < d.fin_blocks; k += AUX_THREADS) {
        e += d.fin_part[k].x;
        tr += d.fin_part[k].y;
    }
    double2 s = block_sum2(e, tr);
    if (threadIdx.x == 0) {
        d.ctl->band_energy = s.x;
        d.ctl->trace_D = s.y;
    }
}

__global__ void k_fill_trivial(float *D, int n, float diag) {
    const size_t total = (size_t)n * n;
    for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += (size_t)gridDim.x * blockDim.x)
        D[idx] = ((idx / n) == (idx % n)) ? diag : 0.0f;
}

int grid_for(size_t work, int per_block, int cap) {
    size_t g = (work + per_block - 1) / per_block;
    if (g < 1) g = 1;
    if (g > (size_t)cap) g = cap;
    return (int)g;
}

}  // namespace

cudaError_t launch_gershgorin(InstDesc *inst, int B, int max_n, bool user_bounds, cudaStream_t s) {
    (void)user_bounds;  // bounds are computed anyway: the same pass detects non-finite input
    dim3 grid(grid_for((size_t)max_n, AUX_THREADS / 32, 2048), B);
    k_gershgorin<<<grid, AUX_THREADS, 0, s>>>(inst);
    return cudaGetLastError();
}

cudaError_t launch_maxabs(InstDesc *inst, int B, int max_n, cudaStream_t s) {
    dim3 grid(grid_for((size_t)max_n * max_n, AUX_THREADS * 8, 2048), B);
    k_maxabs<<<grid, AUX_THREADS, 0, s>>>(inst);
    return cudaGetLastError();
}

// One or more rows per block; the host sizes the partial buffers with the same rule.
int init_blocks_for(int np) { return np < INIT_BLOCKS_MAX ? np : INIT_BLOCKS_MAX; }

cudaError_t launch_init_x(InstDesc *inst, int B, int max_np, int path, int precision, bool user_bounds,
                          cudaStream_t s) {
    dim3 grid(init_blocks_for(max_np), B);
    // Every instance must be covered by the same number of blocks it reports in
    // init_parts: the grid-stride loop handles any np with this grid.
    const int ub = user_bounds ? 1 : 0;
    if (path == PATH_SIMT) k_init_x<PATH_SIMT, SP2_FP16_SPLIT><<<grid, AUX_THREADS, 0, s>>>(inst, ub);
    else if (precision == SP2_BF16_SPLIT) k_init_x<PATH_TC, SP2_BF16_SPLIT><<<grid, AUX_THREADS, 0, s>>>(inst, ub);
    else k_init_x<PATH_TC, SP2_FP16_SPLIT><<<grid, AUX_THREADS, 0, s>>>(inst, ub);
    return cudaGetLastError();
}

cudaError_t launch_init_x_from(InstDesc *inst, const float *X0, int np, int path, int precision, cudaStream_t s) {
    // Same block count rule as the input layer: the partial buffer holds
    // max(tiles, init_blocks_for(np)) entries and every block writes one.
    const int grid = init_blocks_for(np);
    if (path == PATH_SIMT) k_init_x_from<PATH_SIMT, SP2_FP16_SPLIT><<<grid, AUX_THREADS, 0, s>>>(inst, X0);
    else if (precision == SP2_BF16_SPLIT) k_init_x_from<PATH_TC, SP2_BF16_SPLIT><<<grid, AUX_THREADS, 0, s>>>(inst, X0);
    else k_init_x_from<PATH_TC, SP2_FP16_SPLIT><<<grid, AUX_THREADS, 0, s>>>(inst, X0);
    return cudaGetLastError();
}

cudaError_t launch_init_y(InstDesc *inst, int mode, int precision, cudaStream_t s) {
    const int grid = 1024;
    if (precision == SP2_BF16_SPLIT) k_init_y<SP2_BF16_SPLIT><<<grid, AUX_THREADS, 0, s>>>(inst, mode);
    else k_init_y<SP2_FP16_SPLIT><<<grid, AUX_THREADS, 0, s>>>(inst, mode);
    return cudaGetLastError();
}

cudaError_t launch_finalize(InstDesc *inst, int B, int max_n, int mode, cudaStream_t s) {
    (void)max_n;
    dim3 grid(FIN_BLOCKS_MAX, B);
    k_finalize<<<grid, AUX_THREADS, 0, s>>>(inst, mode);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_finalize_reduce<<<B, AUX_THREADS, 0, s>>>(inst);
    return cudaGetLastError();
}

cudaError_t launch_fill_trivial(float *D, int n, float diag_value, cudaStream_t s) {
    k_fill_trivial<<<grid_for((size_t)n * n, 256, 4096), 256, 0, s>>>(D, n, diag_value);
    return cudaGetLastError();
}

}  // namespace sp2i
