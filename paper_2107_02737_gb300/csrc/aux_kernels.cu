// aux_kernels.cu -- the HBM-bound steps around the layer loop:
//   * Gershgorin spectral bounds of H in FP64 (one read of H's lower triangle,
//     then one FP64 sum per row),
//   * the input layer X_0 = (eps_max I - H)/(eps_max - eps_min) with its FP32
//     master, split operands and FP64 trace partials (one read of H's lower
//     triangle, one write of X),
//   * the response / adjoint stream start Y_0 (scaled by a power of two),
//   * the output copy D = X_L with FP64 Tr[D H] and Tr D.
#include <algorithm>

#include "device_common.cuh"

namespace sp2i {

namespace {

constexpr int AUX_THREADS = 256;

// ---------------------------------------------------------------------------
// FP64 -> FP32 pairs with 32-bit integer and FP32 operations only.  GB300 runs
// FP64 arithmetic and its conversion instructions (FP64 <-> FP32, integer ->
// float, FP32 -> FP16 one value at a time) at a small fraction of its FP32 and
// integer rates, so the HBM-bound kernels that read FP64 matrices unpack them
// here.  split_f64(v, hi, lo24): hi = v with its mantissa truncated to 24
// bits, lo24 = 2^24 x (the next 24 bits, truncated), so that
// 0 <= |v| - (|hi| + 2^-24 |lo24|) < 2^-47 |v| for |v| >= 2^-98; below that
// lo24 is 0 and the cut is < 2^-121.  The 2^24 keeps lo24 a normal float.
// The 24-bit integer becomes a float exactly by the exponent-field identity
// float(2^23 + m) = bits(0x4B000000 | m) for m < 2^23, and one more exact add
// for its top bit.  Values below 2^-126 give hi = 0; non-finite inputs and
// |v| >= 2^128 set `bad`.
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
    // The top 24 of the remaining 29 bits, (l32 & 0x1FFFFFFF) >> 5, weigh
    // 2^(e - 1023 - 47) each; times 2^24 that is the float exponent field e32 - 23.
    const unsigned int rem = (l32 & 0x1FFFFFFFu) >> 5;
    const float m = __uint_as_float(0x4B000000u | (rem & 0x7FFFFFu)) - 0x1p23f;   // low 23 bits, exact
    const float q = m + ((rem >> 23) ? 0x1p23f : 0.0f);                           // < 2^24, exact
    const float r = q * __uint_as_float((unsigned int)(e32 > 28 ? e32 - 23 : 1) << 23);
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

// ---------------------------------------------------------------------------
// Passes over the lower triangle.  H is symmetric, so the bounds, the input
// layer and the output read only its 64 x 64 tiles (ti, tj) with tj <= ti, and
// write what lies above the diagonal from the transposed tile.  A warp owns
// eight rows of a tile (w, w + 8, ...) and each lane two adjacent columns, so
// that every row of the tile is one 512-byte FP64 access per warp and a thread
// has sixteen loads in flight before it uses any.
// ---------------------------------------------------------------------------
constexpr int AT = 64;                             // tile side
constexpr int AT_RPW = AT / (AUX_THREADS / 32);    // rows per warp: 8
constexpr int AT_BLOCKS_PER_SM = 4;                // residency the tile kernels are compiled for
constexpr int FIN_BLOCKS_PER_SM = 3;               // the output kernel's (sixteen FP64 loads per thread)

// k -> (ti, tj), tj <= ti, row-major over the lower triangle of tiles: an FP32
// root (FP64 is slow on this GPU) corrected to the exact integer.
__device__ __forceinline__ void lower_tile(long long k, int &ti, int &tj) {
    int t = (int)((sqrtf(8.0f * (float)k + 1.0f) - 1.0f) * 0.5f);
    while ((long long)(t + 1) * (t + 2) / 2 <= k) ++t;
    while ((long long)t * (t + 1) / 2 > k) --t;
    ti = t;
    tj = (int)(k - (long long)t * (t + 1) / 2);
}

// (M_ij, M_i,j+1) of an n x n FP64 matrix, j even, zero outside it; one 16-byte load
// when `vec` (n even and M 16-byte aligned).
__device__ __forceinline__ void load_pair(const double *__restrict__ M, int n, bool vec, int i, int j, double &a,
                                          double &b) {
    a = 0.0;
    b = 0.0;
    if (i >= n || j >= n) return;
    const double *p = M + (size_t)i * n + j;
    if (vec) {
        const double2 v = *(const double2 *)p;
        a = v.x;
        b = v.y;
    } else {
        a = p[0];
        if (j + 1 < n) b = p[1];
    }
}

// (out_ij, out_i,j+1) = (a, b) inside the n x n matrix, j even; one 8-byte store when `vec`.
__device__ __forceinline__ void store_pair(float *__restrict__ out, int n, bool vec, int i, int j, float a, float b) {
    if (i >= n || j >= n) return;
    float *p = out + (size_t)i * n + j;
    if (vec) {
        *(float2 *)p = make_float2(a, b);
    } else {
        p[0] = a;
        if (j + 1 < n) p[1] = b;
    }
}

// Compensated sum of the 16 floats v[0], v[stride], ..., v[15 stride].
__device__ __forceinline__ FF ff_chain16(const float *v, int stride) {
    FF a = {0.f, 0.f};
#pragma unroll
    for (int k = 0; k < 16; ++k) ff_add(a, v[k * stride]);
    return a;
}

// Sum of the 64 floats v[0], v[stride], ..., v[63 stride]: four compensated chains
// of sixteen, combined pairwise.
__device__ __forceinline__ FF ff_sum64(const float *v, int stride) {
    FF a = ff_chain16(v, stride), b = ff_chain16(v + 16 * stride, stride);
    FF c = ff_chain16(v + 32 * stride, stride), e = ff_chain16(v + 48 * stride, stride);
    ff_add_ff(a, b);
    ff_add_ff(c, e);
    ff_add_ff(a, c);
    return a;
}

__device__ __forceinline__ float f_sum64(const float *v, int stride) {
    float a = 0.0f;
#pragma unroll 16
    for (int k = 0; k < 64; ++k) a += v[k * stride];
    return a;
}

// Gershgorin discs, first pass: per lower tile, the absolute off-diagonal entries
// are unpacked with integer operations into |hi| + 2^-24 |lo24| (short of |H_ij| by
// < 2^-47 relative, or by < 2^-121 absolute for tiny entries) and staged in shared
// memory.  One thread per tile row sums its row (the rows of tile row ti, column
// block tj) and one thread per tile column its column (by symmetry, the rows of
// tile row tj, column block ti), so that row i receives exactly one partial per
// column block b, stored in P[b n + i]; a diagonal tile gives each of its rows one
// partial from its row and its column.  The |hi| of a partial are summed as four
// (diagonal tile: eight) compensated FP32 chains of sixteen combined pairwise, the
// |lo24| in FP32, and the partial is converted to FP64 once: its error is below
// 2^-39 of its value.  P is the second FP32 master buffer (4 np^2 bytes, at least
// 8 n ceil(n / 64) are needed), which nothing uses before the layers.
__global__ void __launch_bounds__(AUX_THREADS, AT_BLOCKS_PER_SM) k_gersh_tiles(InstDesc *inst) {
    __shared__ float sh[AT][AT + 1], sl[AT][AT + 1];
    const InstDesc &d = inst[blockIdx.y];
    const int n = d.n;
    const double *__restrict__ H = d.H;
    double *__restrict__ P = (double *)d.xf[1];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int nt = (n + AT - 1) / AT;
    const long long ntiles = (long long)nt * (nt + 1) / 2;
    const bool vec = ((n & 1) == 0) && (((uintptr_t)H & 15) == 0);
    int bad = 0;
    for (long long k = blockIdx.x; k < ntiles; k += gridDim.x) {
        int ti, tj;
        lower_tile(k, ti, tj);
        const int i0 = ti * AT, j0 = tj * AT, c0 = 2 * lane;
        const bool dg = (ti == tj);
        double h[AT_RPW][2];
#pragma unroll
        for (int q = 0; q < AT_RPW; ++q) load_pair(H, n, vec, i0 + w + 8 * q, j0 + c0, h[q][0], h[q][1]);
#pragma unroll
        for (int q = 0; q < AT_RPW; ++q) {
            const int r = w + 8 * q;
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                const int c = c0 + e;
                float a, b;
                split_f64(h[q][e], a, b, bad);   // zero outside the matrix
                const bool keep = !dg || c < r;  // strictly below the diagonal
                sh[r][c] = keep ? fabsf(a) : 0.0f;
                sl[r][c] = keep ? fabsf(b) : 0.0f;
            }
        }
        __syncthreads();
        const int t = threadIdx.x;
        if (t < AT) {                         // rows of tile row ti
            FF a = ff_sum64(&sh[t][0], 1);
            float lo = f_sum64(&sl[t][0], 1);
            if (dg) {                         // and the column part of the diagonal tile
                ff_add_ff(a, ff_sum64(&sh[0][t], AT + 1));
                lo += f_sum64(&sl[0][t], AT + 1);
            }
            if (i0 + t < n) P[(size_t)tj * n + i0 + t] = (double)a.s + (double)a.c + (double)lo * 0x1p-24;
        } else if (t < 2 * AT && !dg) {       // rows of tile row tj, from column block ti
            const int c = t - AT;
            FF a = ff_sum64(&sh[0][c], AT + 1);
            const float lo = f_sum64(&sl[0][c], AT + 1);
            if (j0 + c < n) P[(size_t)ti * n + j0 + c] = (double)a.s + (double)a.c + (double)lo * 0x1p-24;
        }
        __syncthreads();
    }
    bad = __syncthreads_or(bad);
    if (threadIdx.x == 0 && bad) atomicOr(&d.ctl->nonfinite, 1);
}

// Gershgorin discs, second pass: per row the FP64 sum of its partials (warp w of a
// block adds column blocks w, w + 8, ... for 32 consecutive rows, then the eight
// sums are added in warp order; error < 2^-45 of the sum for n <= 65536), then
// the radius widened to r (1 + 2^-36) + 2^-50 |d| + N 2^-120, which covers the
// unpacking cut, both passes' sums and the rounding of d -/+ r, so the bounds
// contain every exact disc and exceed it by about 2^-36 relative.  Centres and
// bounds are FP64; each block folds its extreme disc ends into the order-
// preserving keys with one atomic each.
constexpr int GR_ROWS = 32;   // rows per block of the second pass
__global__ void __launch_bounds__(AUX_THREADS) k_gersh_rows(InstDesc *inst) {
    __shared__ double sp[AUX_THREADS / 32][GR_ROWS];
    const InstDesc &d = inst[blockIdx.y];
    const int n = d.n;
    const double *__restrict__ P = (const double *)d.xf[1];
    const int nt = (n + AT - 1) / AT;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int row = blockIdx.x * GR_ROWS + lane;
    if (blockIdx.x * GR_ROWS >= n) return;   // block-uniform
    double part = 0.0;
    if (row < n) {
#pragma unroll 4
        for (int b = w; b < nt; b += AUX_THREADS / 32) part += P[(size_t)b * n + row];
    }
    sp[w][lane] = part;
    __syncthreads();
    if (w == 0) {
        double lo = INFINITY, hi = -INFINITY;
        if (row < n) {
            double rs = 0.0;
#pragma unroll
            for (int k = 0; k < AUX_THREADS / 32; ++k) rs += sp[k][lane];
            const double dv = d.H[(size_t)row * n + row];
            rs = rs * (1.0 + 0x1p-36) + fabs(dv) * 0x1p-50 + (double)n * 0x1p-120;
            lo = dv - rs;
            hi = dv + rs;
        }
        for (int o = 16; o > 0; o >>= 1) {
            lo = fmin(lo, __shfl_down_sync(0xffffffffu, lo, o));
            hi = fmax(hi, __shfl_down_sync(0xffffffffu, hi, o));
        }
        if (lane == 0 && lo <= hi) {
            atomicMin(&d.ctl->emin_key, dkey(lo));
            atomicMax(&d.ctl->emax_key, dkey(hi));
        }
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

// The 16-bit split (hi, lo) of two adjacent values, as packed pairs (element j in
// the low half): the same values as split2 gives one at a time, from conversions
// of two floats at once and exact scaling in the 16-bit domain.
template <int PREC, int SHIFT>
__device__ __forceinline__ void split2_pair(float a, float b, uint32_t &hi, uint32_t &lo) {
    if (PREC == SP2_FP16_SPLIT) {
        const __half2 h = __floats2half2_rn(a, b);
        const float2 hf = __half22float2(h);
        const __half2 hs = __hmul2(h, __float2half2_rn((float)(1 << SHIFT)));   // exact (|x| <= 1)
        const __half2 l = __floats2half2_rn(__fsub_rn(a, hf.x) * (float)(1 << SHIFT),
                                            __fsub_rn(b, hf.y) * (float)(1 << SHIFT));
        hi = *reinterpret_cast<const uint32_t *>(&hs);
        lo = *reinterpret_cast<const uint32_t *>(&l);
    } else {
        const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
        const float2 hf = __bfloat1622float2(h);
        const __nv_bfloat162 l = __floats2bfloat162_rn(__fsub_rn(a, hf.x), __fsub_rn(b, hf.y));
        hi = *reinterpret_cast<const uint32_t *>(&h);
        lo = *reinterpret_cast<const uint32_t *>(&l);
    }
}

// X_0 on the tensor-core path, from the lower triangle of H.  A tile (ti, tj) below
// the diagonal gives X_0 there, its FP32 master (the layers and the output read
// the master on and below the diagonal only) and the split operands of
// Y_0 = X_0 - I/2, and, transposed through shared memory, the split operands of
// the mirror tile (tj, ti); a diagonal tile completes its upper half the same way.
// Each element is the same function of H_ij as in the full pass, so X_0 is the same
// for a symmetric H (for any H, that of the symmetric matrix with H's lower
// triangle, as the bounds see it); ||X_0||_F^2 counts an element below the
// diagonal twice.
template <int PREC>
__global__ void __launch_bounds__(AUX_THREADS, AT_BLOCKS_PER_SM) k_init_x_tc(InstDesc *inst, int user_bounds) {
    __shared__ uint32_t sp[AT][AT + 1];   // (hi | lo << 16) of the tile, for the mirror
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
    const double *__restrict__ H = d.H;
    float *__restrict__ xf = xmaster(d, 0, false);
    uint16_t *__restrict__ op1 = d.xop;                    // hi
    uint16_t *__restrict__ op2 = d.xop + (size_t)np * np;  // lo
    // ft: Tr X_0; fq: ||X_0||_F^2; fw: ||Y_0||_F^2 - ||X_0||_F^2, which only the
    // diagonal (y = x - 1/2 there) contributes.
    FF ft = {0.f, 0.f}, fq = {0.f, 0.f}, fw = {0.f, 0.f};
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, c0 = 2 * lane;
    const int nt = np / AT;                          // np is a multiple of 128
    const long long ntiles = (long long)nt * (nt + 1) / 2;
    const bool vec = ((n & 1) == 0) && (((uintptr_t)H & 15) == 0);
    for (long long k = blockIdx.x; k < ntiles; k += gridDim.x) {
        int ti, tj;
        lower_tile(k, ti, tj);
        const int i0 = ti * AT, j0 = tj * AT;
        const bool dg = (ti == tj);
        double h[AT_RPW][2];
#pragma unroll
        for (int q = 0; q < AT_RPW; ++q) load_pair(H, n, vec, i0 + w + 8 * q, j0 + c0, h[q][0], h[q][1]);
#pragma unroll
        for (int q = 0; q < AT_RPW; ++q) {
            const int r = w + 8 * q, i = i0 + r;
            float x[2], yy[2];
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                const int j = j0 + c0 + e;
                float v = 0.0f, y = 0.0f;
                if (i < n && j < n && (!dg || c0 + e <= r)) {   // on or below the diagonal
                    if (i == j) {
                        // the diagonal in FP64 (emax - H_ii) / delta; its terms of the diagonal sums
                        v = (float)((emax - h[q][e]) * inv);
                        y = v - 0.5f;
                        ff_add(ft, v);
                        ff_add_sq(fw, y, 1.0f);
                        ff_add_sq(fw, v, -1.0f);
                    } else {
                        float a, lo24;  // -h / (eps_max - eps_min): one rounding of a sum of small terms
                        split_f64(h[q][e], a, lo24, bad_unused);
                        v = -fmaf(a, inv_hi, fmaf(a, inv_lo, lo24 * inv_lo24));
                        y = v;
                    }
                }
                ff_add_sq(fq, v, (i == j) ? 1.0f : 2.0f);   // an element below the diagonal counts twice
                x[e] = v;
                yy[e] = y;
            }
            uint32_t hp, lp;   // (hi, lo) of columns c0, c0 + 1
            split2_pair<PREC, X_SHIFT>(yy[0], yy[1], hp, lp);
            sp[r][c0] = __byte_perm(hp, lp, 0x5410);       // hi | lo << 16 of column c0
            sp[r][c0 + 1] = __byte_perm(hp, lp, 0x7632);   // ... and of column c0 + 1
            const size_t idx = (size_t)i * np + j0 + c0;
            *(float2 *)(xf + idx) = make_float2(x[0], x[1]);   // above the diagonal of a diagonal tile: unread
            if (!dg) {
                *(uint32_t *)(op1 + idx) = hp;
                *(uint32_t *)(op2 + idx) = lp;
            }
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < AT_RPW; ++q) {
            const int r = w + 8 * q;
            uint32_t u0, u1;
            size_t idx;
            if (dg) {   // block-uniform: the diagonal tile, its upper half from its lower half
                u0 = (c0 <= r) ? sp[r][c0] : sp[c0][r];
                u1 = (c0 + 1 <= r) ? sp[r][c0 + 1] : sp[c0 + 1][r];
                idx = (size_t)(i0 + r) * np + i0 + c0;
            } else {    // the mirror tile: row j0 + r, columns i0 + c0, i0 + c0 + 1
                u0 = sp[c0][r];
                u1 = sp[c0 + 1][r];
                idx = (size_t)(j0 + r) * np + i0 + c0;
            }
            *(uint32_t *)(op1 + idx) = __byte_perm(u0, u1, 0x5410);
            *(uint32_t *)(op2 + idx) = __byte_perm(u0, u1, 0x7632);
        }
        __syncthreads();
    }
    ff_add_ff(fw, fq);   // ||Y_0||_F^2
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
// Tr D per block; the response / adjoint output (SECOND) is the Y stream with its
// scale removed.  The layer kernels keep only the lower triangle and the diagonal
// of the FP32 masters current (the next layer reads nothing else), so the output
// is assembled from the lower 64 x 64 tiles: a tile below the diagonal is written
// to (ti, tj) from registers and, transposed through shared memory, to (tj, ti); a
// diagonal tile is completed from its lower half.  H is symmetric, so Tr[D H] is
// summed over the lower triangle with off-diagonal weight 2.  d.fin_blocks blocks
// per instance, as many as are resident at once.
template <bool SECOND>
__global__ void __launch_bounds__(AUX_THREADS, SECOND ? 2 : FIN_BLOCKS_PER_SM) k_finalize(InstDesc *inst, int mode) {
    __shared__ float sx[AT][AT + 1];
    __shared__ float sy[SECOND ? AT : 1][AT + 1];
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
    float ys = 0.0f;
    if (mode == MODE_RESPONSE) ys = (float)(1.0 / ctl->y_scale);
    if (mode == MODE_ADJOINT) ys = (float)(-1.0 / (ctl->y_scale * (ctl->eps_max - ctl->eps_min)));
    // Tr[D H]: each H_ij unpacked to an FP32 pair (h1 + 2^-24 h2), x * h1 split exactly
    // into product and error (FMA), all summed in a compensated FP32 pair.
    FF fe = {0.f, 0.f}, ftr = {0.f, 0.f};   // compensated FP32 pairs (FP64 is slow on this part)
    int bad_unused = 0;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, c0 = 2 * lane;
    const int nt = (n + AT - 1) / AT;
    const long long ntiles = (long long)nt * (nt + 1) / 2;
    const bool hvec = ((n & 1) == 0) && (((uintptr_t)H & 15) == 0);
    const bool ovec = ((n & 1) == 0) && (((uintptr_t)out & 7) == 0);
    const bool ovec1 = ((n & 1) == 0) && (((uintptr_t)out1 & 7) == 0);
    for (long long k = blockIdx.x; k < ntiles; k += d.fin_blocks) {
        int ti, tj;
        lower_tile(k, ti, tj);
        const int i0 = ti * AT, j0 = tj * AT;
        const bool dg = (ti == tj);
        float2 x[AT_RPW], yv[SECOND ? AT_RPW : 1];
        double h[AT_RPW][2];
#pragma unroll
        for (int q = 0; q < AT_RPW; ++q) {
            const int i = i0 + w + 8 * q;
            // rows below n lie inside the padded np x np masters
            x[q] = (i < n) ? *(const float2 *)(X + (size_t)i * np + j0 + c0) : make_float2(0.f, 0.f);
            if (SECOND) yv[q] = (i < n) ? *(const float2 *)(Y + (size_t)i * np + j0 + c0) : make_float2(0.f, 0.f);
            if (H) load_pair(H, n, hvec, i, j0 + c0, h[q][0], h[q][1]);
        }
#pragma unroll
        for (int q = 0; q < AT_RPW; ++q) {
            const int r = w + 8 * q, i = i0 + r;
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                const int c = c0 + e, j = j0 + c;
                float xv = e ? x[q].y : x[q].x;
                float yw = 0.0f;
                if (SECOND) yw = (e ? yv[q].y : yv[q].x) * ys;
                if (!(i < n && j < n && (!dg || c <= r))) {
                    xv = 0.0f;   // outside the matrix, or above the diagonal (stale)
                    yw = 0.0f;
                } else {
                    if (i == j) {
                        xv += xoff;  // true X_L = stored X_L + c_L I
                        ff_add(ftr, xv);
                    }
                    if (H) {
                        float h1, h2;
                        split_f64(h[q][e], h1, h2, bad_unused);
                        const float wgt = (i == j) ? 1.0f : 2.0f;
                        const float p = __fmul_rn(xv, h1);
                        const float perr = __fmaf_rn(xv, h1, -p);
                        ff_add(fe, __fmul_rn(wgt, p));
                        fe.c = __fadd_rn(fe.c, __fmul_rn(wgt, __fmaf_rn(xv, h2 * 0x1p-24f, perr)));
                    }
                }
                sx[r][c] = xv;
                if (SECOND) sy[r][c] = yw;
                if (e) {
                    x[q].y = xv;
                    if (SECOND) yv[q].y = yw;
                } else {
                    x[q].x = xv;
                    if (SECOND) yv[q].x = yw;
                }
            }
            if (!dg) {
                if (out) store_pair(out, n, ovec, i, j0 + c0, x[q].x, x[q].y);
                if (SECOND) store_pair(out1, n, ovec1, i, j0 + c0, yv[q].x, yv[q].y);
            }
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < AT_RPW; ++q) {
            const int r = w + 8 * q;
            if (dg) {  // the diagonal tile's upper half is its lower half transposed
                const int ca = c0, cb = c0 + 1;
                const float a = r >= ca ? sx[r][ca] : sx[ca][r], b = r >= cb ? sx[r][cb] : sx[cb][r];
                if (out) store_pair(out, n, ovec, i0 + r, i0 + c0, a, b);
                if (SECOND) {
                    const float a1 = r >= ca ? sy[r][ca] : sy[ca][r], b1 = r >= cb ? sy[r][cb] : sy[cb][r];
                    store_pair(out1, n, ovec1, i0 + r, i0 + c0, a1, b1);
                }
            } else {   // the mirror tile (tj, ti): row j0 + r, columns i0 + c0, i0 + c0 + 1
                if (out) store_pair(out, n, ovec, j0 + r, i0 + c0, sx[c0][r], sx[c0 + 1][r]);
                if (SECOND) store_pair(out1, n, ovec1, j0 + r, i0 + c0, sy[c0][r], sy[c0 + 1][r]);
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

// Streaming multiprocessors of the current device (0 if the query fails).
static int sm_count() {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                  cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return sms;
}

// Lower 64 x 64 tiles of an n x n matrix.
static long long lower_tiles(int n) {
    const long long nt = (n + AT - 1) / AT;
    return nt * (nt + 1) / 2;
}

// Blocks of a lower-triangle pass over up to `tiles` tiles: as many as are resident at once.
static int tile_grid(long long tiles) {
    const int sms = sm_count();
    const long long cap = (long long)(sms > 0 ? sms : 1) * AT_BLOCKS_PER_SM;
    return (int)std::max(1LL, std::min(tiles, cap));
}

cudaError_t launch_gershgorin(InstDesc *inst, int B, int max_n, bool user_bounds, cudaStream_t s) {
    (void)user_bounds;  // bounds are computed anyway: the same pass detects non-finite input
    k_gersh_tiles<<<dim3(tile_grid(lower_tiles(max_n)), B), AUX_THREADS, 0, s>>>(inst);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_gersh_rows<<<dim3((max_n + GR_ROWS - 1) / GR_ROWS, B), AUX_THREADS, 0, s>>>(inst);
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
    // Every instance must be covered by the same number of blocks it reports in
    // init_parts (at most init_blocks_for(max_np), the partial buffers' floor): the
    // grid-stride loops handle any np with these grids.
    const int ub = user_bounds ? 1 : 0;
    if (path == PATH_SIMT) {
        k_init_x<PATH_SIMT, SP2_FP16_SPLIT><<<dim3(init_blocks_for(max_np), B), AUX_THREADS, 0, s>>>(inst, ub);
        return cudaGetLastError();
    }
    const int g = std::min(init_blocks_for(max_np), tile_grid(lower_tiles(max_np)));
    if (precision == SP2_BF16_SPLIT) k_init_x_tc<SP2_BF16_SPLIT><<<dim3(g, B), AUX_THREADS, 0, s>>>(inst, ub);
    else k_init_x_tc<SP2_FP16_SPLIT><<<dim3(g, B), AUX_THREADS, 0, s>>>(inst, ub);
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

int finalize_blocks() {
    const int sms = sm_count();
    return std::min(FIN_BLOCKS_MAX, (sms > 0 ? sms : 1) * FIN_BLOCKS_PER_SM);
}

cudaError_t launch_finalize(InstDesc *inst, int B, int fin_blocks, int mode, cudaStream_t s) {
    dim3 grid(fin_blocks, B);
    if (mode == MODE_RESPONSE || mode == MODE_ADJOINT) k_finalize<true><<<grid, AUX_THREADS, 0, s>>>(inst, mode);
    else k_finalize<false><<<grid, AUX_THREADS, 0, s>>>(inst, mode);
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
