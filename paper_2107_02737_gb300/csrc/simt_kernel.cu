// simt_kernel.cu -- the FP32 CUDA-core SP2 chain (the plain-precision comparator).
//
// One cooperative persistent launch runs every layer: per round each CTA takes
// upper-triangle 128 x 128 tiles (bi <= bj) of X_{n+1} = X_n^2 or 2 X_n - X_n^2
// (or the accelerated layer), computes the tile's product with FP32 FMAs on the
// centred operand X - I/2 (the B operand is rows of X because X is symmetric),
// writes the tile and its mirror, and records FP64 partials of
// Tr X_{n+1} and ||X_{n+1}||_F^2.  A grid barrier ends the round; every CTA then
// takes the same layer decision from the same partials (no host round trip).
#include "device_common.cuh"

namespace sp2i {

namespace {

constexpr int BK = 16;
constexpr int LDS = SIMT_T + 4;  // padded smem row (floats), keeps float4 alignment

struct SimtSmem {
    float A[2][BK][LDS];
    float B[2][BK][LDS];
    double red[SIMT_THREADS / 32][2];
};
static_assert(sizeof(float) * 2 * BK * LDS >= 4 * MAX_BATCH * sizeof(double) + 4 * (SIMT_THREADS / 32) * sizeof(double),
              "round sums reuse the A staging buffers");

// acc = Y^2 over the tile for the centred operand Y = X - I/2 (I on the n real
// diagonal entries): Y has the eigenvalues of X shifted into [-1/2, 1/2], so the
// FP32 sums run over smaller terms; the epilogue adds X - I/4 back.
__device__ __forceinline__ void simt_tile_mma(const float *__restrict__ X, int np, int n, int r0, int c0,
                                              SimtSmem &sm, float acc[8][8]) {
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    const int lrow = tid >> 1, lk = (tid & 1) * 8;
    const float *Ap = X + (size_t)(r0 + lrow) * np + lk;
    const float *Bp = X + (size_t)(c0 + lrow) * np + lk;
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = 0.0f;

    float4 ra0 = *(const float4 *)Ap, ra1 = *(const float4 *)(Ap + 4);
    float4 rb0 = *(const float4 *)Bp, rb1 = *(const float4 *)(Bp + 4);
    auto stash = [&](int buf, int kt) {
        const float a[8] = {ra0.x, ra0.y, ra0.z, ra0.w, ra1.x, ra1.y, ra1.z, ra1.w};
        const float b[8] = {rb0.x, rb0.y, rb0.z, rb0.w, rb1.x, rb1.y, rb1.z, rb1.w};
        const int k0 = kt * BK + lk;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int k = k0 + q;
            sm.A[buf][lk + q][lrow] = (k == r0 + lrow && k < n) ? a[q] - 0.5f : a[q];
            sm.B[buf][lk + q][lrow] = (k == c0 + lrow && k < n) ? b[q] - 0.5f : b[q];
        }
    };
    stash(0, 0);
    __syncthreads();
    const int nk = np / BK;
    for (int kt = 0; kt < nk; ++kt) {
        const int buf = kt & 1;
        if (kt + 1 < nk) {
            const float *a = Ap + (size_t)(kt + 1) * BK, *b = Bp + (size_t)(kt + 1) * BK;
            ra0 = *(const float4 *)a;
            ra1 = *(const float4 *)(a + 4);
            rb0 = *(const float4 *)b;
            rb1 = *(const float4 *)(b + 4);
        }
#pragma unroll
        for (int k = 0; k < BK; ++k) {
            const float4 a0 = *(const float4 *)&sm.A[buf][k][ty * 4];
            const float4 a1 = *(const float4 *)&sm.A[buf][k][64 + ty * 4];
            const float4 b0 = *(const float4 *)&sm.B[buf][k][tx * 4];
            const float4 b1 = *(const float4 *)&sm.B[buf][k][64 + tx * 4];
            const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            const float b[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
        }
        if (kt + 1 < nk) stash(buf ^ 1, kt + 1);
        __syncthreads();
    }
}

// SP2 update of one tile, mirror store and FP64 partials.
// X_{n+1} = k2 X^2 + k1 X + k0 I (I on the n real diagonal entries): the plain
// layer (1, 0, 0) or (-1, 2, 0); the accelerated one T^2 with T = aX + (1 - a) I,
// (a^2, 2a(1 - a), (1 - a)^2), or 2T - T^2 with T = aX, (-a^2, 2a, 0).  With
// X^2 = acc + X - I/4 (acc = Y^2 of the centred operands) this is
// k2 acc + (k2 + k1) X + (k0 - k2/4) I.
__device__ __forceinline__ void simt_tile_epilogue(const float *__restrict__ Xold, float *__restrict__ Xnew, int np,
                                                   int n, int r0, int c0, int flip, float alpha,
                                                   const float acc[8][8], FF &ft, FF &fq) {
    const int tid = threadIdx.x;
    const float k2 = flip ? -alpha * alpha : alpha * alpha;
    const float kx = alpha * (2.0f - alpha);
    const float kd = flip ? 0.25f * alpha * alpha : (1.0f - alpha) * (1.0f - alpha) - 0.25f * alpha * alpha;
    const int tx = tid & 15, ty = tid >> 4;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int r = r0 + (i < 4 ? ty * 4 + i : 64 + ty * 4 + (i - 4));
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int cb = c0 + (h == 0 ? tx * 4 : 64 + tx * 4);
            float v[4];
            const float4 xo = *(const float4 *)(Xold + (size_t)r * np + cb);
            const float xov[4] = {xo.x, xo.y, xo.z, xo.w};
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float s = acc[i][h * 4 + q];
                const bool dg = (r == cb + q) && (r < n);
                v[q] = fmaf(k2, s, fmaf(kx, xov[q], dg ? kd : 0.0f));
            }
            const bool all_owned = (r <= cb);
            if (all_owned) {
                *(float4 *)(Xnew + (size_t)r * np + cb) = make_float4(v[0], v[1], v[2], v[3]);
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int c = cb + q;
                if (r > c) continue;
                if (!all_owned) Xnew[(size_t)r * np + c] = v[q];
                if (r < c) {
                    Xnew[(size_t)c * np + r] = v[q];
                    ff_add_sq(fq, v[q], 2.0f);
                } else {
                    ff_add(ft, v[q]);
                    ff_add_sq(fq, v[q], 1.0f);
                }
            }
        }
    }
}

// Two CTAs per SM at 128 registers per thread (the comparator's throughput halves
// at one; a launch bound forcing it makes the kernel spill and costs 4 %).
__global__ void __launch_bounds__(SIMT_THREADS) k_simt_persistent(const __grid_constant__ RunParams p) {
    __shared__ RoundCtl rc;
    __shared__ __align__(16) SimtSmem sm;
    if (threadIdx.x == 0) round_ctl_init(rc, p);
    __syncthreads();
    unsigned int target = 0;
    bool first = true;
    while (true) {
        if (!first) {
            __syncthreads();
            if (threadIdx.x == 0) {
                const bool withhold = (p.test_hook == 1 && blockIdx.x == 0 && target == 0);
                target += gridDim.x;
                if (!grid_barrier(p.barrier, target, p.err, p.timeout_ns, withhold)) rc.abort = 1;
            }
            __syncthreads();
            if (rc.abort) break;
        }
        first = false;
        // The operand staging buffers are idle here: use them for the sums.
        double *sums = (double *)&sm.A[0][0][0];
        reduce_round_partials_block(rc, p, sums, sums + 4 * MAX_BATCH);
        if (threadIdx.x == 0) decide_round(rc, p, sums);
        __syncthreads();
        if (rc.abort || rc.total == 0) break;
        for (int g = blockIdx.x; g < rc.total; g += gridDim.x) {
            int i, job, tile;
            map_tile(rc, p.B, p.inst, g, i, job, tile);
            const InstDesc &d = p.inst[i];
            const int2 bt = p.tiles[d.tile_off + tile];
            const int n = rc.layer[i];
            const float *X = d.xf[n & 1];
            float *Xn = d.xf[(n + 1) & 1];
            float acc[8][8];
            simt_tile_mma(X, d.np, d.n, bt.x * SIMT_T, bt.y * SIMT_T, sm, acc);
            FF ft = {0.f, 0.f}, fq = {0.f, 0.f};
            simt_tile_epilogue(X, Xn, d.np, d.n, bt.x * SIMT_T, bt.y * SIMT_T, rc.choice[i] == SP2_CHOICE_FLIP,
                               rc.alpha[i], acc, ft, fq);
            // Deterministic block reduction of the tile partials.
            double t = ff_value(ft), q = ff_value(fq);
            for (int o = 16; o > 0; o >>= 1) {
                t += __shfl_down_sync(0xffffffffu, t, o);
                q += __shfl_down_sync(0xffffffffu, q, o);
            }
            if ((threadIdx.x & 31) == 0) {
                sm.red[threadIdx.x >> 5][0] = t;
                sm.red[threadIdx.x >> 5][1] = q;
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                Part s;
                s.t = s.q = s.w = s.p = 0.0;
                for (int w = 0; w < SIMT_THREADS / 32; ++w) {
                    s.t += sm.red[w][0];
                    s.q += sm.red[w][1];
                }
                d.part[(n + 1) % 3][tile] = s;
            }
            __syncthreads();
        }
    }
}

}  // namespace

int simt_blocks_per_sm() {
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_simt_persistent, SIMT_THREADS, 0) != cudaSuccess) return 0;
    return b;
}

cudaError_t launch_simt_persistent(const RunParams &p, int grid, cudaStream_t s) {
    void *args[] = {(void *)&p};
    // Cooperative launch in the attribute form (also capturable in a CUDA graph).
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(SIMT_THREADS);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelExC(&cfg, (const void *)k_simt_persistent, args);
}

}  // namespace sp2i
