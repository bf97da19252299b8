// exact_kernel.cu -- FP64-accurate matrix products on the FP16 tensor cores.
//
// Used by the refinement layers of the chain (section "Deep-neural network
// electronic structure solver": a few last layers with X held in double
// precision purify the eigenvalues toward 0 and 1) and by the congruences of
// the non-orthogonal route (section "The density matrix").  The arithmetic is
// an error-free splitting into small-integer slices (see exact.h): each product
// of two FP16 slices is an integer matrix, the products of one level s + t are
// summed in one FP32 tensor-memory accumulator where the integer sum stays
// exact, and the levels are combined in 64-bit integer arithmetic.
//
// Kernel structure (CTA pairs, tile 256 x 128, UMMA M = 256, N = 128, K = 16):
//   warp 0     TMA producer: per K block, the stages of the current sub-pass,
//              each one A slice (this CTA's 128 rows) and / or one B slice (its
//              64 of the tile's 128 columns), into a ring of eight 24 KB stages.
//   warp 1     MMA issuer (even CTA): for every product (A slice s, B slice t)
//              four K = 16 instructions into the accumulator of level s + t.
//              Tensor memory holds four 128-column accumulators, levels 0..3.
//              With five or six slices, levels 0..3 are first folded into one
//              int64 per element (kept in the columns of accumulators 0 and 1)
//              and two more sub-passes accumulate levels 4 and 5 in
//              accumulators 2 and 3.
//   warps 2-9  epilogue: the exact integer product P per element, then
//              SP2 mode: Y_{n+1} = Y_n +- (P - I/4) in fixed point (lower
//                triangle), the slices of Y_{n+1} for the next layer (both
//                orientations), FP64 partials of Tr Y and ||Y||_F^2;
//              general modes: C = P 2^(e_i + e_j - ...) in FP64.
// Tiles are independent (no grid barrier); every wait has a time limit, after
// which the pair stops and the error word is set.  Teardown after an abort
// waits until every bulk copy either CTA issued has landed, by byte counts on
// the even CTA's barriers (not by time).
#include <cmath>
#include <mutex>

#include "device_common.cuh"
#include "exact.h"
#include "tc_ptx.cuh"

namespace sp2i {

namespace {

constexpr int XS_THREADS = 320;
constexpr int XS_EPI_WARPS = 8;
constexpr int XS_RING = 8;
constexpr uint32_t XS_A_BYTES = 128 * TC_BK * 2;   // 16 KB: this CTA's 128 rows of one K block
constexpr uint32_t XS_B_BYTES = 64 * TC_BK * 2;    // 8 KB: this CTA's 64 of the tile's 128 columns
constexpr uint32_t XS_STAGE_BYTES = XS_A_BYTES + XS_B_BYTES;
constexpr int XS_MAX_ST = 4;

// Schedule of one tile, fixed at compile time by the slice count S (so that the
// single MMA thread issues from registers, without table look-ups).  Sub-pass 0
// holds stages (A_s, B_s), s < min(S, 4), and issues every product of levels
// 0..3 into accumulator l = s + t.  With S >= 5 two more sub-passes (phase B)
// issue the products of levels 4 and 5 into accumulators 2 and 3:
//   sub-pass 1: stages (A2, B0), (A3, B1), (A4, B2) [, (A5, -)]
//   sub-pass 2: stages (A0, B3), (A1, B4) [, (A2, B5)]
// so that no K block needs more than four 24 KB stages.
struct Prod {
    int a, b, acc;   // stage holding the A slice, stage holding the B slice, accumulator
};
__host__ __device__ constexpr int sched_nst(int S, int sp) {
    return sp == 0 ? (S < 4 ? S : 4) : sp == 1 ? (S == 6 ? 4 : 3) : (S == 6 ? 3 : 2);
}
__host__ __device__ constexpr int sched_sa(int S, int sp, int st) {
    return sp == 0 ? st : sp == 1 ? 2 + st : st;
}
__host__ __device__ constexpr int sched_sb(int S, int sp, int st) {
    return sp == 0 ? st : sp == 1 ? (st < 3 ? st : -1) : 3 + st;
}
__host__ __device__ constexpr int sched_nprod(int S, int sp) {
    return sp == 0 ? (S >= 4 ? 10 : S == 3 ? 6 : 3) : sp == 1 ? (S == 6 ? 6 : 3) : (S == 6 ? 5 : 2);
}
__host__ __device__ constexpr Prod sched_prod(int S, int sp, int pr) {
    // sub-pass 0: (s, t) of level l in order l = 0, 1, 2, 3; stages hold slice s.
    constexpr int s0[10] = {0, 0, 1, 0, 1, 2, 0, 1, 2, 3}, t0[10] = {0, 1, 0, 2, 1, 0, 3, 2, 1, 0};
    constexpr int l0[10] = {0, 1, 1, 2, 2, 2, 3, 3, 3, 3};
    // sub-pass 1 (stages A2..A5 / B0..B2): (2,2) (3,1) (4,0) -> level 4; (3,2) (4,1) (5,0) -> level 5
    constexpr int a1[6] = {0, 1, 2, 1, 2, 3}, b1[6] = {2, 1, 0, 2, 1, 0}, c1[6] = {2, 2, 2, 3, 3, 3};
    // sub-pass 2 (stages A0..A2 / B3..B5): (0,4) (1,3) -> level 4; (0,5) (1,4) (2,3) -> level 5
    constexpr int a2[5] = {0, 1, 0, 1, 2}, b2[5] = {1, 0, 2, 1, 0}, c2[5] = {2, 2, 3, 3, 3};
    return sp == 0 ? Prod{s0[pr], t0[pr], l0[pr]} : sp == 1 ? Prod{a1[pr], b1[pr], c1[pr]} : Prod{a2[pr], b2[pr], c2[pr]};
}
// The first product into an accumulator within its phase starts it (accumulate = 0).
__host__ __device__ constexpr bool sched_first(int S, int sp, int pr) {
    if (sp == 2) return false;
    for (int q = 0; q < pr; ++q)
        if (sched_prod(S, sp, q).acc == sched_prod(S, sp, pr).acc) return false;
    return true;
}

struct XsParams {   // 64-byte aligned through its tensor maps
    CUtensorMap amap[XS_MAX_SLICES];   // A-side slices, box 64 (K) x 128 rows
    CUtensorMap bmap[XS_MAX_SLICES];   // B-side slices, box 64 (K) x 64 rows
    int mode, n, np, slices, beta, ntiles, nbj, unit;
    const int *ea, *eb;
    const long long *y_in;
    long long *y_out;
    uint16_t *next;
    const int *choice;
    double2 *part;
    double *c;
    long long *scratch;                // per CTA: the tile's products, 128 x 128 int64
    int *err;
    unsigned long long timeout_ns;
};

struct XsSmemTail {
    uint64_t full[XS_RING];
    uint64_t empty[XS_RING];
    uint64_t tfa, tea, tfb, teb, drain;
    uint32_t tmem_base;
    int abort;
    unsigned int issued;               // producer: stages issued (this CTA)
    unsigned int consumed;             // MMA (even CTA): stages whose copies it has waited for
    uint32_t slot_bytes[XS_RING];      // producer: bytes this CTA issued into each slot, latest use
    double red[XS_EPI_WARPS][2];
};

constexpr size_t XS_SMEM = 1024 + (size_t)XS_RING * XS_STAGE_BYTES + sizeof(XsSmemTail);
static_assert(XS_SMEM <= 232448, "shared memory of the exact-slice kernel");

__device__ __forceinline__ void tile_of(const XsParams &p, int g, int &bi, int &bj) {
    if (p.mode == XS_GEN) {
        bi = g / p.nbj;
        bj = g - bi * p.nbj;
        return;
    }
    // Upper-triangle tiles: row block bi (256 rows) holds column blocks 2 bi .. nbj - 1.
    int b = 0;
    for (;;) {
        const int cnt = p.nbj - 2 * b;
        if (g < cnt) {
            bi = b;
            bj = 2 * b + g;
            return;
        }
        g -= cnt;
        ++b;
    }
}

// Slices of a fixed-point value v (units of the last slice times 2^sh_last):
// a_0 = round(v / 2^sh0), then each remainder in steps of 2^beta.  Returns
// false when |a_0| exceeds 2048 (not exactly representable in FP16).
__device__ __forceinline__ bool make_slices(long long v, int slices, int beta, int sh0, uint16_t (&out)[XS_MAX_SLICES]) {
    bool ok = true;
    int sh = sh0;
#pragma unroll
    for (int s = 0; s < XS_MAX_SLICES; ++s) {
        if (s < slices) {
            const long long a = (v + (1ll << (sh - 1))) >> sh;   // sh >= 1: callers keep a bit below the last slice
            v -= a << sh;
            if (s == 0 && (a > 2048 || a < -2048)) ok = false;
            // |a| <= 2^11 for the leading slice, <= 2^beta after it: exact through int32 and FP16
            out[s] = __half_as_ushort(__int2half_rn((int)a));
            sh -= beta;
        } else {
            out[s] = 0;
        }
    }
    return ok;
}

__device__ __forceinline__ double pow2(int k) { return __longlong_as_double((long long)(k + 1023) << 52); }

__device__ __forceinline__ void set_abort(XsSmemTail &tl, uint32_t peer_abort_addr) {
    tl.abort = 1;
    asm volatile("st.shared::cluster.u32 [%0], %1;" ::"r"(peer_abort_addr), "r"(1) : "memory");
}

// Producer: one sub-pass of a tile, every K block's stages into the ring.
template <int S, int SP>
__device__ __forceinline__ bool produce_subpass(const XsParams &p, XsSmemTail &tl, uint8_t *stages, unsigned int &idx,
                                                int row_a, int row_b, bool leader, uint32_t lead_full0,
                                                uint32_t peer_abort, const volatile int *abort) {
    constexpr int NST = sched_nst(S, SP);
    const int nkb = p.np / TC_BK;
    for (int kb = 0; kb < nkb; ++kb) {
#pragma unroll
        for (int st = 0; st < NST; ++st) {
            const int sa = sched_sa(S, SP, st), sb = sched_sb(S, SP, st);
            const uint32_t slot = idx % XS_RING, ph = (idx / XS_RING) & 1u;
            if (!mbar_wait(&tl.empty[slot], ph ^ 1u, abort, p.timeout_ns, p.err)) {
                set_abort(tl, peer_abort);
                return false;
            }
            const uint32_t bytes = (sa >= 0 ? XS_A_BYTES : 0u) + (sb >= 0 ? XS_B_BYTES : 0u);
            tl.slot_bytes[slot] = bytes;
            // Both CTAs' bytes complete on the even CTA's barrier.
            if (leader) mbar_expect_tx(&tl.full[slot], 2 * bytes);
            uint8_t *dst = stages + (size_t)slot * XS_STAGE_BYTES;
            const uint32_t fb = lead_full0 + slot * 8u;
            if (sa >= 0) tma_load_2d_pair(dst, &p.amap[sa], kb * TC_BK, row_a, fb);
            if (sb >= 0) tma_load_2d_pair(dst + XS_A_BYTES, &p.bmap[sb], kb * TC_BK, row_b, fb);
            ++idx;
            *(volatile unsigned int *)&tl.issued = idx;
        }
        if (*abort) return false;
    }
    return true;
}

// MMA issuer: one sub-pass of a tile.  Every product is four K = 16 instructions
// (M = 256, N = 128) into the accumulator of its level.
template <int S, int SP>
__device__ __forceinline__ bool mma_subpass(const XsParams &p, XsSmemTail &tl, uint8_t *stages, unsigned int &idx,
                                            uint32_t tmem_base, const volatile int *abort) {
    constexpr int NST = sched_nst(S, SP), NP = sched_nprod(S, SP);
    const uint32_t idesc = idesc_f16_mn(0u, XS_TILE_M, XS_TILE_N);
    const int nkb = p.np / TC_BK;
    for (int kb = 0; kb < nkb; ++kb) {
        uint32_t sad[NST];
#pragma unroll
        for (int st = 0; st < NST; ++st) {
            const uint32_t j = idx + st, slot = j % XS_RING;
            if (!mbar_wait(&tl.full[slot], (j / XS_RING) & 1u, abort, p.timeout_ns, p.err)) return false;
            sad[st] = smem_u32(stages + (size_t)slot * XS_STAGE_BYTES);
        }
        tc_fence_after();
#pragma unroll
        for (int pr = 0; pr < NP; ++pr) {
            const Prod q = sched_prod(S, SP, pr);
            const bool first = sched_first(S, SP, pr);
            const uint32_t a = sad[q.a], b = sad[q.b] + XS_A_BYTES;
            const uint32_t d = tmem_base + (uint32_t)q.acc * XS_TILE_N;
#pragma unroll
            for (int k = 0; k < TC_BK / 16; ++k)
                umma_f16<2>(d, sdesc_sw128(a + k * 32), sdesc_sw128(b + k * 32), idesc,
                            (first && kb == 0 && k == 0) ? 0u : 1u);
        }
#pragma unroll
        for (int st = 0; st < NST; ++st) umma_commit<2>(&tl.empty[(idx + st) % XS_RING]);
        idx += NST;
        *(volatile unsigned int *)&tl.consumed = idx;
    }
    return true;
}

template <int S>
__global__ void __launch_bounds__(XS_THREADS, 1) k_exact_product(const __grid_constant__ XsParams p) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t *stages = smem;
    XsSmemTail &tl = *(XsSmemTail *)(smem + (size_t)XS_RING * XS_STAGE_BYTES);
    const volatile int *abort = &tl.abort;
    constexpr bool PHASE_B = (S >= 5);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t rank = cluster_rank();
    const bool leader = (rank == 0);
    const int cluster_id = blockIdx.x >> 1, nclusters = gridDim.x >> 1;

    if (threadIdx.x == 0) {
        for (int s = 0; s < XS_RING; ++s) {
            mbar_init(&tl.full[s], 1);
            mbar_init(&tl.empty[s], 1);
            tl.slot_bytes[s] = 0;
        }
        mbar_init(&tl.tfa, 1);
        mbar_init(&tl.tfb, 1);
        mbar_init(&tl.drain, 1);
        mbar_init(&tl.tea, XS_EPI_WARPS * 2);   // one arrival per epilogue warp of the pair
        mbar_init(&tl.teb, XS_EPI_WARPS * 2);
        tl.abort = 0;
        tl.issued = 0;
        tl.consumed = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tl.tmem_base)),
                     "r"(512)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
        tc_fence_before();
    }
    __syncthreads();
    cluster_sync_all();
    tc_fence_after();
    const uint32_t tmem_base = tl.tmem_base;
    const uint32_t lead_full0 = cluster_addr(&tl.full[0], 0);
    const uint32_t lead_tea = cluster_addr(&tl.tea, 0), lead_teb = cluster_addr(&tl.teb, 0);
    const uint32_t peer_abort = cluster_addr(&tl.abort, rank ^ 1u);

    if (warp == 0) {
        // ------------------------------ TMA producer ------------------------------
        if (lane == 0) {
            unsigned int idx = 0;
            for (int g = cluster_id; g < p.ntiles && !*abort; g += nclusters) {
                int bi, bj;
                tile_of(p, g, bi, bj);
                const int row_a = bi * XS_TILE_M + (int)rank * 128;
                const int row_b = bj * XS_TILE_N + (int)rank * 64;
                if (!produce_subpass<S, 0>(p, tl, stages, idx, row_a, row_b, leader, lead_full0, peer_abort, abort))
                    break;
                if constexpr (PHASE_B) {
                    if (!produce_subpass<S, 1>(p, tl, stages, idx, row_a, row_b, leader, lead_full0, peer_abort, abort))
                        break;
                    if (!produce_subpass<S, 2>(p, tl, stages, idx, row_a, row_b, leader, lead_full0, peer_abort, abort))
                        break;
                }
            }
        }
    } else if (warp == 1) {
        // ------------------------------- MMA issuer -------------------------------
        if (lane == 0 && leader) {
            unsigned int idx = 0;
            int it = 0;
            bool ok = true;
            for (int g = cluster_id; g < p.ntiles; g += nclusters, ++it) {
                if (!mbar_wait(&tl.teb, (uint32_t)(it & 1) ^ 1u, abort, p.timeout_ns, p.err)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                if (!mma_subpass<S, 0>(p, tl, stages, idx, tmem_base, abort)) {
                    ok = false;
                    break;
                }
                umma_commit<2>(&tl.tfa);
                if constexpr (PHASE_B) {
                    // Levels 0..3 complete: the epilogue folds them into int64 words in
                    // accumulators 0 and 1 and frees 2 and 3 for levels 4 and 5.
                    if (!mbar_wait(&tl.tea, (uint32_t)(it & 1), abort, p.timeout_ns, p.err)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    if (!mma_subpass<S, 1>(p, tl, stages, idx, tmem_base, abort) ||
                        !mma_subpass<S, 2>(p, tl, stages, idx, tmem_base, abort)) {
                        ok = false;
                        break;
                    }
                    umma_commit<2>(&tl.tfb);
                }
            }
            if (!ok) set_abort(tl, peer_abort);
            // Whatever was issued completes before tensor memory or the stages go away.
            umma_commit<2>(&tl.drain);
            const unsigned long long t0 = global_ns();
            while (!mbar_try_wait(&tl.drain, 0u) && global_ns() - t0 < p.timeout_ns) {
            }
        }
    } else {
        // -------------------------------- epilogue --------------------------------
        const int ew = warp - 2, quarter = warp & 3, half = ew >> 2;
        const uint32_t lane_base = tmem_base + ((uint32_t)(quarter * 32) << 16);
        const int beta = p.beta;
        // This CTA's product scratch: row (quarter * 32 + lane) of the tile, 128 int64.
        long long *scr = p.scratch + (size_t)blockIdx.x * (128 * XS_TILE_N) + (size_t)(quarter * 32 + lane) * XS_TILE_N;
        int it = 0;
        // Every epilogue warp walks every tile of its pair (no early exit), so the
        // named barrier below is reached the same number of times by all eight.
        for (int g = cluster_id; g < p.ntiles; g += nclusters, ++it) {
            int bi, bj;
            tile_of(p, g, bi, bj);
            int ok = 1;
            if (lane == 0) ok = mbar_wait(&tl.tfa, (uint32_t)(it & 1), abort, p.timeout_ns, p.err) ? 1 : 0;
            ok = __shfl_sync(0xffffffffu, ok, 0);
            tc_fence_after();
            const int rw0 = bi * XS_TILE_M + (int)rank * 128 + quarter * 32;   // first row of this warp
            const int r = rw0 + lane;
            // Chunks of 16 columns this warp finishes (the same test in both loops below).
            auto chunk_live = [&](int j) {
                const int cb = bj * XS_TILE_N + half * 64 + j * 16;
                return rw0 < p.np && cb < p.np && !(p.mode != XS_GEN && cb + 15 < rw0);
            };
            if constexpr (PHASE_B) {
                if (ok) {
                    // Fold levels 0..3 into one int64 per element (level-3 units).
#pragma unroll 1
                    for (int j = 0; j < 4; ++j) {
                        if (!chunk_live(j)) continue;
                        const uint32_t col = (uint32_t)(half * 64 + j * 16);
                        float t0[16], t1[16], t2[16], t3[16];
                        tmem_ld16(lane_base + 0 * XS_TILE_N + col, t0);
                        tmem_ld16(lane_base + 1 * XS_TILE_N + col, t1);
                        tmem_ld16(lane_base + 2 * XS_TILE_N + col, t2);
                        tmem_ld16(lane_base + 3 * XS_TILE_N + col, t3);
                        uint32_t lo[16], hi[16];
#pragma unroll
                        for (int e = 0; e < 16; ++e) {
                            long long v = __float2ll_rn(t0[e]);
                            v = (v << beta) + __float2ll_rn(t1[e]);
                            v = (v << beta) + __float2ll_rn(t2[e]);
                            v = (v << beta) + __float2ll_rn(t3[e]);
                            lo[e] = (uint32_t)(unsigned long long)v;
                            hi[e] = (uint32_t)((unsigned long long)v >> 32);
                        }
                        tmem_st16(lane_base + 0 * XS_TILE_N + col, lo);
                        tmem_st16(lane_base + 1 * XS_TILE_N + col, hi);
                    }
                    tmem_wait_st();
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive_cluster(lead_tea);
                if (lane == 0 && ok) ok = mbar_wait(&tl.tfb, (uint32_t)(it & 1), abort, p.timeout_ns, p.err) ? 1 : 0;
                ok = __shfl_sync(0xffffffffu, ok, 0);
                tc_fence_after();
            }
            // The exact integer products of this warp's chunks, from tensor memory to
            // the scratch; then tensor memory goes back to the MMA side at once, and
            // the stores below overlap the next tile's products.
            if (ok) {
#pragma unroll 1
                for (int j = 0; j < 4; ++j) {
                    if (!chunk_live(j)) continue;
                    const uint32_t col = (uint32_t)(half * 64 + j * 16);
                    long long P[16];
                    if constexpr (PHASE_B) {
                        float lo[16], hi[16], t4[16], t5[16];
                        tmem_ld16(lane_base + 0 * XS_TILE_N + col, lo);
                        tmem_ld16(lane_base + 1 * XS_TILE_N + col, hi);
                        tmem_ld16(lane_base + 2 * XS_TILE_N + col, t4);
                        if constexpr (S == 6) tmem_ld16(lane_base + 3 * XS_TILE_N + col, t5);
#pragma unroll
                        for (int e = 0; e < 16; ++e) {
                            long long v = (long long)(((unsigned long long)__float_as_uint(hi[e]) << 32) |
                                                      (unsigned long long)__float_as_uint(lo[e]));
                            v = (v << beta) + __float2ll_rn(t4[e]);
                            if constexpr (S == 6) v = (v << beta) + __float2ll_rn(t5[e]);
                            P[e] = v;
                        }
                    } else {
                        float t[16];
#pragma unroll
                        for (int e = 0; e < 16; ++e) P[e] = 0;
#pragma unroll
                        for (int l = 0; l < S; ++l) {
                            tmem_ld16(lane_base + (uint32_t)l * XS_TILE_N + col, t);
#pragma unroll
                            for (int e = 0; e < 16; ++e) P[e] = (P[e] << beta) + __float2ll_rn(t[e]);
                        }
                    }
                    longlong2 *dst = (longlong2 *)(scr + col);
#pragma unroll
                    for (int e = 0; e < 8; ++e) dst[e] = make_longlong2(P[2 * e], P[2 * e + 1]);
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive_cluster(lead_teb);

            double ft = 0.0, fq = 0.0;
            int flag = 0;
            if (ok) {
                const int sign = (p.mode == XS_SP2 && *p.choice == SP2_CHOICE_FLIP) ? -1 : 1;
                const size_t mat = (size_t)p.np * p.np;
#pragma unroll 1
                for (int j = 0; j < 4; ++j) {
                    if (!chunk_live(j)) continue;
                    const int cb = bj * XS_TILE_N + half * 64 + j * 16;   // first column of the chunk
                    const uint32_t col = (uint32_t)(half * 64 + j * 16);
                    long long P[16];
                    const longlong2 *src = (const longlong2 *)(scr + col);
#pragma unroll
                    for (int e = 0; e < 8; ++e) {
                        const longlong2 v = src[e];
                        P[2 * e] = v.x;
                        P[2 * e + 1] = v.y;
                    }
                    if (p.mode == XS_SP2) {
                        // Y_{n+1} = Y_n + sign (P - I/4): exact in the int64 fixed point.
                        const long long quarter_unit = 1ll << (p.unit - 2);
                        const int sh0 = p.unit - 12;
                        const double inv_unit = pow2(-p.unit);
                        long long yo[16];
#pragma unroll
                        for (int e = 0; e < 16; ++e) {
                            const int c = cb + e;
                            yo[e] = (r <= c && r < p.np && c < p.np) ? __ldcs(p.y_in + (size_t)c * p.np + r) : 0;
                        }
                        uint16_t direct[XS_MAX_SLICES][16];
#pragma unroll
                        for (int e = 0; e < 16; ++e) {
                            const int c = cb + e;
                            const bool own = (r <= c) && (r < p.np) && (c < p.np);
                            const bool dg = (r == c) && (r < p.n);
                            const long long d = P[e] - (dg ? quarter_unit : 0ll);
                            const long long yn = yo[e] + (sign > 0 ? d : -d);
                            uint16_t a[XS_MAX_SLICES];
                            if (!make_slices(yn, S, beta, sh0, a) && own) flag = 1;
#pragma unroll
                            for (int s = 0; s < XS_MAX_SLICES; ++s) direct[s][e] = a[s];
                            if (own) {
                                const size_t m = (size_t)c * p.np + r;   // mirror (c, r): consecutive r per lane
                                __stcs(p.y_out + m, yn);
#pragma unroll
                                for (int s = 0; s < S; ++s) __stcs(p.next + (size_t)s * mat + m, a[s]);
                                const double y = (double)yn * inv_unit;
                                if (r == c) {
                                    ft += y;
                                    fq = fma(y, y, fq);
                                } else {
                                    fq = fma(2.0 * y, y, fq);
                                }
                            }
                        }
                        // Direct (r, c) slices: 16 consecutive columns of this lane's row.
                        if (r < p.np) {
                            if (cb > r && cb + 15 < p.np) {
#pragma unroll
                                for (int s = 0; s < S; ++s) {
                                    uint32_t w[8];
#pragma unroll
                                    for (int q = 0; q < 8; ++q)
                                        w[q] = (uint32_t)direct[s][2 * q] | ((uint32_t)direct[s][2 * q + 1] << 16);
                                    uint4 *dst = (uint4 *)(p.next + (size_t)s * mat + (size_t)r * p.np + cb);
                                    __stcs(dst, make_uint4(w[0], w[1], w[2], w[3]));
                                    __stcs(dst + 1, make_uint4(w[4], w[5], w[6], w[7]));
                                }
                            } else {
#pragma unroll
                                for (int e = 0; e < 16; ++e) {
                                    const int c = cb + e;
                                    if (r < c && c < p.np)
#pragma unroll
                                        for (int s = 0; s < S; ++s)
                                            __stcs(p.next + (size_t)s * mat + (size_t)r * p.np + c, direct[s][e]);
                                }
                            }
                        }
                    } else {
                        // C_ij = P 2^(e_i + e_j - 22 - beta (S - 1)).
                        const int base = -22 - beta * (S - 1);
                        const int er = (r < p.n) ? p.ea[r] : 0;
#pragma unroll
                        for (int e = 0; e < 16; ++e) {
                            const int c = cb + e;
                            if (r >= p.n || c >= p.n) continue;
                            if (p.mode == XS_GEN_SYM && r > c) continue;
                            const double v = __ll2double_rn(P[e]) * pow2(er + p.eb[c] + base);
                            p.c[(size_t)r * p.n + c] = v;
                            if (p.mode == XS_GEN_SYM && r < c) p.c[(size_t)c * p.n + r] = v;
                        }
                    }
                }
            }
            if (__any_sync(0xffffffffu, flag) && lane == 0) set_error(p.err, SP2_ERR_NOT_CONVERGED);
            if (p.mode == XS_SP2) {
                for (int o = 16; o > 0; o >>= 1) {
                    ft += __shfl_down_sync(0xffffffffu, ft, o);
                    fq += __shfl_down_sync(0xffffffffu, fq, o);
                }
                if (lane == 0) {
                    tl.red[ew][0] = ft;
                    tl.red[ew][1] = fq;
                }
                asm volatile("bar.sync 1, %0;" ::"n"(XS_EPI_WARPS * 32) : "memory");
                if (ew == 0 && lane == 0) {
                    double2 s2 = make_double2(0.0, 0.0);
                    for (int k = 0; k < XS_EPI_WARPS; ++k) {
                        s2.x += tl.red[k][0];
                        s2.y += tl.red[k][1];
                    }
                    p.part[(size_t)g * 2 + rank] = s2;
                }
                asm volatile("bar.sync 1, %0;" ::"n"(XS_EPI_WARPS * 32) : "memory");
            }
        }
    }

    // -------------------------------- teardown --------------------------------
    __syncthreads();
    cluster_sync_all();   // both CTAs' producers have stopped issuing copies
    if (threadIdx.x == 0 && leader) {
        uint32_t peer_issued_addr = cluster_addr(&tl.issued, 1), peer_abort_addr = cluster_addr(&tl.abort, 1);
        unsigned int odd_issued;
        int odd_abort;
        asm volatile("ld.shared::cluster.u32 %0, [%1];" : "=r"(odd_issued) : "r"(peer_issued_addr) : "memory");
        asm volatile("ld.shared::cluster.u32 %0, [%1];" : "=r"(odd_abort) : "r"(peer_abort_addr) : "memory");
        const unsigned int own = tl.issued, done = tl.consumed;
        const unsigned int top = own > odd_issued ? own : odd_issued;
        if (tl.abort || odd_abort || top > done) {
            // Every stage index in [done, top) may still have copies in flight.  The
            // even CTA's full barrier of that slot counts both CTAs' bytes: arm it for
            // a copy only the odd CTA issued, retire the odd CTA's share when only this
            // CTA issued (both CTAs load the same pattern, so the shares are equal),
            // then wait, bounded, for the phase to complete.
            for (unsigned int i = done; i < top; ++i) {
                const uint32_t slot = i % XS_RING, ph = (i / XS_RING) & 1u;
                const uint32_t bytes = tl.slot_bytes[slot];
                if (i >= own) {
                    uint32_t ob_addr = cluster_addr(&tl.slot_bytes[slot], 1), ob;
                    asm volatile("ld.shared::cluster.u32 %0, [%1];" : "=r"(ob) : "r"(ob_addr) : "memory");
                    mbar_expect_tx(&tl.full[slot], ob);
                } else if (i >= odd_issued) {
                    asm volatile("mbarrier.complete_tx.relaxed.cta.shared::cta.b64 [%0], %1;" ::"r"(
                                     smem_u32(&tl.full[slot])),
                                 "r"(bytes)
                                 : "memory");
                }
                const unsigned long long t0 = global_ns();
                while (!mbar_try_wait(&tl.full[slot], ph) && global_ns() - t0 < p.timeout_ns) {
                }
            }
        }
    }
    __syncthreads();
    cluster_sync_all();   // neither CTA leaves while its peer may still signal it
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(512) : "memory");
    }
}

// ------------------------------- set-up kernels -------------------------------
constexpr int XT = 256;

// round(d 2^unit) for an FP32 value d, in integer arithmetic (d = m 2^(e - 150),
// m the 24-bit significand): exact shifts, rounding half away from zero below.
__device__ __forceinline__ long long fixed_of_float(float d, int unit) {
    const uint32_t bits = __float_as_uint(d);
    const int e = (int)((bits >> 23) & 0xFF);
    if (e == 0) return 0;   // |d| < 2^-126: far below the last unit
    const long long m = (long long)((bits & 0x7FFFFF) | 0x800000);
    const int sh = e - 150 + unit;
    long long f;
    if (sh >= 0) f = m << sh;   // |d| <= 1 and unit <= 60 keep this below 2^61
    else if (sh > -25) f = (m + (1ll << (-sh - 1))) >> (-sh);
    else f = 0;
    return (bits >> 31) ? -f : f;
}

// Y_0 = D - I/2 in fixed point, its slices, and per-row partials (Tr Y, ||Y||_F^2).
// Off the diagonal y = d is an FP32 value: its square goes into a compensated
// float pair; the n diagonal entries are summed in FP64.
__global__ void __launch_bounds__(XT) k_xs_init_sp2(const float *__restrict__ D, int n, int np, int slices, int beta,
                                                    int unit, long long *__restrict__ y, uint16_t *__restrict__ sl,
                                                    double2 *part, int *err) {
    const int r = blockIdx.x;
    const size_t mat = (size_t)np * np;
    const long long half_unit = 1ll << (unit - 1);
    double t = 0.0, qd = 0.0;
    FF q = {0.f, 0.f};
    int bad = 0;
    for (int c = threadIdx.x; c < np; c += XT) {
        const float d = (r < n && c < n) ? D[(size_t)r * n + c] : 0.0f;
        const bool dg = (r == c) && (r < n);
        const long long f = fixed_of_float(d, unit) - (dg ? half_unit : 0ll);
        uint16_t a[XS_MAX_SLICES];
        if (!make_slices(f, slices, beta, unit - 12, a)) bad = 1;
#pragma unroll
        for (int s = 0; s < XS_MAX_SLICES; ++s)
            if (s < slices) sl[(size_t)s * mat + (size_t)r * np + c] = a[s];
        if (c <= r) y[(size_t)r * np + c] = f;
        if (dg) {
            const double yv = (double)d - 0.5;
            t += yv;
            qd = fma(yv, yv, qd);
        } else {
            ff_add_sq(q, d, 1.0f);
        }
    }
    double qv = ff_value(q) + qd;
    __shared__ double st[XT / 32], sq[XT / 32];
    for (int o = 16; o > 0; o >>= 1) {
        t += __shfl_down_sync(0xffffffffu, t, o);
        qv += __shfl_down_sync(0xffffffffu, qv, o);
    }
    if ((threadIdx.x & 31) == 0) {
        st[threadIdx.x >> 5] = t;
        sq[threadIdx.x >> 5] = qv;
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) set_error(err, SP2_ERR_NOT_CONVERGED);
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int k = 0; k < XT / 32; ++k) {
            a += st[k];
            b += sq[k];
        }
        part[r] = make_double2(a, b);
    }
}

// One warp: fixed-order sum of the partials, the statistics of X = Y + I/2 and the sign.
__global__ void k_xs_decide(const double2 *part, int nparts, int n, double n_occ, int *choice, double *rec) {
    const int lane = threadIdx.x;
    double t = 0.0, q = 0.0;
    for (int k = lane; k < nparts; k += 32) {
        t += part[k].x;
        q += part[k].y;
    }
    for (int o = 16; o > 0; o >>= 1) {
        t += __shfl_down_sync(0xffffffffu, t, o);
        q += __shfl_down_sync(0xffffffffu, q, o);
    }
    if (lane == 0) {
        // Tr X = Tr Y + n/2 and ||X||_F^2 = ||Y||_F^2 + Tr Y + n/4 (X = Y + I/2 on the first n entries).
        const double tr = t + 0.5 * n, qq = q + t + 0.25 * n;
        rec[0] = tr;
        rec[1] = qq;
        rec[2] = tr - qq;
        *choice = layer_rule(tr, qq, n_occ);
    }
}

// D = Y 2^-unit + I/2 (FP64, n x n, ld n) from the lower triangle of Y, 32 x 32 tiles.
__global__ void k_xs_finish(const long long *__restrict__ y, int n, int np, int unit, double *__restrict__ D) {
    __shared__ double tile[32][33];
    const int tb = blockIdx.x, sb = blockIdx.y;   // lower tile (tb >= sb): rows tb*32.., cols sb*32..
    if (sb > tb) return;
    const double inv = pow2(-unit);
    const int tx = threadIdx.x, ty = threadIdx.y;   // 32 x 8
    for (int k = ty; k < 32; k += 8) {
        const int r = tb * 32 + k, c = sb * 32 + tx;
        double v = 0.0;
        if (r < n && c < n && c <= r) v = (double)y[(size_t)r * np + c] * inv + (r == c ? 0.5 : 0.0);
        tile[k][tx] = v;
        if (r < n && c < n && c <= r) D[(size_t)r * n + c] = v;
    }
    __syncthreads();
    for (int k = ty; k < 32; k += 8) {
        const int r = sb * 32 + k, c = tb * 32 + tx;   // upper element (r, c), r < c, from (c, r)
        if (r < n && c < n && r < c) D[(size_t)r * n + c] = tile[tx][k];
    }
}

// out = M^T (n x n FP64, ld n), 32 x 32 tiles.
__global__ void k_transpose64(const double *__restrict__ M, int n, double *__restrict__ out) {
    __shared__ double tile[32][33];
    const int bx = blockIdx.x * 32, by = blockIdx.y * 32, tx = threadIdx.x, ty = threadIdx.y;
    for (int k = ty; k < 32; k += 8) {
        const int r = by + k, c = bx + tx;
        if (r < n && c < n) tile[k][tx] = M[(size_t)r * n + c];
    }
    __syncthreads();
    for (int k = ty; k < 32; k += 8) {
        const int r = bx + k, c = by + tx;
        if (r < n && c < n) out[(size_t)r * n + c] = tile[tx][k];
    }
}

// One warp per row: exponent e with 2^e >= the row's 2-norm, then the slices of
// the fixed-point value round(x 2^(12 - e + beta (S - 1))) (one bit below the last
// slice, so that its rounding shift is 1); rows and columns beyond n are zero.
__global__ void k_xs_slice_rows(const double *__restrict__ M, int n, int np, int slices, int beta,
                                uint16_t *__restrict__ sl, int *__restrict__ exps, int *err) {
    const int row = blockIdx.x * (XT / 32) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (row >= np) return;
    const size_t mat = (size_t)np * np;
    int e = 0;
    if (row < n) {
        double ss = 0.0;
        for (int k = lane; k < n; k += 32) {
            const double x = M[(size_t)row * n + k];
            ss = fma(x, x, ss);
        }
        for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
        if (ss > 0.0) {
            int k2;
            frexp(sqrt(ss) * (1.0 + 0x1p-50), &k2);   // sqrt(ss) < 2^k2
            e = k2;
        }
    }
    if (lane == 0) exps[row] = e;
    const double sc = pow2(12 - e + beta * (slices - 1));
    int bad = 0;
    for (int k = lane; k < np; k += 32) {
        const double x = (row < n && k < n) ? M[(size_t)row * n + k] : 0.0;
        uint16_t a[XS_MAX_SLICES];
        if (!make_slices(__double2ll_rn(x * sc), slices, beta, beta * (slices - 1) + 1, a)) bad = 1;
#pragma unroll
        for (int s = 0; s < XS_MAX_SLICES; ++s)
            if (s < slices) sl[(size_t)s * mat + (size_t)row * np + k] = a[s];
    }
    if (__any_sync(0xffffffffu, bad) && lane == 0) set_error(err, SP2_ERR_NOT_CONVERGED);
}

// ------------------------------- host helpers -------------------------------
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encoder() {
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *q = nullptr;
        cudaDriverEntryPointQueryResult res;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &q, 12000, cudaEnableDefault, &res) ==
                cudaSuccess &&
            res == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)q;
    });
    return fn;
}

bool encode_slice_map(CUtensorMap *m, const uint16_t *base, int np, int box_rows) {
    EncodeTiledFn fn = encoder();
    if (!fn) return false;
    cuuint64_t dims[2] = {(cuuint64_t)np, (cuuint64_t)np};
    cuuint64_t strides[1] = {(cuuint64_t)np * 2};
    cuuint32_t box[2] = {(cuuint32_t)TC_BK, (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, const_cast<uint16_t *>(base), dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int S>
const void *product_kernel() {
    return (const void *)k_exact_product<S>;
}

const void *product_kernel_for(int S) {
    switch (S) {
        case 4: return product_kernel<4>();
        case 5: return product_kernel<5>();
        case 6: return product_kernel<6>();
        default: return nullptr;
    }
}

int grid_1d(size_t work, int per_block) {
    size_t g = (work + per_block - 1) / per_block;
    return g < 1 ? 1 : (int)g;
}

}  // namespace

bool xs_available() { return encoder() != nullptr; }

int xs_choose_beta(int slices, int K) {
    const double rho0 = 2048.0 + 0.5 * std::sqrt((double)K);
    for (int b = 7; b >= 3; --b) {
        const double rho = std::ldexp(1.0, b) * std::sqrt(K / 12.0);
        bool ok = true;
        const int top = slices - 1 < 4 ? slices - 1 : 4;   // level 5 may round: it is below 2^-50 of the product
        for (int l = 1; l <= top && ok; ++l) {
            // sum_{s+t=l} rho_s rho_t: two terms with slice 0, l - 1 with noise slices only
            const double bound = 2.0 * rho0 * rho + (l - 1) * rho * rho;
            if (bound > 16777216.0) ok = false;
        }
        if (ok) return b;
    }
    return 3;
}

int xs_tile_count(int np, int mode) {
    const int nbj = np / XS_TILE_N, nbi = (np + XS_TILE_M - 1) / XS_TILE_M;
    if (mode == XS_GEN) return nbi * nbj;
    int t = 0;
    for (int b = 0; b < nbi; ++b)
        if (nbj - 2 * b > 0) t += nbj - 2 * b;
    return t;
}

size_t xs_part_bytes(int np) {
    const size_t a = (size_t)xs_tile_count(np, XS_SP2) * 2, b = (size_t)np;
    return sizeof(double2) * (a > b ? a : b);
}

int xs_resident_pairs(int sm_count) {
    for (int S = 4; S <= XS_MAX_SLICES; ++S)
        if (cudaFuncSetAttribute(product_kernel_for(S), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)XS_SMEM) !=
            cudaSuccess) {
            cudaGetLastError();
            return 0;
        }
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(sm_count);
    cfg.blockDim = dim3(XS_THREADS);
    cfg.dynamicSmemBytes = XS_SMEM;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int nc = 0;
    if (cudaOccupancyMaxActiveClusters(&nc, product_kernel_for(XS_MAX_SLICES), &cfg) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return nc < sm_count / 2 ? nc : sm_count / 2;
}

size_t xs_scratch_bytes(int grid_pairs) { return (size_t)2 * grid_pairs * 128 * XS_TILE_N * sizeof(long long); }

cudaError_t xs_product(const XsProduct &q, int grid_pairs, cudaStream_t s) {
    const void *fn = product_kernel_for(q.slices);
    if (!fn || q.np % XS_TILE_N != 0 || grid_pairs < 1 || !q.scratch) return cudaErrorInvalidValue;
    XsParams p;
    memset(&p, 0, sizeof(p));
    for (int k = 0; k < q.slices; ++k) {
        const size_t off = (size_t)k * q.np * q.np;
        if (!encode_slice_map(&p.amap[k], q.a.base + off, q.np, 128) ||
            !encode_slice_map(&p.bmap[k], q.b.base + off, q.np, 64))
            return cudaErrorInvalidValue;
    }
    p.mode = q.mode;
    p.n = q.n;
    p.np = q.np;
    p.slices = q.slices;
    p.beta = q.beta;
    p.ntiles = xs_tile_count(q.np, q.mode);
    p.nbj = q.np / XS_TILE_N;
    p.unit = 24 + q.beta * (q.slices - 1);
    p.ea = q.a.exps;
    p.eb = q.b.exps;
    p.y_in = q.y_in;
    p.y_out = q.y_out;
    p.next = q.next_slices;
    p.choice = q.choice;
    p.part = q.part;
    p.c = q.c;
    p.scratch = q.scratch;
    p.err = q.err;
    p.timeout_ns = q.timeout_ns;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)XS_SMEM);
    if (e != cudaSuccess) return e;
    int pairs = grid_pairs;
    if (pairs > p.ntiles) pairs = p.ntiles;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(2 * pairs);
    cfg.blockDim = dim3(XS_THREADS);
    cfg.dynamicSmemBytes = XS_SMEM;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    void *args[] = {(void *)&p};
    return cudaLaunchKernelExC(&cfg, fn, args);
}

cudaError_t xs_init_sp2(const float *D, int n, int np, int slices, int beta, long long *y, uint16_t *sl,
                        double2 *part, int *nparts, int *err, cudaStream_t s) {
    k_xs_init_sp2<<<np, XT, 0, s>>>(D, n, np, slices, beta, 24 + beta * (slices - 1), y, sl, part, err);
    *nparts = np;
    return cudaGetLastError();
}

cudaError_t xs_decide(const double2 *part, int nparts, int n, double n_occ, int *choice, double *rec, cudaStream_t s) {
    k_xs_decide<<<1, 32, 0, s>>>(part, nparts, n, n_occ, choice, rec);
    return cudaGetLastError();
}

cudaError_t xs_finish_sp2(const long long *y, int n, int np, int slices, int beta, double *D, cudaStream_t s) {
    const int nb = (n + 31) / 32;
    k_xs_finish<<<dim3(nb, nb), dim3(32, 8), 0, s>>>(y, n, np, 24 + beta * (slices - 1), D);
    return cudaGetLastError();
}

cudaError_t xs_slice_rows(const double *M, bool transpose, int n, int np, int slices, int beta, XsOperand out,
                          double *scratch, int *err, cudaStream_t s) {
    const double *src = M;
    if (transpose) {
        const int nb = (n + 31) / 32;
        k_transpose64<<<dim3(nb, nb), dim3(32, 8), 0, s>>>(M, n, scratch);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        src = scratch;
    }
    k_xs_slice_rows<<<grid_1d((size_t)np, XT / 32), XT, 0, s>>>(src, n, np, slices, beta, out.base, out.exps, err);
    return cudaGetLastError();
}

}  // namespace sp2i
