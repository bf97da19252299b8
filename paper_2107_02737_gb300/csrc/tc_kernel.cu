// tc_kernel.cu -- split-precision SP2 chain on the 5th-generation tensor cores.
//
// The activation f(X) = X^2 of every layer (Eq. activ) is evaluated from the
// dual 16-bit representation X = X^(0) + X^(1) as X^(0)X^(0) + X^(0)X^(1) +
// X^(1)X^(0) (the paper's A + B + B^T; the X^(1)X^(1) term is dropped), all
// three products accumulated in one FP32 accumulator in tensor memory:
//   S[i,j] = sum_k hi[i,k] lo[j,k] + lo[i,k] hi[j,k] + hi[i,k] hi[j,k]
// (rows of X; X is symmetric), all three issued from the same staged K block.
// FP16 stores both parts times 2^11 (so lo stays in FP16's normal range): every
// product carries 2^22, removed in the epilogue.  BF16 needs no scaling.
//
// Centred operands and accumulator-bias removal: the FP32 accumulator of the
// tensor cores truncates once per MMA instruction, a relative bias of order
// (K/16) 2^-24 that would make the chain converge to (1 + beta) times the
// projector.  The operands are therefore the split of Y = X - I/2 (near
// convergence Y^2 ~ I/4, so the product error is mostly a multiple of the
// identity), the square is rebuilt as X^2 = Y^2 + X - I/4, and the identity
// component of the error is measured exactly from Tr(Y^2) = ||Y||_F^2 (both
// reduced in FP64) and carried to the next layer as a scalar offset c
// (true X = stored X + c I).
//
// Kernel structure (one persistent launch for the whole chain: cooperative for
// single-CTA tiles, a cluster launch sized to the resident pairs for CTA pairs):
//   warp 0      TMA producer: 2-D tiled bulk copies (128B swizzle) into a ring of
//               stages of one A block (this CTA's rows) and one B block; a square
//               tile takes each K block in two stages, (hi, hi) and (lo, lo), a
//               response tile in four, (X hi, Y hi), (X lo, Y lo), (Y hi, X hi),
//               (Y lo, X lo).  The tensor cores' FP32 accumulator truncates once per
//               MMA instruction; the small cross products of each K block are issued
//               before its hi x hi product.
//   warp 1      tcgen05.mma issuer (one thread): M=128, N=256, K=16 per
//               instruction, FP32 accumulator in TMEM, double-buffered (2 x 256
//               columns) so the epilogue of tile t overlaps the MMAs of t+1.
//   warps 2..9  epilogue, two warps per SM sub-partition (the epilogue is bound by
//               instruction latency, so a second warp hides it): warp w reads TMEM
//               lanes 32 (w mod 4) .. +31 and the tile's column half (w - 2) / 4, in
//               16-column chunks; X_{n+1} = S or 2 X_n - S, FP32 master + split
//               operands written for the tile and its mirror (only tiles with rows <=
//               columns are computed; the direct orientation of a chunk above the
//               diagonal leaves as two TMA tensor stores), compensated partials of
//               Tr X and ||X||_F^2 (FP32 pairs, one FP64 record per tile and CTA).
// Between layers, two schedules.  A single density solve runs without a grid
// barrier (dataflow): each tile of layer n + 1 starts its K blocks once the tiles
// of layer n that wrote them have completed, and the epilogue warps alone wait for
// the whole layer to take its decision.  Batches, responses and adjoints run in
// rounds ended by a grid barrier, after which every CTA takes the same decisions.
// The response / adjoint stream reuses the same machinery with six products per K
// block: (C + C^T)[i,j] = sum_k X[i,k] Y[j,k] + Y[i,k] X[j,k] for symmetric X and Y.
#include "device_common.cuh"
#include "tc_ptx.cuh"

namespace sp2i {

namespace {

// Tile configuration.  CG = 1: one CTA computes a 128 x 256 tile (M = 128 MMAs).
// CG = 2: a cluster of two CTAs computes a 256 x 256 tile with M = 256 MMAs
// issued by the even CTA; each CTA loads its own 128 rows of A and 128 of the
// 256 B rows, so a stage is 32 KB per CTA and six stages fit.
template <int CG>
struct Cfg {
    static constexpr int STAGES = (CG == 2) ? 6 : 4;
    static constexpr uint32_t A_BYTES = 128 * TC_BK * 2;                   // 16 KB: own 128 rows
    static constexpr uint32_t B_BYTES = (CG == 2 ? 128 : 256) * TC_BK * 2;  // own B rows
    static constexpr uint32_t STAGE_BYTES = A_BYTES + B_BYTES;
    static constexpr uint32_t TX_BYTES = STAGE_BYTES * CG;               // bytes per stage over the pair
    static constexpr int TILE_M = 128 * CG;                              // output rows per tile
};
constexpr int MAX_STAGES = 6;
constexpr int EPI_WARPS = 8;                              // warps 2..9
constexpr int EPI_CHUNK = 16;                             // accumulator columns per epilogue step
// Per epilogue warp: the transpose buffer of a chunk (32 x (EPI_CHUNK + 1) words) or
// the chunk's hi and lo boxes for the tensor stores, 128-byte aligned.
constexpr uint32_t EPI_T_FLOATS = 576;
static_assert(EPI_CHUNK == EPI_BOX_COLS && EPI_BOX_ROWS == 32, "store box = one warp's chunk");
static_assert(EPI_T_FLOATS >= 32 * (EPI_CHUNK + 1) && EPI_T_FLOATS * 4 >= 2 * EPI_BOX_ROWS * EPI_BOX_COLS * 2 &&
                  (EPI_T_FLOATS * 4) % 128 == 0,
              "epilogue buffer");
constexpr uint32_t TMEM_COLS = 512;                       // two 128 x 256 FP32 accumulators

struct TcSmemTail {
    uint64_t full[MAX_STAGES];
    uint64_t empty[MAX_STAGES];
    uint64_t tfull[2];
    uint64_t tempty[2];
    uint64_t drain;                  // MMA completion, waited for when the launch aborts
    uint32_t tmem_base;
    uint32_t pad;
    unsigned int issued;             // producer: ring stages this CTA has loaded into
    unsigned int consumed;           // MMA thread (even CTA): stages whose copies it has waited for
    FF red[EPI_WARPS][4];            // per epilogue warp: the tile's four partials (compensated pairs)
    double flow_sums[4];             // dataflow: the previous layer's sums
    RoundCtl rc;
};

constexpr size_t STAGE_AREA = 196608;  // 4 x 48 KB or 6 x 32 KB
static_assert(Cfg<1>::STAGES * Cfg<1>::STAGE_BYTES <= STAGE_AREA, "stage area");
static_assert(Cfg<2>::STAGES * Cfg<2>::STAGE_BYTES <= STAGE_AREA, "stage area");
static_assert(EPI_WARPS * EPI_T_FLOATS * 4 >= 4 * MAX_BATCH * sizeof(double) + MAX_BATCH * sizeof(int),
              "round sums and decisions reuse the epilogue transpose buffers");
constexpr size_t SMEM_BYTES = 1024 /*alignment slack*/ + STAGE_AREA + (size_t)EPI_WARPS * EPI_T_FLOATS * 4 +
                              sizeof(TcSmemTail);

// Instruction descriptor, kind::f16: FP32 accumulator, A and B of one 16-bit
// type (0 = FP16, 1 = BF16), both K-major, N = 256, M = 128 * CG.
__host__ __device__ constexpr uint32_t idesc_f16(uint32_t ab, int m) { return idesc_f16_mn(ab, m, TC_BN); }

// ---------------------------------------------------------------------------
// Work description of one tile, identical for the three roles.
// ---------------------------------------------------------------------------
struct TileWork {
    int inst, job, tile, bi, bj;
    int resp;            // 0: square of X (three products per K block), 1: C + C^T of X and Y (six)
    int xslot;           // X operand slot
    int ybuf;            // Y input buffer (resp)
    int flip;            // layer choice is 2X - X^2
    int n;               // forward layer index of the input (square jobs)
    int rec;             // square job recomputing a forward layer in the adjoint's reverse sweep
    float cf;            // offset c of the input X: true X = stored X + c I
    float alpha;         // expansion a of the layer (1 = plain)
};

// Stop this CTA's roles, and for a CTA pair its peer's (so that neither waits for
// signals the other will no longer send).
template <int CG>
__device__ __forceinline__ void tc_abort(RoundCtl &rc, uint32_t peer_abort) {
    rc.abort = 1;
    if (CG == 2) asm volatile("st.shared::cluster.u32 [%0], %1;" ::"r"(peer_abort), "r"(1) : "memory");
}

__device__ __forceinline__ TileWork describe(const RoundCtl &rc, const RunParams &p, int g) {
    TileWork w;
    map_tile(rc, p.B, p.inst, g, w.inst, w.job, w.tile);
    const InstDesc &d = p.inst[w.inst];
    const int2 bt = p.tiles[d.tile_off + w.tile];
    w.bi = bt.x;
    w.bj = bt.y;
    w.rec = 0;
    if (rc.phase == 1 && rc.rec_mode) {  // adjoint reverse, checkpointing: X_{n+1} again from X_n
        const int n = rc.rec_top;
        w.resp = 0;
        w.rec = 1;
        w.xslot = xslot_of(d, n);
        w.ybuf = 0;
        w.flip = rc.chist[n + 1] == SP2_CHOICE_FLIP;
        w.n = n;
        w.cf = (float)rc.chist_c[n];
        w.alpha = rc.chist_a[n + 1];
    } else if (rc.phase == 1) {  // adjoint reverse: G_m from G_{m+1} and X_m
        const int k = rc.layer[0];
        const int m = rc.rev_total - 1 - k;
        w.resp = 1;
        w.xslot = xslot_of(d, m);
        w.ybuf = k & 1;
        w.flip = rc.chist[m + 1] == SP2_CHOICE_FLIP;
        w.n = m;
        w.cf = (float)rc.chist_c[m];
        w.alpha = rc.chist_a[m + 1];
    } else {
        const int n = rc.layer[w.inst];
        w.resp = w.job;
        w.xslot = xslot_of(d, n);
        w.ybuf = n & 1;
        w.flip = rc.choice[w.inst] == SP2_CHOICE_FLIP;
        w.n = n;
        w.cf = (float)rc.coff[w.inst];
        w.alpha = rc.alpha[w.inst];
    }
    return w;
}

// Dataflow schedule: tile g of layer r for the producer and the MMA thread (the
// layer's sign and offset are not needed there).
__device__ __forceinline__ TileWork describe_flow(const RunParams &p, int g, int r) {
    TileWork w;
    const InstDesc &d = p.inst[0];
    const int2 bt = p.tiles[d.tile_off + g];
    w.inst = 0;
    w.job = 0;
    w.tile = g;
    w.bi = bt.x;
    w.bj = bt.y;
    w.resp = 0;
    w.xslot = xslot_of(d, r);
    w.ybuf = 0;
    w.flip = 0;
    w.n = r;
    w.rec = 0;
    w.cf = 0.0f;
    w.alpha = 1.0f;
    return w;
}

// Dataflow schedule, producer.  A 256-column block kt of the operand row blocks pa
// and pb of X_n was written by at most four tiles of the previous layer, each done
// when its counter reaches `target` (CG completions per layer).  The counters are
// read with relaxed loads one block ahead (flow_peek), so their latency hides under
// the current block's copies, and re-polled only while a tile is still running;
// one acquire fence then orders the TMA reads after the tiles' stores.
__device__ __forceinline__ unsigned int ld_relaxed(const unsigned int *p) {
    unsigned int v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void flow_peek(const RunParams &p, int pa, int pb, int kt, unsigned int (&v)[4]) {
    const int *e0 = p.blk_src + (pa * p.nblk + kt) * 2, *e1 = p.blk_src + (pb * p.nblk + kt) * 2;
    const int src[4] = {e0[0], e0[1], e1[0], e1[1]};
#pragma unroll
    for (int k = 0; k < 4; ++k) v[k] = src[k] < 0 ? 0xFFFFFFFFu : ld_relaxed(p.tile_done + src[k]);
}
__device__ __noinline__ bool flow_wait(const RunParams &p, int pa, int pb, int kt, unsigned int target,
                                       unsigned int (&v)[4], const volatile int *abort) {
    const int *e0 = p.blk_src + (pa * p.nblk + kt) * 2, *e1 = p.blk_src + (pb * p.nblk + kt) * 2;
    const int src[4] = {e0[0], e0[1], e1[0], e1[1]};
    const unsigned long long t0 = global_ns();
    for (int k = 0; k < 4; ++k) {
        while (v[k] < target) {
            if (*abort || ld_volatile(p.err) != 0) return false;
            if (global_ns() - t0 > p.timeout_ns) {
                set_error(p.err, SP2_ERR_TIMEOUT);
                return false;
            }
            __nanosleep(32);
            v[k] = ld_relaxed(p.tile_done + src[k]);
        }
    }
    // The tiles' generic-proxy stores, released with their counters, reach the TMA reads.
    asm volatile("fence.acq_rel.gpu;" ::: "memory");
    asm volatile("fence.proxy.async.global;" ::: "memory");
    return true;
}

// Dataflow schedule, the eight epilogue warps: wait for every CTA-tile of layer r - 1
// (`per_layer` completions each), then the same sums in the same order as the
// barrier schedule (one warp) and the same decision for instance 0.  Returns false
// when the chain stopped or the launch is stopping.  `sums` is four doubles of
// shared memory.
__device__ __noinline__ bool flow_decide(RoundCtl &rc, const RunParams &p, double *sums, int r, int ew, int lane,
                                         unsigned int per_layer, const volatile int *abort) {
    if (ew == 0 && lane == 0) {
        int go = 1;
        if (r > 0) {
            const unsigned int target = per_layer * (unsigned int)r;
            const unsigned long long t0 = global_ns();
            while (ld_acquire(p.layer_done) < target) {
                if (*abort || ld_volatile(p.err) != 0) {
                    go = 0;
                    break;
                }
                if (global_ns() - t0 > p.timeout_ns) {
                    set_error(p.err, SP2_ERR_TIMEOUT);
                    go = 0;
                    break;
                }
                __nanosleep(64);
            }
        }
        if (ld_volatile(p.err) != 0) go = 0;
        rc.flow_go = go;
    }
    asm volatile("bar.sync 1, %0;" ::"n"(EPI_WARPS * 32) : "memory");
    if (!rc.flow_go) return false;
    if (ew == 0) {
        double a[4];
        sum_instance_partials(rc, p, 0, lane, a);
        if (lane == 0)
            for (int c = 0; c < 4; ++c) sums[c] = a[c];
    }
    asm volatile("bar.sync 1, %0;" ::"n"(EPI_WARPS * 32) : "memory");
    if (ew == 0 && lane == 0) {
        const int width = decide_instance(rc, p, sums, 0, blockIdx.x == 0);
        rc.prefix[0] = 0;
        rc.prefix[1] = width;
        rc.total = width;
    }
    asm volatile("bar.sync 1, %0;" ::"n"(EPI_WARPS * 32) : "memory");
    return rc.total > 0;
}

// Element jj of a lane's chunk row into the packed column pairs of its hi and lo boxes.
__device__ __forceinline__ void pack_pair(uint32_t (&hp)[EPI_CHUNK / 2], uint32_t (&lp)[EPI_CHUNK / 2], int jj,
                                          uint16_t a1, uint16_t a2) {
    if (jj & 1) {
        hp[jj >> 1] |= (uint32_t)a1 << 16;
        lp[jj >> 1] |= (uint32_t)a2 << 16;
    } else {
        hp[jj >> 1] = a1;
        lp[jj >> 1] = a2;
    }
}

template <int PREC, int CG>
__global__ void __launch_bounds__(TC_THREADS, 1) k_tc_persistent(const __grid_constant__ RunParams p) {
    using C = Cfg<CG>;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t *stages = smem;
    float *epi_T = (float *)(smem + STAGE_AREA);
    TcSmemTail &tl = *(TcSmemTail *)(epi_T + EPI_WARPS * EPI_T_FLOATS);
    RoundCtl &rc = tl.rc;
    const volatile int *abort = &rc.abort;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t rank = (CG == 2) ? cluster_rank() : 0u;   // position in the CTA pair
    const bool leader = (rank == 0);
    const int cluster_id = blockIdx.x / CG, nclusters = gridDim.x / CG;

    if (threadIdx.x == 0) {
        for (int s = 0; s < C::STAGES; ++s) {
            mbar_init(&tl.full[s], 1);
            mbar_init(&tl.empty[s], 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(&tl.tfull[a], 1);
            mbar_init(&tl.tempty[a], EPI_WARPS * CG);  // one arrival per epilogue warp of the pair
        }
        mbar_init(&tl.drain, 1);
        tl.issued = 0;
        tl.consumed = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        round_ctl_init(rc, p);
    }
    if (warp == 1) {
        if (CG == 2) {
            asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                             smem_u32(&tl.tmem_base)),
                         "r"(TMEM_COLS)
                         : "memory");
            asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
        } else {
            asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                             smem_u32(&tl.tmem_base)),
                         "r"(TMEM_COLS)
                         : "memory");
            asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
        }
        tc_fence_before();
    }
    __syncthreads();
    if (CG == 2) cluster_sync_all();  // both CTAs' barriers exist before any cross-CTA signal
    tc_fence_after();
    const uint32_t tmem_base = tl.tmem_base;

    // Cluster addresses of the even CTA's barriers (the pair's MMA side) and of the
    // peer's abort flag.
    uint32_t lead_full0 = 0, lead_tempty0 = 0, peer_abort = 0;
    if (CG == 2) {
        lead_full0 = cluster_addr(&tl.full[0], 0);
        lead_tempty0 = cluster_addr(&tl.tempty[0], 0);
        peer_abort = cluster_addr(&rc.abort, rank ^ 1u);
    }

    // Pipeline state, private to each role and carried across tiles and rounds.
    uint32_t stage = 0, phase = 0;      // producer / MMA ring
    uint32_t acc = 0, acc_phase = 0;    // MMA / epilogue accumulators
    int pend[MAX_STAGES];               // producer: parity + 1 of a load not yet released
    for (int s = 0; s < MAX_STAGES; ++s) pend[s] = 0;
    unsigned int issued = 0, consumed = 0;   // producer / MMA thread: ring stages so far
    const uint32_t idesc = idesc_f16(PREC == SP2_BF16_SPLIT ? 1u : 0u, C::TILE_M);

    // ---------- per-tile work of the three roles (both schedules below) ----------
    // Producer: every K block of tile w into the ring.  In the dataflow schedule a
    // 256-column block of X_n is loaded only once the tiles of the previous layer
    // that wrote it (and its mirror) have completed.
    int df_round = -1;   // dataflow: layer whose inputs are known to be complete everywhere
    auto produce_tile = [&](const TileWork &w) {
        // Dataflow: the column block checked last, the one peeked ahead and its counters.
        int df_kt = -1, df_next = -1;
        unsigned int df_v[4] = {0u, 0u, 0u, 0u};
        bool df_ready = !p.dataflow || w.n == 0 || df_round == w.n;
        if (!df_ready) {
            if (ld_relaxed(p.layer_done) >= (unsigned int)(CG * p.inst[0].ntiles * w.n)) {
                df_round = w.n;   // every tile of the previous layer is done
                df_ready = true;
            } else {
                // Or every tile that wrote this tile's two operand row blocks is: one pass
                // of relaxed loads (all in flight together), no per-block checks then.
                const int pa = (w.bi * C::TILE_M + (int)rank * 128) / 256, pb = w.bj;
                const int nb = (p.inst[0].np + 255) / 256;
                unsigned int mn = 0xFFFFFFFFu;
                for (int kt = 0; kt < nb; ++kt) {
                    unsigned int v[4];
                    flow_peek(p, pa, pb, kt, v);
                    mn = min(mn, min(min(v[0], v[1]), min(v[2], v[3])));
                }
                df_ready = mn >= (unsigned int)(CG * w.n);
            }
            if (df_ready) {
                asm volatile("fence.acq_rel.gpu;" ::: "memory");
                asm volatile("fence.proxy.async.global;" ::: "memory");
            }
        }
        const InstDesc &d = p.inst[w.inst];
        const int nkb = d.np / TC_BK;
        // Successive waves of tiles walk K in opposite directions, so that a
        // wave starts on the K blocks the previous one left in L2.
        const bool kdown = ((w.tile / d.kwave) & 1) != 0;
        const int row_a = w.bi * C::TILE_M + (int)rank * 128;
        const int row_b = w.bj * TC_BN + (CG == 2 ? (int)rank * 128 : 0);
        // Square tiles: each K block in two consecutive ring slots, (hi, hi) then
        // (lo, lo), which feed all three products.  Response tiles: the six
        // segments one after another, one K block per slot.
        const int nslot = (w.resp ? 4 : 2) * nkb;
        const CUtensorMap *X3 = d.xmap + w.xslot * MAPS_PER_SLOT;   // maps hi, hi, lo
        for (int kb = 0; kb < nslot; ++kb) {
            int kx;
            const CUtensorMap *am, *bm;
            if (w.resp) {
                // Response / adjoint tiles: per K block (X hi, Y hi), (X lo, Y lo),
                // (Y hi, X hi), (Y lo, X lo) -- rows bi on the A side, rows bj on the B
                // side -- feeding X Y^T and Y X^T.
                const CUtensorMap *Y3 = d.ymap + w.ybuf * MAPS_PER_SLOT;
                const int q = kb & 3;
                kx = (kdown ? nkb - 1 - (kb >> 2) : (kb >> 2)) * TC_BK;
                const CUtensorMap *xm = (q & 1) ? X3 + 2 : X3 + 1, *ym = (q & 1) ? Y3 + 2 : Y3 + 1;
                am = (q < 2) ? xm : ym;
                bm = (q < 2) ? ym : xm;
            } else {
                kx = (kdown ? nkb - 1 - (kb >> 1) : (kb >> 1)) * TC_BK;
                am = bm = (kb & 1) ? X3 + 2 : X3 + 1;
            }
            if (!df_ready && kx / 256 != df_kt) {
                // Dataflow: this 256-column block of both operand panels must come
                // from tiles of the previous layer that have completed.
                df_kt = kx / 256;
                const int pa = row_a / 256, pb = row_b / 256;
                if (df_next != df_kt) flow_peek(p, pa, pb, df_kt, df_v);
                if (!flow_wait(p, pa, pb, df_kt, (unsigned int)(CG * w.n), df_v, abort)) {
                    tc_abort<CG>(rc, peer_abort);
                    break;
                }
                const int nx = kdown ? df_kt - 1 : df_kt + 1;   // next block of this walk
                df_next = -1;
                if (nx >= 0 && nx * 256 < d.np) {
                    flow_peek(p, pa, pb, nx, df_v);
                    df_next = nx;
                }
            }
            if (!mbar_wait(&tl.empty[stage], phase ^ 1u, abort, p.timeout_ns, p.err)) {
                tc_abort<CG>(rc, peer_abort);
                break;
            }
            pend[stage] = 0;
            uint8_t *sa = stages + (size_t)stage * C::STAGE_BYTES;
            if (CG == 1) {
                mbar_expect_tx(&tl.full[stage], C::TX_BYTES);
                tma_load_2d(sa, am, kx, row_a, &tl.full[stage]);
                tma_load_2d(sa + C::A_BYTES, bm, kx, row_b, &tl.full[stage]);
                tma_load_2d(sa + C::A_BYTES + C::B_BYTES / 2, bm, kx, row_b + 128, &tl.full[stage]);
            } else {
                // Both CTAs' bytes complete on the even CTA's barrier.
                if (leader) mbar_expect_tx(&tl.full[stage], C::TX_BYTES);
                const uint32_t fb = lead_full0 + stage * 8u;
                tma_load_2d_pair(sa, am, kx, row_a, fb);
                tma_load_2d_pair(sa + C::A_BYTES, bm, kx, row_b, fb);
            }
            pend[stage] = (int)phase + 1;
            *(volatile unsigned int *)&tl.issued = ++issued;
            if (++stage == C::STAGES) {
                stage = 0;
                phase ^= 1u;
            }
        }
    };
    // MMA issuer: tile w's products into the next accumulator; false when a wait
    // gave up (the launch is stopping).
    auto mma_tile = [&](const TileWork &w) -> bool {
        const InstDesc &d = p.inst[w.inst];
        if (!mbar_wait(&tl.tempty[acc], acc_phase ^ 1u, abort, p.timeout_ns, p.err)) {
            tc_abort<CG>(rc, peer_abort);
            return false;
        }
        tc_fence_after();
        const uint32_t d_tmem = tmem_base + acc * TC_BN;
        bool ok = true;
        if (!w.resp) {
            // Square: per K block the (hi, hi) and (lo, lo) slots, then hi lo, lo hi
            // (the small cross terms first) and hi hi.
            for (int kb = 0; kb < d.np / TC_BK; ++kb) {
                uint32_t sh, sl;
                const uint32_t st_h = stage;
                if (!mbar_wait(&tl.full[stage], phase, abort, p.timeout_ns, p.err)) {
                    tc_abort<CG>(rc, peer_abort);
                    ok = false;
                    break;
                }
                *(volatile unsigned int *)&tl.consumed = ++consumed;
                sh = smem_u32(stages + (size_t)stage * C::STAGE_BYTES);
                if (++stage == C::STAGES) {
                    stage = 0;
                    phase ^= 1u;
                }
                const uint32_t st_l = stage;
                if (!mbar_wait(&tl.full[stage], phase, abort, p.timeout_ns, p.err)) {
                    tc_abort<CG>(rc, peer_abort);
                    ok = false;
                    break;
                }
                *(volatile unsigned int *)&tl.consumed = ++consumed;
                sl = smem_u32(stages + (size_t)stage * C::STAGE_BYTES);
                if (++stage == C::STAGES) {
                    stage = 0;
                    phase ^= 1u;
                }
                tc_fence_after();
#pragma unroll
                for (int k = 0; k < TC_BK / 16; ++k)   // hi x lo
                    umma_f16<CG>(d_tmem, sdesc_sw128(sh + k * 32), sdesc_sw128(sl + C::A_BYTES + k * 32),
                                 idesc, (kb | k) != 0 ? 1u : 0u);
#pragma unroll
                for (int k = 0; k < TC_BK / 16; ++k)   // lo x hi
                    umma_f16<CG>(d_tmem, sdesc_sw128(sl + k * 32), sdesc_sw128(sh + C::A_BYTES + k * 32),
                                 idesc, 1u);
#pragma unroll
                for (int k = 0; k < TC_BK / 16; ++k)   // hi x hi
                    umma_f16<CG>(d_tmem, sdesc_sw128(sh + k * 32), sdesc_sw128(sh + C::A_BYTES + k * 32),
                                 idesc, 1u);
                umma_commit<CG>(&tl.empty[st_h]);
                umma_commit<CG>(&tl.empty[st_l]);
            }
        }
        if (w.resp) {
            // Response: per K block the slots (X hi, Y hi), (X lo, Y lo) for X Y^T,
            // released as soon as those products are issued, then (Y hi, X hi),
            // (Y lo, X lo) for Y X^T; cross terms before hi x hi in each.
            for (int kb = 0; ok && kb < d.np / TC_BK; ++kb) {
#pragma unroll 1
                for (int pr = 0; pr < 2; ++pr) {
                    const uint32_t st_h = stage;
                    if (!mbar_wait(&tl.full[stage], phase, abort, p.timeout_ns, p.err)) {
                        tc_abort<CG>(rc, peer_abort);
                        ok = false;
                        break;
                    }
                    *(volatile unsigned int *)&tl.consumed = ++consumed;
                    const uint32_t sh = smem_u32(stages + (size_t)stage * C::STAGE_BYTES);
                    if (++stage == C::STAGES) {
                        stage = 0;
                        phase ^= 1u;
                    }
                    const uint32_t st_l = stage;
                    if (!mbar_wait(&tl.full[stage], phase, abort, p.timeout_ns, p.err)) {
                        tc_abort<CG>(rc, peer_abort);
                        ok = false;
                        break;
                    }
                    *(volatile unsigned int *)&tl.consumed = ++consumed;
                    const uint32_t sl = smem_u32(stages + (size_t)stage * C::STAGE_BYTES);
                    if (++stage == C::STAGES) {
                        stage = 0;
                        phase ^= 1u;
                    }
                    tc_fence_after();
#pragma unroll
                    for (int k = 0; k < TC_BK / 16; ++k)   // A hi x B lo
                        umma_f16<CG>(d_tmem, sdesc_sw128(sh + k * 32),
                                     sdesc_sw128(sl + C::A_BYTES + k * 32), idesc,
                                     (kb | pr | k) != 0 ? 1u : 0u);
#pragma unroll
                    for (int k = 0; k < TC_BK / 16; ++k)   // A lo x B hi
                        umma_f16<CG>(d_tmem, sdesc_sw128(sl + k * 32),
                                     sdesc_sw128(sh + C::A_BYTES + k * 32), idesc, 1u);
#pragma unroll
                    for (int k = 0; k < TC_BK / 16; ++k)   // A hi x B hi
                        umma_f16<CG>(d_tmem, sdesc_sw128(sh + k * 32),
                                     sdesc_sw128(sh + C::A_BYTES + k * 32), idesc, 1u);
                    umma_commit<CG>(&tl.empty[st_h]);
                    umma_commit<CG>(&tl.empty[st_l]);
                }
            }
        }
        umma_commit<CG>(&tl.tfull[acc]);
        if (++acc == 2) {
            acc = 0;
            acc_phase ^= 1u;
        }
        return ok;
    };
    const int ew = warp - 2;                  // epilogue warp 0 .. EPI_WARPS - 1
    const int quarter = warp & 3;             // TMEM lanes this warp may access
    const int half = ew >> 2;                 // column half of the tile this warp owns
    uint32_t *T = (uint32_t *)(epi_T + (warp >= 2 ? ew : 0) * EPI_T_FLOATS);   // packed split operands
    uint16_t *Bh = (uint16_t *)T, *Bl = Bh + EPI_BOX_ROWS * EPI_BOX_COLS;      // or the hi and lo boxes
    bool flow_first = true;                   // dataflow: no tile completed by this CTA yet
    // Epilogue: the next layer from tile w's accumulator, its FP64 partials and, in
    // the dataflow schedule, the tile's completion flag.
    auto epilogue_tile = [&](const TileWork &w) {
        const InstDesc &d = p.inst[w.inst];
        const int np = d.np;
        const size_t mat = (size_t)np * np;
        int ok = 1;
        if (lane == 0) ok = mbar_wait(&tl.tfull[acc], acc_phase, abort, p.timeout_ns, p.err) ? 1 : 0;
        ok = __shfl_sync(0xffffffffu, ok, 0);
        tc_fence_after();
        const float *__restrict__ old;
        float *__restrict__ outf;
        uint16_t *__restrict__ o1;   // hi
        uint16_t *__restrict__ o2;   // lo
        const CUtensorMap *smap;     // store maps of hi, lo
        if (!w.resp) {
            old = xmaster(d, w.n, w.rec != 0);
            outf = xmaster(d, w.n + 1, w.rec != 0);
            const int so = xslot_of(d, w.n + 1);
            o1 = d.xop + (size_t)so * 2 * mat;
            o2 = o1 + mat;
            smap = d.xmap + (size_t)so * MAPS_PER_SLOT + 3;
        } else {
            const int yout = w.ybuf ^ 1;
            old = d.yf[w.ybuf];
            outf = d.yf[yout];
            o1 = d.yop + (size_t)yout * 2 * mat;
            o2 = o1 + mat;
            smap = d.ymap + (size_t)yout * MAPS_PER_SLOT + 3;
        }
        const float unscale = product_unscale<PREC>(w.resp != 0);
        const int rw0 = w.bi * C::TILE_M + (int)rank * 128 + quarter * 32;  // first row of this warp
        const int r = rw0 + lane;
        const int nreal = d.n;
        const float cf = w.cf;
        // Accelerated layer (a != 1) in terms of the product P of the stored
        // centred operands Y = X - I/2 (true Y = Y + cI): with T = aY + (1 - a/2) I
        // (X^2 branch) or T = aY + (a/2) I (2X - X^2 branch),
        //   X_{n+1} = ka (P + 2cY) + kb (Y + cI) + kc I,
        // ka = +-a^2, kb = a (2 - a), kc = (1 - a/2)^2 or a (1 - a/4); the
        // response / adjoint stream takes ka P + (kb + 2c ka) X1.
        const bool accel = (w.alpha != 1.0f);
        const float al = w.alpha;
        const float ka = w.flip ? -al * al : al * al;
        const float kb = al * (2.0f - al);
        const float kc = w.flip ? al * (1.0f - 0.25f * al) : (1.0f - 0.5f * al) * (1.0f - 0.5f * al);
        const float kx1 = fmaf(2.0f * cf, ka, kb);
        // ||Y||_F^2 of the next operands equals ||X||_F^2 off the diagonal (y = x
        // there); the diagonal difference y^2 - x^2 is accumulated apart (exact squares).
        FF ft = {0.f, 0.f}, fq = {0.f, 0.f}, fp = {0.f, 0.f}, fw = {0.f, 0.f};
        if (ok && rw0 < np) {
            // The chunks this warp finishes form one range [j0, j1): chunks entirely
            // below the diagonal come first, chunks past np last.
            int j0 = 0, j1 = 128 / EPI_CHUNK;
            while (j1 > 0 && w.bj * TC_BN + half * 128 + (j1 - 1) * EPI_CHUNK >= np) --j1;
            while (j0 < j1 && w.bj * TC_BN + half * 128 + j0 * EPI_CHUNK + EPI_CHUNK - 1 < rw0) ++j0;
            // The previous layer's (r, c) values -- (c, r) by symmetry, coalesced across
            // the warp, evict-first -- are loaded one chunk ahead, so that their latency
            // overlaps the current chunk's arithmetic and stores.
            float xnx[EPI_CHUNK];
            if (j0 < j1) {
                const int cb0 = w.bj * TC_BN + half * 128 + j0 * EPI_CHUNK;
#pragma unroll
                for (int jj = 0; jj < EPI_CHUNK; ++jj) xnx[jj] = __ldcs(old + (size_t)(cb0 + jj) * np + r);
            }
#pragma unroll 1
            for (int j = j0; j < j1; ++j) {
                const int c0 = half * 128 + j * EPI_CHUNK;   // column offset in the tile
                const int cb = w.bj * TC_BN + c0;
                float xov[EPI_CHUNK];
#pragma unroll
                for (int jj = 0; jj < EPI_CHUNK; ++jj) xov[jj] = xnx[jj];
                if (j + 1 < j1) {
#pragma unroll
                    for (int jj = 0; jj < EPI_CHUNK; ++jj)
                        xnx[jj] = __ldcs(old + (size_t)(cb + EPI_CHUNK + jj) * np + r);
                }
                float v[EPI_CHUNK];
                tmem_ld16(tmem_base + ((uint32_t)(quarter * 32) << 16) + acc * TC_BN + c0, v);
                // Each element's next split operands are computed once, stored to the
                // mirror (c, r) and staged packed (hi | lo << 16) for the direct (r, c)
                // stores below.  The FP32 master gets the mirror and the diagonal only.
                const bool upper = (cb > rw0 + 31);     // every element has r < c
                // Strictly upper chunks of plain layers write their direct (r, c) operands
                // as two boxes of tensor stores; the others through the transpose buffer,
                // once the previous chunk's boxes have left it.
                const bool boxed = upper && !accel;
                if (!boxed) {
                    if (lane == 0) bulk_wait_read();
                    __syncwarp();
                }
                uint32_t hp[EPI_CHUNK / 2], lp[EPI_CHUNK / 2];   // (r, c), (r, c + 1) packed
                if (upper && !w.resp && !accel) {
                    // The common case: a plain square-chain layer, strictly upper chunk.
                    const float twoc = 2.0f * cf;
#pragma unroll
                    for (int jj = 0; jj < EPI_CHUNK; ++jj) {
                        const int c = cb + jj;
                        const float xo = xov[jj];
                        const float t = fmaf(twoc, xo, v[jj] * unscale);
                        const float x = w.flip ? xo - t : t + xo;   // 2X - X^2 or X^2
                        ff_add_sq(fq, x, 2.0f);
                        const size_t m = (size_t)c * np + r;
                        __stcs(outf + m, x);
                        uint16_t a1, a2;
                        split2<PREC, X_SHIFT>(x, a1, a2);
                        __stcs(o1 + m, a1);
                        __stcs(o2 + m, a2);
                        pack_pair(hp, lp, jj, a1, a2);
                    }
                } else if (upper && w.resp && !accel) {
                    // Response / adjoint stream, plain layer, strictly upper chunk:
                    // X X1 + X1 X = P + (1 + 2c) X1, negated for 2X - X^2 (as below).
                    const float kx = w.flip ? 1.0f - 2.0f * cf : 1.0f + 2.0f * cf;
                    const float sg = w.flip ? -unscale : unscale;
#pragma unroll
                    for (int jj = 0; jj < EPI_CHUNK; ++jj) {
                        const int c = cb + jj;
                        const float x = fmaf(kx, xov[jj], v[jj] * sg);
                        const size_t m = (size_t)c * np + r;
                        __stcs(outf + m, x);
                        uint16_t a1, a2;
                        split2<PREC, Y_SHIFT>(x, a1, a2);
                        __stcs(o1 + m, a1);
                        __stcs(o2 + m, a2);
                        pack_pair(hp, lp, jj, a1, a2);
                    }
                } else {
#pragma unroll
                    for (int jj = 0; jj < EPI_CHUNK; ++jj) {
                        const int c = cb + jj;
                        const float P = v[jj] * unscale;            // raw product
                        const float xo = xov[jj];
                        const bool dg = (r == c) && (r < nreal);
                        float x;
                        if (!w.resp) {
                            // P = Y^2 for the stored operands Y = X - I/2; the true input is
                            // X + cI, so X^2 = P + 2cY + cI + X - I/4 (c^2 is below FP32 here).
                            const float yo = dg ? xo - 0.5f : xo;
                            if (accel) {
                                x = fmaf(ka, fmaf(2.0f * cf, yo, P), fmaf(kb, dg ? yo + cf : yo, dg ? kc : 0.0f));
                            } else {
                                const float b = dg ? P - 0.25f : P;
                                if (!w.flip) x = (b + fmaf(2.0f * cf, yo, dg ? cf : 0.0f)) + xo;  // X^2
                                else x = xo - (b + fmaf(2.0f * cf, yo, dg ? -cf : 0.0f));        // 2X - X^2
                            }
                        } else if (accel) {
                            x = fmaf(kx1, xo, ka * P);
                        } else {
                            // P = Y X1 + X1 Y; with X = Y + (1/2 + c) I the chain needs
                            // X X1 + X1 X = P + (1 + 2c) X1.
                            x = w.flip ? fmaf(1.0f - 2.0f * cf, xo, -P) : fmaf(1.0f + 2.0f * cf, xo, P);
                        }
                        const float y = (dg && !w.resp) ? x - 0.5f : x;  // next operands
                        uint16_t a1, a2;
                        if (!w.resp) split2<PREC, X_SHIFT>(y, a1, a2);
                        else split2<PREC, Y_SHIFT>(y, a1, a2);
                        if (r <= c) {
                            if (!w.resp) {
                                ff_add_sq(fq, x, (r == c) ? 1.0f : 2.0f);
                                if (r == c) ff_add(ft, x);
                                if (dg) {
                                    ff_add(fp, P);
                                    ff_add_sq(fw, y, 1.0f);
                                    ff_add_sq(fw, x, -1.0f);
                                }
                            }
                            // mirror (c, r), consecutive r across the warp; the diagonal
                            // element's FP32 master value here too
                            const size_t m = (size_t)c * np + r;
                            __stcs(outf + m, x);   // streaming stores: keep L2 for the operands
                            if (r < c) {
                                __stcs(o1 + m, a1);
                                __stcs(o2 + m, a2);
                            }
                        }
                        T[lane * (EPI_CHUNK + 1) + jj] = (uint32_t)a1 | ((uint32_t)a2 << 16);
                    }
                }
                if (boxed) {
                    // The chunk's 32 x 16 boxes of hi and lo, row-major, to global memory
                    // by the tensor store unit (the operands need both triangles: TMA
                    // loads rows).
                    if (lane == 0) bulk_wait_read();   // the previous boxes have left the buffer
                    __syncwarp();
                    uint4 *bh = (uint4 *)(Bh + lane * EPI_BOX_COLS), *bl = (uint4 *)(Bl + lane * EPI_BOX_COLS);
                    bh[0] = make_uint4(hp[0], hp[1], hp[2], hp[3]);
                    bh[1] = make_uint4(hp[4], hp[5], hp[6], hp[7]);
                    bl[0] = make_uint4(lp[0], lp[1], lp[2], lp[3]);
                    bl[1] = make_uint4(lp[4], lp[5], lp[6], lp[7]);
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    __syncwarp();
                    if (lane == 0) {
                        tma_store_2d(smap, Bh, cb, rw0);
                        tma_store_2d(smap + 1, Bl, cb, rw0);
                        bulk_commit();
                    }
                } else {
                    __syncwarp();
                    // direct (r, c) split-operand stores through the transpose buffer, two
                    // rows per step: lanes 0..15 row ii, lanes 16..31 row ii + 1
                    const int hl = lane >> 4, cl = lane & 15;
#pragma unroll 4
                    for (int it = 0; it < 16; ++it) {
                        const int ii = 2 * it + hl;
                        const int rr = rw0 + ii, cc = cb + cl;
                        if (upper || rr <= cc) {
                            const uint32_t pk = T[ii * (EPI_CHUNK + 1) + cl];
                            const size_t m = (size_t)rr * np + cc;
                            __stcs(o1 + m, (uint16_t)(pk & 0xFFFFu));
                            __stcs(o2 + m, (uint16_t)(pk >> 16));
                        }
                    }
                    __syncwarp();
                }
            }
        }
        // Release the accumulator: every lane's loads have completed
        // (tcgen05.wait::ld); one arrival per warp on the MMA side's barrier.
        tc_fence_before();
        __syncwarp();
        if (lane == 0) {
            if (CG == 2) mbar_arrive_cluster(lead_tempty0 + acc * 8u);
            else mbar_arrive(&tl.tempty[acc]);
        }
        if (++acc == 2) {
            acc = 0;
            acc_phase ^= 1u;
        }
        if (!w.resp) {
            // The tile's partials stay compensated FP32 pairs through the warp and
            // cross-warp sums (FP64 arithmetic is slow on this part); one conversion.
            FF qw = fq;
            ff_add_ff(qw, fw);
            const FF r4[4] = {ff_warp_sum(ft), ff_warp_sum(fq), ff_warp_sum(qw), ff_warp_sum(fp)};
            if (lane == 0)
#pragma unroll
                for (int k = 0; k < 4; ++k) tl.red[ew][k] = r4[k];
            if (p.dataflow) {
                // This warp's stores (generic proxy, and its tensor stores once
                // complete) reach the TMA reads (async proxy) of any CTA that sees the
                // tile's completion flag (the flag's writer fences for the CTA after
                // the barrier below).
                if (lane == 0) {
                    bulk_wait_all();
                    __threadfence();
                }
                asm volatile("fence.proxy.async.global;" ::: "memory");
            }
            asm volatile("bar.sync 1, %0;" ::"n"(EPI_WARPS * 32) : "memory");
            if (ew == 0 && lane == 0) {
                FF a4[4] = {tl.red[0][0], tl.red[0][1], tl.red[0][2], tl.red[0][3]};
                for (int k = 1; k < EPI_WARPS; ++k)
#pragma unroll
                    for (int c = 0; c < 4; ++c) ff_add_ff(a4[c], tl.red[k][c]);
                Part s4;
                s4.t = ff_value(a4[0]);
                s4.q = ff_value(a4[1]);
                s4.w = ff_value(a4[2]);
                s4.p = ff_value(a4[3]);
                d.part[(w.n + 1) % 3][w.tile * CG + (int)rank] = s4;
                if (p.dataflow) {
                    __threadfence();
                    // test_hook: CTA 0 withholds its first completion (a CTA that never
                    // finishes; the other CTAs' waits must run out).
                    if (!(p.test_hook == 1 && blockIdx.x == 0 && w.n == 0 && flow_first)) {
                        atomicAdd(p.tile_done + w.tile, 1u);
                        atomicAdd(p.layer_done, 1u);
                    }
                    flow_first = false;
                }
            }
            if (p.publish && ew == 0) {
                // Round schedule of a density batch: the CTA whose record completes the
                // instance's layer sums it (the order of every CTA's own sum) and
                // publishes the sums for the decision after the grid barrier.
                int last = 0;
                if (lane == 0) {
                    __threadfence();
                    const unsigned int target = (unsigned int)(w.n + 1) * (unsigned int)d.parts;
                    last = (atomicAdd(&d.ctl->psum_done, 1u) + 1u == target) ? 1 : 0;
                }
                last = __shfl_sync(0xffffffffu, last, 0);
                if (last) {
                    __threadfence();   // the other CTAs' records, released before their increments
                    double a[4];
                    sum_layer_partials(p, w.inst, w.n + 1, lane, a);
                    if (lane == 0) {
#pragma unroll
                        for (int c = 0; c < 4; ++c) d.ctl->psum[c] = a[c];
                        d.ctl->psum_n = w.n + 1;
                    }
                }
            }
            asm volatile("bar.sync 1, %0;" ::"n"(EPI_WARPS * 32) : "memory");
        }
    };

    if (p.dataflow) {
        // ------------- dataflow schedule (one instance, density mode) -------------
        // No grid barrier between layers.  The producer and the MMA thread run on into
        // the next layer as soon as their own tiles are done (the producer waits per
        // K block for the tiles that wrote it); only the epilogue needs the layer's
        // sign and offset, so the epilogue warps alone wait for every tile of the
        // previous layer, reduce its partials and take the decision.  When the stop
        // rule fires they halt the CTA: loads and MMAs issued ahead are drained at
        // teardown.  Each tile's arithmetic, and so X and D, is that of the barrier
        // schedule bit for bit.
        const int ntl = p.inst[0].ntiles;
        // When every pair has a few tiles in every layer (fewer than four), layer r's
        // round-robin starts at a rotated position, so that the pairs holding one
        // tile fewer change from layer to layer and the remainder tiles spread evenly
        // over the chain (a tile's arithmetic does not depend on the pair that
        // computes it).  With more tiles per pair the imbalance is small and the fixed
        // assignment keeps more of the operand panels in L2.
        const bool rotate = (ntl >= nclusters && ntl < 4 * nclusters);
        const auto first_tile = [&](int r) {
            return rotate ? (int)(((long long)cluster_id + (long long)r * (ntl % nclusters)) % nclusters) : cluster_id;
        };
        if (cluster_id >= ntl) {
            // no tiles here: only the epilogue warps take part (in the decisions)
        } else if (warp == 0) {
            if (lane == 0)
                for (int r = 0; !*abort; ++r)
                    for (int g = first_tile(r); g < ntl && !*abort; g += nclusters) produce_tile(describe_flow(p, g, r));
        } else if (warp == 1) {
            if (lane == 0 && leader) {
                bool ok = true;
                for (int r = 0; ok && !*abort; ++r)
                    for (int g = first_tile(r); ok && g < ntl && !*abort; g += nclusters)
                        ok = mma_tile(describe_flow(p, g, r));
            }
        } else {
            for (int r = 0;; ++r) {
                if (!flow_decide(rc, p, tl.flow_sums, r, ew, lane, ntl * CG, abort)) {
                    tc_abort<CG>(rc, peer_abort);   // stop rule or error: halt this CTA and its peer
                    break;
                }
                for (int g = first_tile(r); g < rc.total; g += nclusters) epilogue_tile(describe(rc, p, g));
            }
        }
    } else {
        // --------------- barrier schedule (every other mode and batch) ---------------
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
            // The epilogue transpose buffers are idle here: use them for the sums.
            reduce_round_partials(rc, p, (double *)epi_T);
            if (p.mode == MODE_ADJOINT) {
                if (threadIdx.x == 0) decide_round(rc, p, (const double *)epi_T);
            } else {
                decide_round_parallel(rc, p, (const double *)epi_T, (int *)((double *)epi_T + 4 * MAX_BATCH));
            }
            if (threadIdx.x == 0) {
                // Make the previous round's global writes (other CTAs' epilogues,
                // generic proxy) visible to this CTA's TMA reads (async proxy).
                asm volatile("fence.proxy.async.global;" ::: "memory");
            }
            __syncthreads();
            if (rc.abort || rc.total == 0) break;

            // The round's tiles (largest instances first) are dealt to the pairs in a
            // snake order, forward in even waves and backward in odd ones, which evens
            // out the pairs' shares of large and small tiles; each pair then takes its
            // share smallest first, so that the epilogues of its small tiles overlap
            // the MMAs of the large ones after them.
            const auto round_tile = [&](int k) {
                return k * nclusters + ((k & 1) ? nclusters - 1 - cluster_id : cluster_id);
            };
            int nk = 0;
            while (round_tile(nk) < rc.total) ++nk;
            if (warp == 0) {
                if (lane == 0)
                    for (int k = nk - 1; k >= 0 && !*abort; --k) produce_tile(describe(rc, p, round_tile(k)));
            } else if (warp == 1) {
                if (lane == 0 && leader)
                    for (int k = nk - 1; k >= 0 && !*abort; --k)
                        if (!mma_tile(describe(rc, p, round_tile(k)))) break;
            } else {
                for (int k = nk - 1; k >= 0; --k) epilogue_tile(describe(rc, p, round_tile(k)));
                // This warp's tensor stores are complete; order this round's
                // generic-proxy stores before the async-proxy (TMA) reads of the next
                // round, on any SM.
                if (lane == 0) bulk_wait_all();
                __syncwarp();
                asm volatile("fence.proxy.async.global;" ::: "memory");
                __threadfence();
            }
        }
    }

    // ------------------------------ teardown ------------------------------
    // Tensor stores still reading this CTA's shared memory finish before it is released.
    if (warp >= 2 && lane == 0) bulk_wait_all();
    // After an abort: MMAs this launch issued complete before tensor memory and the
    // stages are released (the commit covers every earlier MMA of the issuing thread).
    if (warp == 1 && lane == 0 && leader && rc.abort) {
        umma_commit<CG>(&tl.drain);
        const unsigned long long t0 = global_ns();
        while (!mbar_try_wait(&tl.drain, 0u) && global_ns() - t0 < p.timeout_ns) {
        }
    }
    if (CG == 1 && warp == 0 && lane == 0 && rc.abort) {
        // Let loads still in flight land before the CTA exits: bounded waits on the
        // barriers that count them.
        for (int s = 0; s < C::STAGES; ++s) {
            if (pend[s]) {
                const unsigned long long t0 = global_ns();
                while (!mbar_try_wait(&tl.full[s], (uint32_t)(pend[s] - 1)) && global_ns() - t0 < p.timeout_ns) {
                }
            }
        }
    }
    __syncthreads();
    if (CG == 2) {
        cluster_sync_all();   // both CTAs' producers have stopped issuing copies
        if (threadIdx.x == 0 && leader) {
            // Copies of either CTA land on the even CTA's full barriers, which count
            // both CTAs' bytes of a stage (equal shares).  Every ring stage in
            // [consumed, max(issued)) may still have copies in flight: arm the barrier
            // for the odd CTA's share if only the odd CTA issued that stage, retire the
            // odd CTA's share if only this CTA did, then wait (bounded) for the phase.
            unsigned int odd_issued;
            const uint32_t odd_addr = cluster_addr(&tl.issued, 1);
            asm volatile("ld.shared::cluster.u32 %0, [%1];" : "=r"(odd_issued) : "r"(odd_addr) : "memory");
            const unsigned int own = tl.issued, done = tl.consumed;
            const unsigned int top = own > odd_issued ? own : odd_issued;
            for (unsigned int i = done; i < top; ++i) {
                const uint32_t slot = i % C::STAGES, ph = (i / C::STAGES) & 1u;
                if (i >= own) mbar_expect_tx(&tl.full[slot], C::STAGE_BYTES);
                else if (i >= odd_issued)
                    asm volatile("mbarrier.complete_tx.relaxed.cta.shared::cta.b64 [%0], %1;" ::"r"(
                                     smem_u32(&tl.full[slot])),
                                 "r"(C::STAGE_BYTES)
                                 : "memory");
                const unsigned long long t0 = global_ns();
                while (!mbar_try_wait(&tl.full[slot], ph) && global_ns() - t0 < p.timeout_ns) {
                }
            }
        }
        __syncthreads();
        cluster_sync_all();  // neither CTA leaves while its peer may still signal it
    }
    if (warp == 1) {
        tc_fence_after();
        if (CG == 2)
            asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(TMEM_COLS)
                         : "memory");
        else
            asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(TMEM_COLS)
                         : "memory");
    }
}

template <int CG>
const void *tc_kernel_ptr(int precision) {
    return (precision == SP2_BF16_SPLIT) ? (const void *)k_tc_persistent<SP2_BF16_SPLIT, CG>
                                         : (const void *)k_tc_persistent<SP2_FP16_SPLIT, CG>;
}

}  // namespace

static_assert(SMEM_BYTES <= 232448, "dynamic shared memory above the 227 KB a CTA can hold");
size_t tc_smem_bytes() { return SMEM_BYTES; }

// Number of CTAs of a co-resident persistent grid for the given CTA group size
// (0 when the configuration cannot be launched on this device).
int tc_grid_size(int cta_group, int sm_count) {
    const void *fns[2] = {cta_group == 2 ? tc_kernel_ptr<2>(SP2_FP16_SPLIT) : tc_kernel_ptr<1>(SP2_FP16_SPLIT),
                          cta_group == 2 ? tc_kernel_ptr<2>(SP2_BF16_SPLIT) : tc_kernel_ptr<1>(SP2_BF16_SPLIT)};
    for (const void *f : fns)
        if (cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_BYTES) != cudaSuccess) {
            cudaGetLastError();
            return 0;
        }
    if (cta_group == 1) {
        int b = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, fns[0], TC_THREADS, SMEM_BYTES) != cudaSuccess) {
            cudaGetLastError();
            return 0;
        }
        return b >= 1 ? sm_count : 0;
    }
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(sm_count);
    cfg.blockDim = dim3(TC_THREADS);
    cfg.dynamicSmemBytes = SMEM_BYTES;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int nclusters = 0;
    if (cudaOccupancyMaxActiveClusters(&nclusters, fns[0], &cfg) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    if (nclusters * 2 > sm_count) nclusters = sm_count / 2;
    return nclusters * 2;
}

cudaError_t launch_tc_persistent(const RunParams &p, int cta_group, int grid, cudaStream_t s) {
    void *args[] = {(void *)&p};
    if (cta_group == 1) {
        // Cooperative launch (co-residency of the whole grid), through the
        // attribute form so that it can also be captured in a CUDA graph.
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeCooperative;
        attr[0].val.cooperative = 1;
        cfg.gridDim = dim3(grid);
        cfg.blockDim = dim3(TC_THREADS);
        cfg.dynamicSmemBytes = SMEM_BYTES;
        cfg.stream = s;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        return cudaLaunchKernelExC(&cfg, tc_kernel_ptr<1>(p.precision), args);
    }
    // CTA pairs: a cluster launch of exactly as many pairs as the device holds
    // at once (cudaOccupancyMaxActiveClusters, one CTA per SM), so on an idle GPU
    // every pair is resident for the grid barrier.  Without the cooperative
    // attribute (which the profiler cannot replay together with clusters) that
    // residency is not promised by the API: if concurrent work delays a pair,
    // the barrier's time limit ends the call with SP2_ERR_TIMEOUT.
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(TC_THREADS);
    cfg.dynamicSmemBytes = SMEM_BYTES;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelExC(&cfg, tc_kernel_ptr<2>(p.precision), args);
}

}  // namespace sp2i
