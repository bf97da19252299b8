// device_common.cuh -- device helpers shared by the SP2 kernels:
// compensated FP32 accumulation, order-preserving double keys, the hi/lo
// operand split, the grid barrier with a time limit, and the per-round layer
// decision (trace-correcting sign, idempotency stop rule) taken on the device.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include "sp2_internal.h"

namespace sp2i {

// ---------------------------------------------------------------------------
// Compensated (two-float) accumulation.  Each product x*x of an FP32 value is
// split exactly into p + e with an FMA; the running sum keeps its rounding
// error in a second float (TwoSum).  The pair carries ~48 significant bits,
// enough for the idempotency estimate Tr X - ||X||_F^2 at any size used here,
// at FP32 throughput (GB300 issues FP64 at a small fraction of FP32).
// The __f*_rn intrinsics keep the compiler from contracting the sums into FMAs.
// ---------------------------------------------------------------------------
struct FF {
    float s, c;
};

__device__ __forceinline__ void ff_add(FF &a, float v) {
    float t = __fadd_rn(a.s, v);
    float bp = __fsub_rn(t, a.s);
    float err = __fadd_rn(__fsub_rn(a.s, __fsub_rn(t, bp)), __fsub_rn(v, bp));
    a.s = t;
    a.c = __fadd_rn(a.c, err);
}

// a += w * x * x, w in {1, 2} (exact scaling by 2)
__device__ __forceinline__ void ff_add_sq(FF &a, float x, float w) {
    float p = __fmul_rn(x, x);
    float e = __fmaf_rn(x, x, -p);
    ff_add(a, __fmul_rn(w, p));
    a.c = __fadd_rn(a.c, __fmul_rn(w, e));
}

// a += b for two compensated pairs (two-sum of the leading parts; the small parts
// and the sum's rounding error accumulate in a.c).
__device__ __forceinline__ void ff_add_ff(FF &a, const FF &b) {
    ff_add(a, b.s);
    a.c = __fadd_rn(a.c, b.c);
}

// Sum of a compensated pair over the 32 lanes of a warp (fixed shuffle tree; lane 0
// holds the result).
__device__ __forceinline__ FF ff_warp_sum(FF a) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        FF b;
        b.s = __shfl_down_sync(0xffffffffu, a.s, o);
        b.c = __shfl_down_sync(0xffffffffu, a.c, o);
        ff_add_ff(a, b);
    }
    return a;
}

__device__ __forceinline__ double ff_value(const FF &a) { return (double)a.s + (double)a.c; }

// ---------------------------------------------------------------------------
// Order-preserving 64-bit keys so that min / max of doubles can use integer
// atomics (exact and independent of arrival order).
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ unsigned long long dkey(double v) {
    unsigned long long b;
#ifdef __CUDA_ARCH__
    b = (unsigned long long)__double_as_longlong(v);
#else
    memcpy(&b, &v, 8);
#endif
    return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}
__host__ __device__ __forceinline__ double dkey_value(unsigned long long k) {
    unsigned long long b = (k >> 63) ? (k & 0x7fffffffffffffffull) : ~k;
#ifdef __CUDA_ARCH__
    return __longlong_as_double((long long)b);
#else
    double v;
    memcpy(&v, &b, 8);
    return v;
#endif
}

// ---------------------------------------------------------------------------
// The split X = X^(0) + X^(1) (section "Deep-neural network electronic structure
// solver", the dual matrix representation), with round-to-nearest-even, and
// both parts stored times 2^SHIFT (exact power-of-two scaling):
//   hi = FP16[x],  stored FP16[hi * 2^SHIFT],  lo = FP16[(x - hi) * 2^SHIFT].
// x - hi is exact in FP32.  The X stream uses SHIFT = 11: lo ~ 2^-11 |x| then stays
// in FP16's normal range, hi * 2^11 <= 2^11 cannot overflow (|x| <= 1), and all
// three products of the square carry 2^22, removed in the epilogue.  The second
// stream (response / adjoint), whose entries grow along the chain, keeps SHIFT = 0
// (the full FP16 range for hi; a subnormal lo costs at most 2^-24 absolute).
// BF16 needs no scaling (its exponent range is FP32's): SHIFT is ignored.
// ---------------------------------------------------------------------------
constexpr int X_SHIFT = LO_SHIFT;   // X stream
constexpr int Y_SHIFT = 0;          // response / adjoint stream

template <int SHIFT>
__device__ __forceinline__ void split_fp16(float x, uint16_t &hi, uint16_t &lo) {
    __half h = __float2half_rn(x);
    const float hf = __half2float(h);
    hi = __half_as_ushort(__float2half_rn(hf * (float)(1 << SHIFT)));
    lo = __half_as_ushort(__float2half_rn(__fsub_rn(x, hf) * (float)(1 << SHIFT)));
}
__device__ __forceinline__ void split_bf16(float x, uint16_t &hi, uint16_t &lo) {
    __nv_bfloat16 h = __float2bfloat16_rn(x);
    hi = __bfloat16_as_ushort(h);
    lo = __bfloat16_as_ushort(__float2bfloat16_rn(__fsub_rn(x, __bfloat162float(h))));
}
template <int PREC, int SHIFT>
__device__ __forceinline__ void split2(float x, uint16_t &hi, uint16_t &lo) {
    if (PREC == SP2_FP16_SPLIT) split_fp16<SHIFT>(x, hi, lo);
    else split_bf16(x, hi, lo);
}
// Factor that turns an accumulated product back into X X (resp = 0) or X Y (resp = 1).
template <int PREC>
__host__ __device__ __forceinline__ float product_unscale(bool resp) {
    if (PREC != SP2_FP16_SPLIT) return 1.0f;
    return resp ? 1.0f / (float)(1 << (X_SHIFT + Y_SHIFT)) : 1.0f / ((float)(1 << X_SHIFT) * (float)(1 << X_SHIFT));
}

// ---------------------------------------------------------------------------
// Timers and memory-order helpers.
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ unsigned int ld_acquire(const unsigned int *p) {
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ int ld_volatile(const int *p) { return *(const volatile int *)p; }

__device__ __forceinline__ void set_error(int *err, int code) { atomicCAS(err, 0, code); }

// Grid barrier for a cooperative (co-resident) launch: every CTA's thread 0
// adds one arrival and waits until `target` arrivals are counted.  Gives up
// after `timeout_ns` (or when another CTA reported an error) and returns false.
__device__ __forceinline__ bool grid_barrier(unsigned int *counter, unsigned int target, int *err,
                                             unsigned long long timeout_ns, bool withhold = false) {
    __threadfence();
    if (!withhold) atomicAdd(counter, 1u);
    unsigned long long t0 = global_ns();
    while (ld_acquire(counter) < target) {
        if (ld_volatile(err) != 0) return false;
        if (global_ns() - t0 > timeout_ns) {
            set_error(err, SP2_ERR_TIMEOUT);
            return false;
        }
        __nanosleep(64);
    }
    __threadfence();
    return true;
}

// ---------------------------------------------------------------------------
// Where X_n lives.  Without checkpointing: operand slot n mod nslots_x and FP32
// master xf[n & 1].  With checkpoint stride s (adjoint): the kept X_{ks} in
// operand slot k and FP32 master ckf[k]; every other X_n in slot K + (n mod s) - 1
// and, while the forward chain runs, xf[n & 1] (so X_L stays there for the
// output), while the reverse sweep recomputes it, rf[n & 1].
// ---------------------------------------------------------------------------
__device__ __forceinline__ int xslot_of(const InstDesc &d, int n) {
    if (d.ckpt_s > 0) {
        const int r = n % d.ckpt_s;
        return r == 0 ? n / d.ckpt_s : d.ckpt_k + r - 1;
    }
    return n % d.nslots_x;
}
__device__ __forceinline__ float *xmaster(const InstDesc &d, int n, bool recompute) {
    if (d.ckpt_s > 0) {
        if (n % d.ckpt_s == 0) return d.ckf + (size_t)(n / d.ckpt_s) * d.np * d.np;
        return recompute ? d.rf[n & 1] : d.xf[n & 1];
    }
    return d.xf[n & 1];
}

// ---------------------------------------------------------------------------
// Per-round control state kept in shared memory by every CTA.  Every CTA
// computes the same decisions from the same FP64 partials in the same order,
// so no broadcast between CTAs is needed; CTA 0 alone writes the statistics.
// ---------------------------------------------------------------------------
struct RoundCtl {
    int abort;
    int total;                       // tiles in this round over all instances
    int phase;                       // adjoint: 0 forward, 1 reverse
    int rev_left;                    // adjoint: reverse layers still to do
    int rev_total;                   // adjoint: forward layer count L
    int rec_mode;                    // adjoint reverse round: 0 reverse layer, 1 recompute X_{rec_top + 1}
    int rec_top;                     // adjoint checkpointing: highest n whose X_n is held for the segment
    int rec_seg;                     // adjoint checkpointing: segment (m / s) of the layers held
    int prefix[MAX_BATCH + 1];       // active tile prefix over instances
    int layer[MAX_BATCH];            // index n of the current X_n
    int jobs[MAX_BATCH];             // 0 (inactive), 1 (square) or 2 (square + response)
    signed char choice[MAX_BATCH];   // sign of the layer computed this round
    unsigned char active[MAX_BATCH];
    unsigned char ran[MAX_BATCH];    // instance computed a layer in the previous round
    double ehist[MAX_BATCH][2];
    double wprev[MAX_BATCH];         // ||Y_n||_F^2 of the operands of the current square
    double coff[MAX_BATCH];          // c_n: true X_n = stored X_n + c_n I
    signed char chist[MAX_L + 2];    // adjoint (B = 1): choice that produced X_n
    double chist_c[MAX_L + 2];       // adjoint (B = 1): c_n per layer
    float chist_a[MAX_L + 2];        // adjoint (B = 1): a_n of the layer that produced X_n
    float alpha[MAX_BATCH];          // a of the layer computed this round (1 = plain)
    float xl[MAX_BATCH], xh[MAX_BATCH];  // accelerated chain: images of eps_lumo, eps_homo
    int flow_go;                     // dataflow schedule: the previous layer is complete
};

__host__ __device__ __forceinline__ int layer_rule(double t, double q, double n_occ) {
    return fabs(q - n_occ) <= fabs(2.0 * t - q - n_occ) ? SP2_CHOICE_SQUARE : SP2_CHOICE_FLIP;
}

__device__ __forceinline__ void round_ctl_init(RoundCtl &rc, const RunParams &p) {
    rc.abort = 0;
    rc.total = 0;
    rc.phase = 0;
    rc.rev_left = 0;
    rc.rev_total = 0;
    rc.rec_mode = 0;
    rc.rec_top = 0;
    rc.rec_seg = 0;
    for (int i = 0; i < p.B; ++i) {
        InstCtl *ctl = p.inst[i].ctl;
        rc.layer[i] = 0;
        rc.jobs[i] = 0;
        rc.choice[i] = SP2_CHOICE_INPUT;
        rc.active[i] = (ctl->status == 0) ? 1 : 0;
        rc.ran[i] = 0;
        rc.ehist[i][0] = rc.ehist[i][1] = 0.0;
        rc.wprev[i] = 0.0;
        rc.coff[i] = 0.0;
        rc.alpha[i] = 1.0f;
        // Images of the estimated interval under the input layer, clipped to
        // [0, 1]; (0, 1) keeps every a_n = 1, the plain chain.
        float xl = 0.0f, xh = 1.0f;
        const InstDesc &d = p.inst[i];
        if (d.accel) {
            const double span = ctl->eps_max - ctl->eps_min;
            const double l = (ctl->eps_max - d.gap_lumo) / span, h = (ctl->eps_max - d.gap_homo) / span;
            if (span > 0.0 && l < h) {
                xl = (float)fmin(fmax(l, 0.0), 1.0);
                xh = (float)fmin(fmax(h, 0.0), 1.0);
            }
        }
        rc.xl[i] = xl;
        rc.xh[i] = xh;
    }
    rc.chist[0] = SP2_CHOICE_INPUT;
    rc.chist_a[0] = 1.0f;
}

// One warp: the sums of instance i's partial records of layer n, lane l adding
// entries l, l + 32, ... in increasing order, then a fixed shuffle tree (valid in
// lane 0).  The order depends only on the instance's own records, so every CTA --
// and a batch or a lone call alike -- gets the same bits and takes the same decision.
__device__ __forceinline__ void sum_layer_partials(const RunParams &p, int i, int n, int lane, double (&a)[4]) {
    const InstDesc &d = p.inst[i];
    const int cnt = (n == 0) ? d.ctl->init_parts : d.parts;
    const Part *part = d.part[n % 3];
    a[0] = a[1] = a[2] = a[3] = 0.0;
#pragma unroll 4
    for (int k = lane; k < cnt; k += 32) {
        const Part v = part[k];
        a[0] += v.t;
        a[1] += v.q;
        a[2] += v.w;
        a[3] += v.p;
    }
#pragma unroll
    for (int c = 0; c < 4; ++c)
        for (int o = 16; o > 0; o >>= 1) a[c] += __shfl_down_sync(0xffffffffu, a[c], o);
}

// The sums of the layer instance i just finished.
__device__ __forceinline__ void sum_instance_partials(const RoundCtl &rc, const RunParams &p, int i, int lane,
                                                      double (&a)[4]) {
    sum_layer_partials(p, i, rc.layer[i] + (rc.ran[i] ? 1 : 0), lane, a);
}

// All threads of a CTA: the sums, for every instance still running, of the
// partials of the layer just finished into sums[4 i .. 4 i + 3] (shared memory),
// one warp per instance (warp w takes instances w, w + nwarps, ...).  In a density
// batch's round schedule the CTA that completed an instance's layer has already
// published these sums (same function, same order, same bits): they are read back.
// `sums` is followed by MAX_BATCH ints of scratch (the decision's buffer, free here).
__device__ inline void reduce_round_partials(const RoundCtl &rc, const RunParams &p, double *sums) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (rc.phase == 1) return;
    int *got = (int *)(sums + 4 * MAX_BATCH);
    // Published sums first, one thread per instance, every load in flight at once.
    for (int i = threadIdx.x; i < p.B; i += blockDim.x) {
        int ok = 0;
        const int n = rc.layer[i] + (rc.ran[i] ? 1 : 0);
        if (p.publish && rc.active[i] && n > 0) {
            const InstCtl *ctl = p.inst[i].ctl;
            const int pn = __ldcg(&ctl->psum_n);
            double v[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) v[c] = __ldcg(&ctl->psum[c]);
            if (pn == n) {
#pragma unroll
                for (int c = 0; c < 4; ++c) sums[i * 4 + c] = v[c];
                ok = 1;
            }
        }
        got[i] = ok;
    }
    __syncthreads();
    for (int i = wid; i < p.B; i += nw) {
        if (!rc.active[i] || got[i]) continue;
        double a[4];
        sum_layer_partials(p, i, rc.layer[i] + (rc.ran[i] ? 1 : 0), lane, a);
        if (lane == 0)
            for (int c = 0; c < 4; ++c) sums[i * 4 + c] = a[c];
    }
    __syncthreads();
}

// The decision for instance i from the sums of the layer just finished: record
// its statistics (CTA 0), apply the stop rule and pick the next sign.  Returns
// the number of tiles instance i computes this round, or -1 when an adjoint
// forward chain stopped and the round was set up for the reverse sweep.
static __device__ __noinline__ int decide_instance(RoundCtl &rc, const RunParams &p, const double *sums, int i, bool writer);

// Thread 0 of every CTA: the whole round's decision, instance by instance (the
// adjoint's reverse sweep and its switch to it live here; that path has B = 1).
__device__ inline void decide_round(RoundCtl &rc, const RunParams &p, const double *sums) {
    const bool writer = (blockIdx.x == 0);
    if (ld_volatile(p.err) != 0) {
        rc.abort = 1;
        return;
    }
    if (rc.phase == 1) {  // adjoint reverse sweep (B == 1); layer[0] counts reverse rounds done
        const InstDesc &d0 = p.inst[0];
        if (rc.rec_mode) {
            rc.rec_top += 1;  // X_{rec_top + 1} was recomputed
        } else {
            rc.layer[0] += 1;
            rc.rev_left -= 1;
        }
        rc.prefix[0] = 0;
        if (rc.rev_left <= 0) {
            if (writer) d0.ctl->final_y = rc.layer[0] & 1;  // Y buffer holding G_0
            rc.prefix[1] = 0;
            rc.total = 0;
            return;
        }
        // The next reverse layer m needs X_m.  With checkpointing, entering a new
        // segment leaves only its kept X_{seg s}; X_{seg s + 1} .. X_m are recomputed
        // first, one round each, with the forward's own signs, offsets and expansions.
        rc.rec_mode = 0;
        if (d0.ckpt_s > 0) {
            const int m = rc.rev_total - 1 - rc.layer[0];
            const int seg = m / d0.ckpt_s;
            if (seg != rc.rec_seg) {
                rc.rec_seg = seg;
                rc.rec_top = seg * d0.ckpt_s;
            }
            if (m > rc.rec_top) rc.rec_mode = 1;
        }
        rc.jobs[0] = 1;
        rc.prefix[1] = d0.ntiles;
        rc.total = d0.ntiles;
        return;
    }
    int acc = 0;
    rc.prefix[0] = 0;
    for (int i = 0; i < p.B; ++i) {
        const int width = decide_instance(rc, p, sums, i, writer);
        if (width < 0) return;
        acc += width;
        rc.prefix[i + 1] = acc;
    }
    rc.total = acc;
}

// Compiled out of line: inlined into the persistent kernels it raises their
// register allocation (the FP32 kernel then drops from two CTAs per SM to one).
static __device__ __noinline__ int decide_instance(RoundCtl &rc, const RunParams &p, const double *sums, int i, bool writer) {
    const InstDesc &d = p.inst[i];
    InstCtl *ctl = d.ctl;
    int width = 0;
    if (rc.active[i]) {
        if (rc.ran[i]) rc.layer[i] += 1;
        const int n = rc.layer[i];
        const double ts = sums[i * 4 + 0], qs = sums[i * 4 + 1], ws = sums[i * 4 + 2], ps = sums[i * 4 + 3];
        const int made = (n == 0) ? SP2_CHOICE_INPUT : rc.choice[i];
        // Accumulator bias of the square that made X_n: in exact arithmetic
        // Tr(Y^2) = ||Y||_F^2 for the symmetric operand Y, so the deficit of the
        // computed trace, spread over the N diagonal entries, is the identity
        // component of the product error.  It is removed as the offset c_n of
        // X_n (sign of the layer: X^2 keeps it, 2X - X^2 negates it).  Both
        // sums are zero on the FP32 path, where c_n stays 0.
        // An accelerated layer multiplies the product by +-a^2 (X^2: +, 2X - X^2: -).
        double c = 0.0;
        const float a_made = (n == 0) ? 1.0f : rc.alpha[i];
        if (n > 0) {
            const double gam = (rc.wprev[i] - ps) / (double)d.n;
            const double a2 = (double)a_made * (double)a_made;
            c = (made == SP2_CHOICE_SQUARE) ? a2 * gam : -a2 * gam;
        }
        const double t = ts + (double)d.n * c;
        const double q = qs + 2.0 * c * ts + (double)d.n * c * c;
        rc.wprev[i] = ws;
        rc.coff[i] = c;
        if (p.B == 1) rc.chist_c[n] = c;  // layer history for the adjoint (one instance)
        if (writer) {
            LayerStatDev st;
            st.trace = t;
            st.trace_sq = q;
            st.idem = t - q;
            st.choice = made;
            st.reserved = 0;
            st.alpha = (double)a_made;
            ctl->stat[n] = st;
        }
        if (p.B == 1) {
            rc.chist[n] = (signed char)made;
            rc.chist_a[n] = a_made;
        }
        const double e = fabs(t - q);
        const double e2 = rc.ehist[i][n & 1];
        rc.ehist[i][n & 1] = e;
        int reason = 0, status = 0;
        bool stop = false;
        if (!isfinite(t) || !isfinite(q)) {
            stop = true;
            status = SP2_ERR_NONFINITE;
        } else if (ctl->degenerate) {
            stop = true;
            status = SP2_ERR_NOT_CONVERGED;
            reason = SP2_STOP_MAX;
        } else if (d.nforced >= 0) {
            if (n >= d.nforced) {
                stop = true;
                if (e <= p.tol) reason = SP2_STOP_TOL;
                else if (n >= 2 && e <= STALL_MAX && e >= e2) reason = SP2_STOP_STALL;
                else reason = SP2_STOP_NONE;
            }
        } else if (e <= p.tol) {
            stop = true;
            reason = SP2_STOP_TOL;
        } else if (n >= 2 && e <= STALL_MAX && e >= e2) {
            stop = true;
            reason = SP2_STOP_STALL;
        } else if (n >= p.max_layers) {
            stop = true;
            reason = SP2_STOP_MAX;
            status = SP2_ERR_NOT_CONVERGED;
        }
        if (stop) {
            rc.active[i] = 0;
            rc.ran[i] = 0;
            if (writer) {
                ctl->layers = n;
                ctl->stop_reason = reason;
                ctl->status = status;
                ctl->final_x = n & 1;
                ctl->final_y = n & 1;
                ctl->x_offset = c;
            }
            if (p.mode == MODE_ADJOINT && status == 0) {
                // Switch to the reverse sweep: G_L is in Y buffer 0.  Reverse round
                // k (= layer[0]) maps G_{m+1} to G_m with m = L - 1 - k, reading Y
                // buffer k & 1 and X_m from slot m.
                rc.phase = 1;
                rc.rev_total = n;
                rc.rev_left = n;
                rc.layer[0] = 0;
                // The forward chain left X_{s floor((L-1)/s)} .. X_{L-1} in place.
                rc.rec_mode = 0;
                rc.rec_seg = (d.ckpt_s > 0 && n > 0) ? (n - 1) / d.ckpt_s : 0;
                rc.rec_top = n - 1;
                rc.prefix[1] = 0;
                rc.total = 0;
                if (n == 0) {
                    if (writer) ctl->final_y = 0;
                    return -1;
                }
                rc.jobs[0] = 1;
                rc.prefix[1] = d.ntiles;
                rc.total = d.ntiles;
                return -1;
            }
        } else {
            const int c = (d.nforced >= 0) ? d.forced[n] : layer_rule(t, q, d.n_occ);
            rc.choice[i] = (signed char)c;
            // Expansion of the accelerated layer: the tracked ends of the interval
            // are balanced around the branch's fixed point, then follow the layer.
            float a = 1.0f;
            if (d.nforced >= 0 && d.forced_alpha) {
                a = (float)d.forced_alpha[n];
            } else if (d.accel) {
                a = (c == SP2_CHOICE_SQUARE) ? 2.0f / (2.0f - rc.xl[i]) : 2.0f / (1.0f + rc.xh[i]);
                if (c == SP2_CHOICE_SQUARE) {
                    const float tl = fmaf(a, rc.xl[i], 1.0f - a), th = fmaf(a, rc.xh[i], 1.0f - a);
                    rc.xl[i] = tl * tl;
                    rc.xh[i] = th * th;
                } else {
                    const float tl = a * rc.xl[i], th = a * rc.xh[i];
                    rc.xl[i] = fmaf(-tl, tl, 2.0f * tl);
                    rc.xh[i] = fmaf(-th, th, 2.0f * th);
                }
            }
            rc.alpha[i] = a;
            rc.ran[i] = 1;
            rc.jobs[i] = (p.mode == MODE_RESPONSE) ? 2 : 1;
            width = rc.jobs[i] * d.ntiles;
        }
    }
    if (!rc.active[i]) rc.jobs[i] = 0;
    return width;
}

// All threads of every CTA: the round's decision with one thread per instance
// (density, response and layer-application runs; the adjoint, a single instance,
// goes through decide_round).  `wbuf` holds MAX_BATCH ints of shared memory.
__device__ inline void decide_round_parallel(RoundCtl &rc, const RunParams &p, const double *sums, int *wbuf) {
    if (threadIdx.x == 0 && ld_volatile(p.err) != 0) rc.abort = 1;
    __syncthreads();
    if (rc.abort) return;
    const bool writer = (blockIdx.x == 0);
    for (int i = threadIdx.x; i < p.B; i += blockDim.x) wbuf[i] = decide_instance(rc, p, sums, i, writer);
    __syncthreads();
    if (threadIdx.x == 0) {
        int acc = 0;
        rc.prefix[0] = 0;
        for (int i = 0; i < p.B; ++i) {
            acc += wbuf[i];
            rc.prefix[i + 1] = acc;
        }
        rc.total = acc;
    }
}

// All threads of a CTA, for the FP32 CUDA-core kernel: the same sums with thread k
// adding entries k, k + blockDim.x, ..., a fixed shuffle tree and a fixed sum over
// warps, instance after instance.  That kernel runs two CTAs per SM, and there
// one warp per instance over its 2N^2/128^2 partials costs more than the
// block-wide pass (measured: +56 ms over a 32-layer chain at N = 8192).  The order
// again depends only on the instance's partials and the block size.
__device__ inline void reduce_round_partials_block(const RoundCtl &rc, const RunParams &p, double *sums,
                                                   double *wscratch) {
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
    if (rc.phase == 1) return;
    for (int i = 0; i < p.B; ++i) {
        if (!rc.active[i]) continue;
        const InstDesc &d = p.inst[i];
        const int n = rc.layer[i] + (rc.ran[i] ? 1 : 0);
        const int cnt = (n == 0) ? d.ctl->init_parts : d.parts;
        const Part *part = d.part[n % 3];
        double a[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll 4
        for (int k = tid; k < cnt; k += blockDim.x) {
            const Part v = part[k];
            a[0] += v.t;
            a[1] += v.q;
            a[2] += v.w;
            a[3] += v.p;
        }
#pragma unroll
        for (int c = 0; c < 4; ++c)
            for (int o = 16; o > 0; o >>= 1) a[c] += __shfl_down_sync(0xffffffffu, a[c], o);
        if (lane == 0)
            for (int c = 0; c < 4; ++c) wscratch[wid * 4 + c] = a[c];
        __syncthreads();
        if (tid == 0) {
            double r[4] = {0.0, 0.0, 0.0, 0.0};
            for (int w = 0; w < nw; ++w)
                for (int c = 0; c < 4; ++c) r[c] += wscratch[w * 4 + c];
            for (int c = 0; c < 4; ++c) sums[i * 4 + c] = r[c];
        }
        __syncthreads();
    }
}

// Map a round-global tile index to (instance, job, tile).
__device__ __forceinline__ void map_tile(const RoundCtl &rc, int B, const InstDesc *inst, int g, int &i,
                                         int &job, int &tile) {
    int lo = 0, hi = B;  // find i with prefix[i] <= g < prefix[i+1]
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (rc.prefix[mid] <= g) lo = mid;
        else hi = mid;
    }
    i = lo;
    int local = g - rc.prefix[i];
    int nt = inst[i].ntiles;
    job = local / nt;
    tile = local - job * nt;
}

}  // namespace sp2i
