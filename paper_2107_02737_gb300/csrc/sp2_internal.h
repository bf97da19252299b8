// sp2_internal.h -- data layout shared by the host launcher and the device kernels.
//
// Device memory per instance (all row-major, padded size np = round_up(N, 128)):
//   xf[2]       FP32 master copy of X_n, ping-pong by layer parity.  The tensor-core
//               layers keep its lower triangle and diagonal current (the next layer
//               reads (c, r) for its tiles' r <= c); the output kernel mirrors it.
//   xop slots   split operands of X_n, two 16-bit matrices per slot, hi and lo
//               (FP16: both stored times 2^11), from which each K block of the
//               square issues hi*lo, lo*hi and hi*hi into one FP32 accumulator
//               (Eq. activ: A + B + B^T with the lo*lo term dropped).
//   yf[2], yop  the response / adjoint stream (FP32 master + hi, lo).
//   adjoint with checkpoint stride s: operand slots 0..K-1 hold X_0, X_s, ...,
//               X_{(K-1)s} (with FP32 masters in ckf), slots K..K+s-2 the others
//               by n mod s; the reverse sweep recomputes a segment's layers from
//               its kept X into those slots (FP32 ping-pong rf).
//   part[3]     FP64 partials per tile, by layer n mod 3: Tr X, ||X||_F^2,
//               ||Y||_F^2 and Tr P (see Part).
//   dataflow schedule (one instance, density mode, tensor cores): three operand
//               slots; per tile a completion counter (CTAs done, all layers) and a
//               table of the tiles that write each 256 x 256 block of X.
// Tensor-core path: the operands are the split of Y = X - I/2 (identity on the
// first N diagonal entries only), and the true X_n is the stored FP32 X_n plus
// c_n I, where the scalar c_n removes the measured accumulator bias of the
// previous square (see the tensor-core kernel).
// Padding lives in X space: rows and columns N..np-1 of X_0 are zero, and zero
// rows and columns stay zero under both X^2 and 2X - X^2.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "sp2.h"

namespace sp2i {

constexpr int PAD = 128;            // np is a multiple of this
constexpr int TC_BM = 128;          // tcgen05 tile rows (UMMA M)
constexpr int TC_BN = 256;          // tcgen05 tile columns (UMMA N)
constexpr int TC_BK = 64;           // K block: 64 x 16-bit = one 128-byte swizzle row
constexpr int TC_STAGES = 4;        // TMA -> MMA pipeline depth
constexpr int MAPS_PER_SLOT = 5;    // per operand slot: loads hi, hi, lo (64 x 128 boxes); stores hi, lo
constexpr int EPI_BOX_COLS = 16;    // store box: one epilogue warp's chunk of 32 rows x 16 columns
constexpr int EPI_BOX_ROWS = 32;
constexpr int TC_THREADS = 320;     // warp 0 TMA, warp 1 MMA, warps 2..9 epilogue (two per SM sub-partition)
constexpr int SIMT_T = 128;         // FP32 SIMT tile (square)
constexpr int SIMT_THREADS = 256;
constexpr int MAX_BATCH = 128;
constexpr int MAX_L = SP2_MAX_LAYERS_LIMIT;
constexpr int INIT_BLOCKS_MAX = 1024;
constexpr int FIN_BLOCKS_MAX = 1024;
constexpr int LO_SHIFT = 11;        // FP16 lo parts are stored times 2^11 (exact scaling)
constexpr double STALL_MAX = 1e-2;

enum Path { PATH_SIMT = 0, PATH_TC = 1 };
enum Mode { MODE_DENSITY = 0, MODE_RESPONSE = 1, MODE_ADJOINT = 2, MODE_APPLY = 3 };

// Per-tile FP64 partial sums written by the input layer and every square.
struct __align__(16) Part {
    double t;   // Tr X (stored X)
    double q;   // ||X||_F^2 (stored X)
    double w;   // ||Y||_F^2 of the split operand matrix Y the next square multiplies (0 on the FP32 path)
    double p;   // Tr P, P the raw product of this square (0 on the FP32 path)
};

struct LayerStatDev {
    double trace, trace_sq, idem;
    int choice, reserved;
    double alpha;
};

struct InstCtl {
    double eps_min, eps_max, band_energy, trace_D;
    double y_scale;                          // power of two applied to the Y stream
    double x_offset;                         // c_L: D = stored X_L + c_L I
    unsigned long long emin_key, emax_key;   // order-preserving keys for atomic min / max
    unsigned long long ymax_key;
    int nonfinite, status, layers, stop_reason;
    int final_x, final_y, init_parts, degenerate;
    // Round schedule of a density batch: the CTA that completes an instance's last
    // tile of layer n sums the layer's partial records (the same fixed order as
    // every CTA's own sum) and publishes them here, tagged with n.
    unsigned int psum_done;                  // CTA-tile completions over all layers
    int psum_n;                              // layer of psum (0: none yet)
    double psum[4];
    LayerStatDev stat[MAX_L + 1];
};

struct InstDesc {
    int n, np, ntiles, tile_off;      // tiles: this instance's slice of the tile table
    int parts;                        // partial records per layer (tiles x CTAs per tile)
    int kwave;                        // tensor-core path: tiles the device runs at once; tile t walks K
                                      // upward when (t / kwave) is even, downward when odd
    double n_occ;
    int nforced, nslots_x;            // nforced < 0: decide on device; nslots_x: 2, L+1 or K+s-1
    int ckpt_s, ckpt_k;               // adjoint checkpointing: every s-th X kept (K of them), 0 = off
    float *ckf;                       // FP32 masters of the kept X_{k s}, k < K (ckpt_s > 0)
    float *rf[2];                     // FP32 ping-pong of X recomputed in the reverse sweep
    const int *forced;                // replayed layer choices (device)
    const double *forced_alpha;       // replayed expansions a_n (device), or null
    int accel;                        // 1: accelerated chain from [gap_homo, gap_lumo]
    int pad_accel;
    double gap_homo, gap_lumo;
    float *xf[2];
    uint16_t *xop;                    // slot s: hi at xop + 2 s np^2, lo at xop + (2 s + 1) np^2
    float *yf[2];
    uint16_t *yop;                    // slot s in {0,1}: hi, lo as for xop
    Part *part[3];                    // by layer n mod 3 (three deep for the dataflow schedule)
    int part_cap, fin_blocks;
    const CUtensorMap *xmap;          // [nslots_x * MAPS_PER_SLOT]: per slot the K segments' loads op0, op1,
                                      // op2 = hi, hi, lo, then the epilogue's stores of hi and lo
    const CUtensorMap *ymap;          // [2 * MAPS_PER_SLOT]
    const double *H;                  // device copy of H (n x n)
    const double *H1;                 // response perturbation or adjoint weight (n x n)
    float *out;                       // D (n x n)
    float *out1;                      // D1 or dH (n x n)
    double2 *fin_part;                // finalisation partials
    InstCtl *ctl;
};

struct RunParams {
    InstDesc *inst;
    const int2 *tiles;                // (bi, bj) per tile, per instance slice
    unsigned int *barrier;            // grid barrier arrival counter (zeroed per launch)
    int *err;                         // first fatal device error (SP2_ERR_*), 0 = none
    double tol;
    unsigned long long timeout_ns;
    int B, mode, precision, max_layers;
    int test_hook;                    // 1: CTA 0 withholds its first barrier arrival (dataflow:
                                      // its first tile completion)
    int dataflow;                     // 1: no grid barrier between layers (see the tensor-core kernel)
    int publish;                      // 1: round schedule of a density batch, sums published per layer
    int nblk;                         // dataflow: 256-row blocks of X (round_up(np, 256) / 256)
    unsigned int *tile_done;          // dataflow: per tile, CTA completions over all layers
    unsigned int *layer_done;         // dataflow: CTA-tile completions over all layers
    const int *blk_src;               // dataflow: [nblk * nblk * 2] tiles writing block (P, Q) of X, -1 none
};

// Host-side launchers (one translation unit each).
cudaError_t launch_gershgorin(InstDesc *inst, int B, int max_n, bool user_bounds, cudaStream_t s);
cudaError_t launch_maxabs(InstDesc *inst, int B, int max_n, cudaStream_t s);
cudaError_t launch_init_x(InstDesc *inst, int B, int max_np, int path, int precision, bool user_bounds,
                          cudaStream_t s);
cudaError_t launch_init_x_from(InstDesc *inst, const float *X0, int np, int path, int precision, cudaStream_t s);
cudaError_t launch_init_y(InstDesc *inst, int mode, int precision, cudaStream_t s);
// Output kernel blocks per instance on the current device (the d.fin_blocks every
// instance of a launch is given, and the grid of launch_finalize).
int finalize_blocks();
cudaError_t launch_finalize(InstDesc *inst, int B, int fin_blocks, int mode, cudaStream_t s);
cudaError_t launch_fill_trivial(float *D, int n, float diag_value, cudaStream_t s);
cudaError_t launch_simt_persistent(const RunParams &p, int grid, cudaStream_t s);
cudaError_t launch_tc_persistent(const RunParams &p, int cta_group, int grid, cudaStream_t s);
int simt_blocks_per_sm();
int tc_grid_size(int cta_group, int sm_count);
size_t tc_smem_bytes();

inline int round_up(int a, int b) { return (a + b - 1) / b * b; }

}  // namespace sp2i
