// exact.h -- host interface of the exact-slice matrix products (exact_kernel.cu).
//
// The refinement layers of the chain (section "Deep-neural network electronic
// structure solver": a few final layers with X in double precision) and the
// congruences of the non-orthogonal route (section "The density matrix",
// H_orth = Z^T H Z, D = Z D_orth Z^T) need products accurate to FP64 level.
// They run on the FP16 tensor cores through an error-free splitting: every
// row of an operand is written, in fixed point relative to a power-of-two row
// scale, as a sum of small-integer slices
//     x = 2^e (a_0 2^-11 + a_1 2^-(11+b) + ... + a_{S-1} 2^-(11+(S-1)b)),
// |a_0| <= 2048 and |a_s| <= 2^(b-1) (all exactly representable in FP16).  A
// product of two slices is an integer matrix; the products of one "level"
// l = s + t are summed in one FP32 tensor-memory accumulator, where the sum of
// integers stays exact while its magnitude is below 2^24 (Cauchy-Schwarz bounds
// it by sum_{s+t=l} ||a_s row|| ||a_t row||; b is chosen so that this bound,
// for remainders spread like uniform noise, stays below 2^24 on every level
// but the last, whose rounding is below 2^-50 of the product).  The levels
// l < S are combined exactly in 64-bit integer arithmetic in the epilogue.
//
// Fixed-point conventions:
//   SP2 mode (the refinement layers):  Y = X - I/2 (identity on the first n
//     diagonal entries) has |Y_ij| <= 1/2, so one global scale serves every
//     row (e = -1, a_0 = round(2^12 Y)).  Y is carried between layers as an
//     int64 matrix in units of 2^-U, U = 24 + b (S - 1), the unit of the
//     product's last level, so that Y_{n+1} = Y_n +- (Y_n^2 - I/4) is exact
//     integer arithmetic on the computed product.  Only the lower triangle
//     (row >= column) of the int64 matrix is kept.
//   General mode (the congruences): per-row scales e_i with 2^e_i >= the row's
//     2-norm, so the product C = A B^T comes out as
//     C_ij = P_ij 2^(e^A_i + e^B_j - 22 - b (S - 1)), P_ij an exact integer.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace sp2i {

constexpr int XS_MAX_SLICES = 6;
constexpr int XS_TILE_M = 256;   // rows of a CTA-pair tile (128 per CTA)
constexpr int XS_TILE_N = 128;   // columns of a tile (UMMA N); four FP32 accumulators fill tensor memory

enum XsMode { XS_SP2 = 0, XS_GEN = 1, XS_GEN_SYM = 2 };

// Slices of one operand: slice s at base + s * np * np (16-bit, row-major,
// np x np), per-row exponents `exps` (general mode; null in SP2 mode).
struct XsOperand {
    uint16_t *base = nullptr;
    int *exps = nullptr;
};

// Slice bits b for S slices over a contraction of length K: the largest b for
// which every level's Cauchy-Schwarz bound, taking noise-like remainders
// (norm 2^b sqrt(K/12) per slice), stays below 2^24.
int xs_choose_beta(int slices, int K);

// Number of tiles of a product over np x np (upper-triangle tiles for the
// symmetric modes).
int xs_tile_count(int np, int mode);

// Bytes of device scratch xs_product needs for its partials (SP2 mode).
size_t xs_part_bytes(int np);

struct XsProduct {
    int mode = XS_SP2;
    int n = 0, np = 0;              // real size and padded size (multiple of 128)
    int slices = 6, beta = 6;
    XsOperand a, b;                 // b = a in SP2 mode
    // SP2 mode
    const long long *y_in = nullptr;  // Y_n, lower triangle, np x np
    long long *y_out = nullptr;       // Y_{n+1} (may be y_in: each element is read and
                                      // rewritten by the one thread that owns it)
    uint16_t *next_slices = nullptr;  // slices of Y_{n+1} (np x np each)
    const int *choice = nullptr;      // device: SP2_CHOICE_SQUARE / SP2_CHOICE_FLIP
    double2 *part = nullptr;          // per tile and CTA: (Tr Y_{n+1}, ||Y_{n+1}||_F^2)
    // general modes
    double *c = nullptr;              // n x n FP64 result, leading dimension n
    // all modes
    long long *scratch = nullptr;     // xs_scratch_bytes(grid_pairs): each CTA's tile products
    int *err = nullptr;               // first device error (SP2_ERR_*), 0 = none
    unsigned long long timeout_ns = 2000000000ull;
};

// Bytes of the per-CTA product scratch of a launch over `grid_pairs` CTA pairs.
size_t xs_scratch_bytes(int grid_pairs);

// One product on `s` (slices: 4, 5 or 6); returns the launch error.  The caller checks *err after
// the stream completes.
cudaError_t xs_product(const XsProduct &p, int grid_pairs, cudaStream_t s);
// CTA pairs the product kernel can keep resident (0 if it cannot run here).
int xs_resident_pairs(int sm_count);

// SP2 mode set-up: from the chain's FP32 output D (n x n, ld n) form Y_0 = D - I/2
// in fixed point (lower triangle), its slices, and the partials of its statistics.
cudaError_t xs_init_sp2(const float *D, int n, int np, int slices, int beta, long long *y, uint16_t *sl,
                        double2 *part, int *nparts, int *err, cudaStream_t s);
// Sum the partials, record (Tr X, ||X||_F^2, Tr X - ||X||_F^2) in rec[0..2] and pick the
// next layer's sign by the trace rule (X = Y + I/2).
cudaError_t xs_decide(const double2 *part, int nparts, int n, double n_occ, int *choice, double *rec,
                      cudaStream_t s);
// D = Y 2^-U + I/2 as FP64 n x n (ld n), both triangles, from the lower-triangle Y.
cudaError_t xs_finish_sp2(const long long *y, int n, int np, int slices, int beta, double *D, cudaStream_t s);

// General mode set-up: slices of M (n x n FP64, ld n) or of its transpose, with
// per-row exponents, padded to np x np.  `scratch` (n x n FP64) is used for the
// transpose.
cudaError_t xs_slice_rows(const double *M, bool transpose, int n, int np, int slices, int beta, XsOperand out,
                          double *scratch, int *err, cudaStream_t s);

// Pull the TMA encoder from the driver (false if unavailable).
bool xs_available();

}  // namespace sp2i
