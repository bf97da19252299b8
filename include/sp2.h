/*
 * sp2.h -- C ABI of libsp2, the GB300 (sm_103a) DNN-SP2 density-matrix library.
 *
 * The library maps an orthogonalised, symmetric N x N Hamiltonian H to the
 * zero-temperature density matrix D = theta(mu I - H) (section "The density
 * matrix", Eq. theta) by the deep-network form of the second-order spectral
 * projection chain (section "Deep-neural network electronic structure solver",
 * Eq. Deep_NN): X_0 = (eps_max I - H)/(eps_max - eps_min), then per layer
 * X_{n+1} = X_n^2 or 2 X_n - X_n^2, the sign chosen from traces so that Tr X
 * moves toward the occupation, until X is idempotent.  The matrix square is the
 * activation f(X) = X^2; in the split precisions it is evaluated from a
 * two-term 16-bit representation X = X^(0) + X^(1) with FP32 accumulation
 * (Eq. activ).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Matrices are dense, row-major, N x N, with leading dimension N.
 *  - Matrix pointers may be device pointers or host pointers (pageable or
 *    pinned); the library detects which and stages host data through device
 *    memory.  Pinned (page-locked, mapped) host memory is accessed in place
 *    across the host link: of H (and of a response's H1) only the lower
 *    triangle, diagonal included, is read, and the FP32 results D (D1, dH)
 *    are written there directly by the output kernel (the FP64 results of
 *    sp2_density_refined / sp2_density_nonorth are copied back).  Pageable host
 *    matrices, and the non-symmetric inputs G and Z, are copied whole.
 *    The caller owns every buffer it passes; the library frees none.
 *  - H must be symmetric (bit-exactly, as produced by (A + A^T)/2).  With the
 *    split precisions the chain reads only H's lower triangle, diagonal
 *    included (the bounds, the input layer and Tr[D H]), so its result for an
 *    asymmetric H is that of the symmetric matrix with H's lower triangle, as
 *    it is at any precision with pinned H; otherwise the result for an
 *    asymmetric H is unspecified but finite.
 *  - `n_occ` must be an integer value in [0, N].  n_occ = 0 gives D = 0 and
 *    n_occ = N gives D = I without layers.
 *  - `workspace` may be NULL, in which case the call allocates device memory
 *    and frees it before returning; otherwise it must be a device pointer of
 *    at least the size the matching *_workspace_bytes function returns,
 *    256-byte aligned.  Host-resident inputs, and pageable host outputs, are
 *    staged in the workspace beyond that size when it is large enough (8 bytes
 *    per FP64 and 4 per FP32 element, each piece rounded up to 256 bytes), else
 *    in memory the call allocates and frees.
 *  - Calls are stream-ordered on `stream` (a cudaStream_t; NULL = legacy
 *    default stream) and synchronise that stream before returning, because
 *    the status and the statistics are read back to the host.
 *  - A wait inside a kernel (the grid barrier between layers; in a single
 *    density solve, the wait for the tiles of the previous layer; a pipeline
 *    barrier) that exceeds `timeout_ms` makes the kernel stop and the call
 *    return SP2_ERR_TIMEOUT; no call leaves a kernel spinning.
 *  - Errors never leave partially written output undefined in size: on any
 *    status other than SP2_OK / SP2_ERR_NOT_CONVERGED the contents of the
 *    output matrices are unspecified.
 */
#ifndef SP2_H
#define SP2_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SP2_OK = 0,
    SP2_ERR_ARG = 1,            /* invalid argument (size, n_occ, pointer, option) */
    SP2_ERR_NONFINITE = 2,      /* H (or H1 / G) holds NaN, Inf or a magnitude >= 2^128 */
    SP2_ERR_NOT_CONVERGED = 3,  /* max_layers reached before the stop rule fired; output holds the last layer */
    SP2_ERR_TIMEOUT = 4,        /* a device-side wait gave up after timeout_ms */
    SP2_ERR_CUDA = 5,           /* a CUDA runtime or driver call failed */
    SP2_ERR_NOMEM = 6,          /* device or host allocation failed */
    SP2_ERR_UNSUPPORTED = 7     /* the device is not sm_103 or lacks a needed feature */
} sp2_status;

typedef enum {
    SP2_FP32_SIMT = 0,   /* X^2 with FP32 CUDA-core FMAs, FP32 storage */
    SP2_FP16_SPLIT = 1,  /* X = hi + lo in FP16 (lo kept scaled by 2^11), tensor cores, FP32 accumulation */
    SP2_BF16_SPLIT = 2   /* X = hi + lo in BF16, tensor cores, FP32 accumulation */
} sp2_precision;

/* Stop reasons (sp2_stats.stop_reason). */
#define SP2_STOP_NONE 0     /* the chain did not end by its own rule (forced sequence ran out) */
#define SP2_STOP_TOL 1      /* |Tr X - ||X||_F^2| <= tol */
#define SP2_STOP_STALL 2    /* |Tr X - ||X||_F^2| <= 1e-2 and no smaller than two layers earlier */
#define SP2_STOP_MAX 3      /* max_layers reached (status SP2_ERR_NOT_CONVERGED) */
#define SP2_STOP_TRIVIAL 4  /* n_occ = 0 or n_occ = N */

/* Layer choices (sp2_layer_stat.choice). */
#define SP2_CHOICE_INPUT (-1)  /* X_0 */
#define SP2_CHOICE_SQUARE 0    /* X_{n+1} = X_n^2 */
#define SP2_CHOICE_FLIP 1      /* X_{n+1} = 2 X_n - X_n^2 */

#define SP2_MAX_LAYERS_LIMIT 200

/* Statistics of one layer X_n, reduced in FP64 from the stored FP32 X_n. */
typedef struct {
    double trace;     /* Tr X_n */
    double trace_sq;  /* ||X_n||_F^2 = Tr X_n^2 for symmetric X_n */
    double idem;      /* Tr X_n - ||X_n||_F^2 = sum_i lambda_i (1 - lambda_i) */
    int choice;       /* SP2_CHOICE_* that produced X_n */
    int reserved;
    double alpha;     /* expansion a_n of the layer that produced X_n (1 in the plain chain
                         and for the input layer; see sp2_opts.accelerate) */
} sp2_layer_stat;

/* Result record, caller-owned host memory.  `layer` may be NULL; otherwise it
 * points to `layer_cap` entries and receives min(layers + 1, layer_cap) of them
 * (entry 0 is the input layer). */
typedef struct {
    int layers;            /* number of square layers applied */
    int stop_reason;       /* SP2_STOP_* */
    double eps_min;        /* spectral bounds used for X_0 */
    double eps_max;
    double band_energy;    /* Tr[D H] in FP64 from the FP32 D */
    double trace_D;        /* Tr D in FP64 from the FP32 D */
    sp2_layer_stat *layer;
    int layer_cap;
    int cta_group;         /* CTAs per tensor-core tile the call used (0 on the FP32 path) */
    float phase_ms[4];     /* with sp2_opts.profile: device time of [0] bounds + input layer
                              (+ response / adjoint stream start), [1] the persistent layer
                              kernel, [2] output copy and FP64 reductions, [3] all three;
                              CUDA events on the call's stream */
} sp2_stats;

/* Options; pass NULL for the defaults listed. */
typedef struct {
    int precision;        /* sp2_precision, default SP2_FP16_SPLIT */
    int max_layers;       /* default 100, at most SP2_MAX_LAYERS_LIMIT */
    double timeout_ms;    /* device wait limit, default 2000 */
    int user_bounds;      /* 0 = Gershgorin bounds (default), 1 = use eps_min / eps_max below */
    int test_hook;        /* 0 in normal use; 1 = CTA 0 withholds its first grid-barrier arrival, so
                             the barrier wait must run out (tests the timeout path); 2 = every
                             device allocation the call makes reports failure (host-side
                             injection; tests the SP2_ERR_NOMEM path); 3 = as 1 but in CTA-pair
                             launches only (a pair that never becomes resident; tests the retry
                             described under cta_group) */
    double eps_min;
    double eps_max;
    int profile;          /* 1 = record per-phase device times into sp2_stats.phase_ms */
    int cta_group;        /* tensor-core tiles: 0 = choose (default), 1 = one CTA per 128 x 256
                             tile (cooperative launch), 2 = a CTA pair per 256 x 256 tile
                             (M = 256 MMAs; a cluster launch sized to the pairs the device
                             holds at once: work running concurrently on the same GPU can
                             deny that residency, and the waits between layers then run out
                             after timeout_ms -- with cta_group = 0 the call is then retried once
                             with single-CTA tiles, with cta_group = 2 it returns
                             SP2_ERR_TIMEOUT; batch plans do not retry) */
    int accelerate;       /* 1 = accelerated chain from an estimated interval [eps_homo, eps_lumo]
                             between the highest occupied and lowest unoccupied eigenvalue
                             (section "GPU and tensor core performance" notes the saving of up
                             to half the layers and leaves the scheme out).  Reading: before each
                             layer X is expanded affinely, T = a X + (1 - a) I with
                             a = 2/(2 - x_lumo) before X^2 and T = a X with a = 2/(1 + x_homo)
                             before 2X - X^2, where x_lumo, x_homo are the images of eps_lumo,
                             eps_homo under the input layer and follow every layer; the branch is
                             still chosen by the trace rule.  The result is theta(mu I - H)
                             whenever the interval overlaps the gap, i.e. eps_lumo is above the
                             true HOMO and eps_homo below the true LUMO; the closer the interval
                             is to the gap, the fewer the layers.  Requires
                             eps_homo < eps_lumo (else SP2_ERR_ARG); sp2_density, sp2_response
                             and sp2_adjoint only (sp2_density_batched: SP2_ERR_ARG).  Response
                             and adjoint replay the forward run's a_n from its stats. */
    double eps_homo;
    double eps_lumo;
    int checkpoint_stride; /* sp2_adjoint only (ignored elsewhere): which forward layers keep their
                             operands for the reverse sweep.  0 = every layer (default; 4 bytes per
                             element per layer).  s >= 2 = every s-th layer X_0, X_s, X_2s, ...
                             (operands and FP32 master, 8 bytes per element each) and a ring of
                             s - 1 layers; the reverse sweep recomputes the layers between two kept
                             ones from the earlier, with the forward's own signs, offsets and
                             expansions, so the gradient is bit-identical to s = 0 at the cost of
                             up to (s - 1)/s of the forward's squares again.  -1 = the s that needs
                             the least memory for the chain's length.  A stride that would not
                             save memory keeps every layer.  Range -1 .. SP2_MAX_LAYERS_LIMIT. */
    int exact_slices;     /* sp2_density_refined, sp2_density_nonorth and sp2_congruence only: integer
                             slices per operand row in their exact-slice products, 4, 5 or 6 (0 = 6).
                             A row keeps 11 + b (S - 1) bits relative to its 2-norm (b = 6 bits per
                             further slice up to N = 8192, fewer above); the products take 10, 15 or
                             21 slice products per tile: fewer slices are faster and less accurate
                             (S = 4: about 2^-29 of the row norms, 5: 2^-35, 6: 2^-41). */
} sp2_opts;

/* Fill `o` with the defaults. */
void sp2_default_opts(sp2_opts *o);

/* Human-readable name of a status code (static storage). */
const char *sp2_status_string(sp2_status s);

/* Device bytes sp2_density needs as workspace for size N (device-resident H and D). */
size_t sp2_density_workspace_bytes(int N, const sp2_opts *o);

/*
 * sp2_density -- D = theta(mu I - H) by the DNN-SP2 chain.
 *   H      [in]  N x N symmetric, FP64.
 *   N      [in]  matrix size, 1 <= N <= 65536.
 *   n_occ  [in]  number of occupied states (integer value).
 *   tol    [in]  stop when |Tr X_n - ||X_n||_F^2| <= tol (the paper's trace-based
 *                idempotency estimate, section "GPU and tensor core performance").
 *   D      [out] N x N FP32, the last layer X_L.
 *   st     [out] statistics (may be NULL).
 * Returns SP2_OK when the stop rule fired, SP2_ERR_NOT_CONVERGED when max_layers
 * was reached (D holds X_max), or an error.
 */
sp2_status sp2_density(const double *H, int N, double n_occ, double tol, float *D,
                       sp2_stats *st, const sp2_opts *o, void *workspace, size_t ws_bytes,
                       void *stream);

/* Device bytes sp2_response needs as workspace. */
size_t sp2_response_workspace_bytes(int N, const sp2_opts *o);

/*
 * sp2_response -- first-order response D1 = dD/dH [H1] of the chain.
 * The chain is differentiated layer by layer with the layer signs held fixed:
 * X1_0 = -H1/(eps_max - eps_min), and per layer with C = X_n X1_n,
 * X1_{n+1} = C + C^T (X^2 layers) or 2 X1_n - (C + C^T) (2X - X^2 layers).
 * The forward chain runs alongside and takes its own decisions exactly as
 * sp2_density does, unless `fwd` (statistics of an earlier sp2_density call on
 * the same H, with its `layer` array filled) is given: then the forward replays
 * fwd's layer sequence and bounds.  The paper gives no response; this is the
 * derivative of its chain.
 *   H1  [in]  N x N symmetric FP64 perturbation.
 *   D   [out] N x N FP32 density matrix (may be NULL).
 *   D1  [out] N x N FP32 response.
 */
sp2_status sp2_response(const double *H, const double *H1, int N, double n_occ, double tol,
                        const sp2_stats *fwd, float *D, float *D1, sp2_stats *st,
                        const sp2_opts *o, void *workspace, size_t ws_bytes, void *stream);

/* Device bytes sp2_adjoint needs for a chain of `layers` layers (0 = o->max_layers),
 * with o->checkpoint_stride taken into account. */
size_t sp2_adjoint_workspace_bytes(int N, int layers, const sp2_opts *o);

/*
 * sp2_adjoint -- gradient dTr[D G]/dH of the chain, by reverse accumulation.
 * Runs the forward chain storing every layer's split operands, or every s-th
 * with o->checkpoint_stride = s and the others recomputed during the reverse
 * sweep (replaying `fwd` when given, else deciding as sp2_density; storage is
 * sized for fwd->layers, else for o->max_layers), then G_L = (G + G^T)/2 and, for
 * the layer that made X_{n+1} from X_n, G_n = G_{n+1} X_n + X_n G_{n+1} (X^2)
 * or 2 G_{n+1} - (G_{n+1} X_n + X_n G_{n+1}) (2X - X^2), and returns
 * dH = -G_0/(eps_max - eps_min).  Layer signs and bounds are held constant.
 *   G   [in]  N x N FP64 weight (need not be symmetric).
 *   dH  [out] N x N FP32 gradient (symmetric).
 */
sp2_status sp2_adjoint(const double *H, const double *G, int N, double n_occ, double tol,
                       const sp2_stats *fwd, float *D, float *dH, sp2_stats *st,
                       const sp2_opts *o, void *workspace, size_t ws_bytes, void *stream);

/* Device bytes sp2_density_batched needs. */
size_t sp2_density_batched_workspace_bytes(int B, const int *N, const sp2_opts *o);

/*
 * sp2_density_batched -- B independent chains in one persistent grouped launch.
 * H[b], D[b] are per-instance pointers (host arrays of B pointers, each matrix
 * device- or host-resident as above), N[b] and n_occ[b] per instance, st[b]
 * per-instance statistics (st may be NULL).  Every instance takes its own layer
 * sequence; an instance that has stopped drops out of the schedule.  Returns
 * the worst status over the instances (errors before NOT_CONVERGED).
 */
sp2_status sp2_density_batched(int B, const double *const *H, const int *N, const double *n_occ,
                               double tol, float *const *D, sp2_stats *st, const sp2_opts *o,
                               void *workspace, size_t ws_bytes, void *stream);

/*
 * Batch plans: the batched solve set up once and launched many times.
 *
 * Quantum-based MD rebuilds one density matrix per Hamiltonian at every time step
 * (section "Microcanonical MD"), so a batch of snapshots or replicas of fixed sizes
 * is solved over and over.  A plan fixes the instance sizes, occupations, device
 * buffers (H[b] read, D[b] written), tolerance and options once, and owns its
 * workspace.  sp2_batch_plan_launch then only enqueues device work on `stream`:
 * a reset of the control blocks (device-to-device copy), a memset, and the same
 * kernels as sp2_density_batched -- no allocation, no host copy, no host
 * synchronisation.  A caller may therefore capture it in a CUDA graph and replay
 * the graph after writing new Hamiltonians into the same H buffers.
 *
 * sp2_batch_plan_create: arguments as sp2_density_batched, but every H[b] and D[b]
 * must be device memory (else SP2_ERR_ARG); sp2_opts.accelerate is rejected.
 * With autotune = 1 and o->cta_group = 0 on a split precision, create times one
 * solve with each tensor-core tile shape (CTA pairs, single CTAs) on these inputs
 * and keeps the faster; the choice is cached per (precision, sizes) for the life
 * of the process, so later plans of the same shape skip the timing.  Create runs
 * (and synchronises) on `stream`; tuning writes D.  *plan receives the handle.
 * sp2_batch_plan_launch: enqueue one solve of every instance on `stream`.
 * sp2_batch_plan_stats: wait for the stream, then fill st[0..B-1] from the last
 * launch (st may be NULL); returns the worst status as sp2_density_batched.
 * sp2_batch_plan_cta_group: tile shape the plan uses (1, 2; 0 on the FP32 path).
 * sp2_batch_plan_destroy: free the plan and its workspace (NULL is ignored); the
 * caller must not destroy a plan with launches in flight.
 * A plan is used by one host thread at a time; overlapping launches of the same
 * plan on different streams share its workspace and race.
 */
typedef struct sp2_batch_plan sp2_batch_plan;

sp2_status sp2_batch_plan_create(int B, const double *const *H, const int *N, const double *n_occ, double tol,
                                 float *const *D, const sp2_opts *o, int autotune, void *stream,
                                 sp2_batch_plan **plan);
sp2_status sp2_batch_plan_launch(sp2_batch_plan *plan, void *stream);
sp2_status sp2_batch_plan_stats(sp2_batch_plan *plan, sp2_stats *st, void *stream);
int sp2_batch_plan_cta_group(const sp2_batch_plan *plan);
void sp2_batch_plan_destroy(sp2_batch_plan *plan);

/*
 * sp2_apply_layers -- apply a given layer sequence to a given X_0 (test and
 * tooling entry point: the matrix-square kernel without the input layer).
 *   X0       [in]  N x N FP32 symmetric start matrix.  With SP2_FP16_SPLIT its entries
 *                   must stay below 32 in magnitude (the split stores hi * 2^11 in FP16);
 *                   a matrix with its spectrum in [0, 1], as every X_n of the chain, has
 *                   entries of magnitude at most 1.
 *   choices  [in]  host array of n_layers SP2_CHOICE_SQUARE / SP2_CHOICE_FLIP.
 *   X        [out] N x N FP32 result X_{n_layers}.
 *   st       [out] per-layer traces (stop fields unused).
 */
sp2_status sp2_apply_layers(const float *X0, int N, const int *choices, int n_layers, float *X,
                            sp2_stats *st, const sp2_opts *o, void *stream);

/*
 * sp2_density_refined -- the chain of sp2_density followed by `refine_layers`
 * further layers with X held in FP64 (section "Deep-neural network electronic
 * structure solver": extra layers with a double-precision representation of X
 * act as a refinement that purifies the eigenvalues closer to 1 and 0).  Each
 * refinement layer takes its sign by the same trace rule, decided on the device.
 * The refinement squares are exact-slice products on the FP16 tensor cores:
 * Y = X - I/2 is carried in 64-bit fixed point (units of 2^-54 up to N = 8192)
 * and split into six small-integer slices (an 11-bit leading slice, then 6 bits
 * each: about 2^-41 of the row norms); the slice products are integer matrices
 * summed exactly in the FP32 accumulators and combined in 64-bit integer
 * arithmetic, so a layer's square is accurate to about 1e-13 per element.
 *   refine_layers [in]  0 .. 8 (the paper uses two).
 *   D             [out] N x N FP64, the refined density matrix.
 *   st            [out] the chain's layers followed by the refinement layers;
 *                       trace_D and band_energy from the FP64 result; with
 *                       o->profile, phase_ms holds the device time of [0] the
 *                       chain (and sp2_density_nonorth's first congruence), [1] the
 *                       refinement layers, [2] the back-transformation and the FP64
 *                       Tr[D H], [3] all of it (CUDA events on the call's stream).
 * Allocates device memory for the FP64 and fixed-point matrices (about 50 bytes
 * per element) and for the chain's workspace, all before the first timed phase,
 * and frees it before returning.
 * Returns SP2_ERR_NOT_CONVERGED also when X leaves [-2^-13, 1 + 2^-13]
 * spectrally during the refinement (its slices could not hold it exactly).
 */
sp2_status sp2_density_refined(const double *H, int N, double n_occ, double tol, int refine_layers, double *D,
                               sp2_stats *st, const sp2_opts *o, void *stream);

/*
 * sp2_density_nonorth -- density matrix in a non-orthogonal basis (section "The
 * density matrix"): with Z an inverse factor of the overlap S (Z^T S Z = I),
 * H_orth = Z^T H Z, D_orth = theta(mu I - H_orth) by the chain (plus
 * `refine_layers` FP64 layers), and D = Z D_orth Z^T.  The congruences are
 * sp2_congruence's products.  D does not depend on which Z is given.
 *   Z [in]  N x N FP64, row-major.
 *   D [out] N x N FP64; band_energy = Tr[D H].
 */
sp2_status sp2_density_nonorth(const double *H, const double *Z, int N, double n_occ, double tol,
                               int refine_layers, double *D, sp2_stats *st, const sp2_opts *o, void *stream);

/*
 * sp2_congruence -- the orthogonalisation step of section "The density matrix":
 *   side = 0: out = Z^T M Z  (H_orth from H in a non-orthogonal basis),
 *   side = 1: out = Z M Z^T  (D from D_orth).
 * Z, M, out: N x N FP64, row-major, device memory; M symmetric; out is exactly
 * symmetric (its lower triangle mirrors the upper).  Both products are
 * exact-slice products on the FP16 tensor cores: every row of an operand is
 * scaled by a power of two at or above its 2-norm and split into six
 * small-integer slices whose products are summed exactly in the FP32
 * accumulators, so each entry of a product is accurate to about 2^-41 of the
 * product of its row's and column's 2-norms.  Allocates about 60 bytes per
 * element of device memory for the call.  Returns SP2_ERR_ARG for host pointers
 * or side not in {0, 1}.
 */
sp2_status sp2_congruence(const double *Z, const double *M, int N, int side, double *out, const sp2_opts *o,
                          void *stream);

/*
 * sp2_density_noalloc -- sp2_density without any device allocation.
 * The paper has no counterpart: this entry point exists for callers that must
 * not allocate device memory once running, such as an MD engine whose memory
 * is reserved by its own pool or by another framework's caching allocator (a
 * new allocation can fail or fragment it), or a step loop that cannot afford
 * an allocation's latency.  The workspace is a statically allocated device
 * array of 6 MiB, which holds one solve of N <= SP2_NOALLOC_MAX_N.  A GPU holds
 * it, until the process exits, from the moment the library's device code is
 * loaded there: with lazy module loading (the CUDA default) that is the first
 * call of this entry point on the device, so make that call before reserving
 * the rest of the device's memory (it returns SP2_ERR_NOMEM if the array cannot
 * be placed then).
 *   H, D   must be device pointers (staging host data would allocate);
 *          arguments and results are those of sp2_density.
 *   o      may be NULL; o->profile must be 0.
 * Returns SP2_ERR_ARG for N > SP2_NOALLOC_MAX_N, host pointers or profiling.
 * The first call on a device looks up the array's device address (with that
 * device current); make that first call before any stream capture.
 * Every call uses the same array: calls whose work overlaps on the GPU (on
 * different streams, or from different host threads) race and corrupt each
 * other's results, so serialise them.  Each call initialises the parts of the
 * array that must start at zero, so no state carries over between calls.
 */
#define SP2_NOALLOC_MAX_N 512
sp2_status sp2_density_noalloc(const double *H, int N, double n_occ, double tol, float *D,
                               sp2_stats *st, const sp2_opts *o, void *stream);

/* Number of streaming multiprocessors and whether the current device runs this
 * library's kernels (compute capability 10.3). */
sp2_status sp2_device_info(int *sm_count, int *cc_major, int *cc_minor);

#ifdef __cplusplus
}
#endif

#endif /* SP2_H */
