// api.cu -- the C ABI declared in include/sp2.h.
//
// Every entry point goes through one runner: validate, lay out the workspace,
// stage host matrices, encode the TMA tensor maps, launch
//   Gershgorin bounds -> input layer -> [response / adjoint stream start]
//   -> one cooperative persistent kernel for all layers -> output copy + FP64
//   Tr[DH], Tr D
// on the caller's stream, then read the per-instance control blocks back.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "device_common.cuh"
#include "host_link.h"

using namespace sp2i;

namespace {

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn get_encode_fn() {
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)p;
    });
    return fn;
}

// 2-D map over an np x np 16-bit matrix, box 64 (K, inner) x 128 rows, 128B swizzle.
bool encode_op_map(CUtensorMap *m, const void *base, int np, int precision) {
    EncodeTiledFn fn = get_encode_fn();
    if (!fn) return false;
    cuuint64_t dims[2] = {(cuuint64_t)np, (cuuint64_t)np};
    cuuint64_t strides[1] = {(cuuint64_t)np * 2};
    cuuint32_t box[2] = {(cuuint32_t)TC_BK, (cuuint32_t)(TC_BN / 2)};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(m, precision == SP2_BF16_SPLIT ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2,
                    const_cast<void *>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

// 2-D map over an np x np 16-bit matrix for the epilogue's stores: box EPI_BOX_COLS
// x EPI_BOX_ROWS, no swizzle (the box sits row-major in shared memory).
bool encode_store_map(CUtensorMap *m, const void *base, int np) {
    EncodeTiledFn fn = get_encode_fn();
    if (!fn) return false;
    cuuint64_t dims[2] = {(cuuint64_t)np, (cuuint64_t)np};
    cuuint64_t strides[1] = {(cuuint64_t)np * 2};
    cuuint32_t box[2] = {(cuuint32_t)EPI_BOX_COLS, (cuuint32_t)EPI_BOX_ROWS};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_UINT16, 2, const_cast<void *>(base), dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

// The MAPS_PER_SLOT maps of one operand slot (matrices hi at `hi`, lo at hi + np^2).
bool encode_slot_maps(CUtensorMap *m, const uint16_t *hi, int np, int precision) {
    const size_t mat = (size_t)np * np;
    for (int k = 0; k < 3; ++k)
        if (!encode_op_map(&m[k], hi + (k == 2 ? mat : 0), np, precision)) return false;
    return encode_store_map(&m[3], hi, np) && encode_store_map(&m[4], hi + mat, np);
}

struct DeviceInfo {
    int sm = 0, major = 0, minor = 0;
    cudaError_t err = cudaSuccess;
};

DeviceInfo query_device() {
    DeviceInfo di;
    int dev = 0;
    di.err = cudaGetDevice(&dev);
    if (di.err != cudaSuccess) return di;
    di.err = cudaDeviceGetAttribute(&di.sm, cudaDevAttrMultiProcessorCount, dev);
    if (di.err != cudaSuccess) return di;
    di.err = cudaDeviceGetAttribute(&di.major, cudaDevAttrComputeCapabilityMajor, dev);
    if (di.err != cudaSuccess) return di;
    di.err = cudaDeviceGetAttribute(&di.minor, cudaDevAttrComputeCapabilityMinor, dev);
    return di;
}

sp2_opts resolve_opts(const sp2_opts *o) {
    sp2_opts r;
    sp2_default_opts(&r);
    if (o) r = *o;
    return r;
}

struct InstSpec {
    int n = 0;
    double n_occ = 0;
    const double *H = nullptr;
    const double *H1 = nullptr;    // response H1 / adjoint G
    const float *X0 = nullptr;     // apply mode
    float *D = nullptr;
    float *D1 = nullptr;
    sp2_stats *st = nullptr;
    const sp2_stats *fwd = nullptr;
    const int *choices = nullptr;  // apply mode (host)
    int nchoices = -1;
};

// Device allocation owned by one call; freed on every exit path.  With `fail`
// set (sp2_opts.test_hook = 2, host-side fault injection) every allocation
// reports failure, as an exhausted device would.
struct Arena {
    std::vector<void *> ptrs;
    cudaStream_t s;
    bool fail = false;
    explicit Arena(cudaStream_t st) : s(st) {}
    void *get(size_t bytes) {
        void *p = nullptr;
        if (bytes == 0) bytes = 256;
        if (fail) return nullptr;
        if (cudaMallocAsync(&p, bytes, s) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        ptrs.push_back(p);
        return p;
    }
    ~Arena() {
        for (void *p : ptrs) cudaFreeAsync(p, s);
        cudaStreamSynchronize(s);
    }
};

struct Carver {
    uint8_t *base;
    size_t off = 0;
    explicit Carver(void *b) : base((uint8_t *)b) {}
    void *take(size_t bytes) {
        off = (off + 255) & ~(size_t)255;
        void *p = base ? base + off : nullptr;
        off += bytes;
        return p;
    }
};

// Tile tables: SIMT uses square 128-tiles with bi <= bj; the tensor-core path
// uses 128 x 256 tiles containing at least one element with row <= column.
// CTA b takes tiles b, b + grid, ..., so each run of `grid` consecutive tiles is
// in flight together.  Tiles are ordered by 2048 x 2048 super-blocks (column
// super-block, then row super-block, then column, then row) so that such a run
// reads a compact set of row and column panels and the operand matrices, which
// are larger than L2, are fetched from HBM about once per run.
void build_tiles_uncached(int path, int np, int cg, std::vector<int2> &t) {
    const int bm = (path == PATH_SIMT) ? SIMT_T : TC_BM * cg;
    const int bn = (path == PATH_SIMT) ? SIMT_T : TC_BN;
    const int nbi = (np + bm - 1) / bm, nbj = (np + bn - 1) / bn;  // a last pair tile may overhang np
    const int sbi = 2048 / bm, sbj = 2048 / bn;  // tiles per super-block side
    std::vector<std::pair<long long, int2>> keyed;
    for (int bj = 0; bj < nbj; ++bj)
        for (int bi = 0; bi < nbi && bi * bm < (bj + 1) * bn; ++bi) {
            const long long key = (((long long)(bj / sbj) * 4096 + bi / sbi) * 4096 + bj) * 4096 + bi;
            keyed.push_back({key, make_int2(bi, bj)});
        }
    std::sort(keyed.begin(), keyed.end(), [](const std::pair<long long, int2> &a, const std::pair<long long, int2> &b) {
        return a.first < b.first;
    });
    for (auto &k : keyed) t.push_back(k.second);
}

// The table for (path, np, cg) is built once per process (calls repeat the same sizes).
void build_tiles(int path, int np, int cg, std::vector<int2> &t) {
    static std::mutex mu;
    static std::map<long long, std::vector<int2>> cache;
    const long long key = ((long long)path * 4 + cg) * (1LL << 32) + np;
    std::lock_guard<std::mutex> lock(mu);
    auto it = cache.find(key);
    if (it == cache.end()) {
        std::vector<int2> v;
        build_tiles_uncached(path, np, cg, v);
        it = cache.emplace(key, std::move(v)).first;
    }
    t.insert(t.end(), it->second.begin(), it->second.end());
}

// Number of tiles of the table above, counted without building it.
int ntiles_for(int path, int np, int cg) {
    const int bm = (path == PATH_SIMT) ? SIMT_T : TC_BM * cg;
    const int bn = (path == PATH_SIMT) ? SIMT_T : TC_BN;
    const int nbi = (np + bm - 1) / bm, nbj = (np + bn - 1) / bn;
    int count = 0;
    for (int bj = 0; bj < nbj; ++bj) count += std::min(nbi, ((bj + 1) * bn + bm - 1) / bm);
    return count;
}

// Partial records per layer: one per tile, per CTA of the tile.
int parts_for(int path, int np, int cg) { return ntiles_for(path, np, cg) * (path == PATH_TC ? cg : 1); }

// Must equal the device-side init_blocks_for: one partial per input-layer block.
int init_blocks_host(int np) { return np < INIT_BLOCKS_MAX ? np : INIT_BLOCKS_MAX; }

struct Plan {
    int mode, path, precision;
    bool dataflow = false;            // see flow_eligible
    int cg = 1;                       // CTAs per tensor-core tile
    std::vector<InstSpec> inst;       // non-trivial instances, in launch order
    std::vector<int> slots;           // nslots_x per instance
    std::vector<int> ckpt_s, ckpt_k;  // adjoint checkpoint stride and kept layers (0: every layer kept)
    int max_np = 0, max_n = 0;
};

// The dataflow schedule of the tensor-core kernel (no grid barrier between layers)
// serves one instance in density mode; it keeps three operand slots, so that a layer's
// operands are not overwritten while a slow CTA may still load them.
bool flow_eligible(const Plan &pl) { return pl.mode == MODE_DENSITY && pl.path == PATH_TC && pl.inst.size() == 1; }
void set_flow(Plan &pl) {
    pl.dataflow = flow_eligible(pl);
    if (pl.dataflow) pl.slots[0] = 3;
}

// Blocks of 256 x 256 of an np x np X and, per block, the (at most two) tiles that
// write its elements, directly or as mirrors; -1 where none.
int flow_nblk(int np) { return (np + 255) / 256; }
void build_block_sources(int np, int cg, const std::vector<int2> &tiles, std::vector<int> &src) {
    const int nb = flow_nblk(np), bm = TC_BM * cg;
    src.assign((size_t)nb * nb * 2, -1);
    auto add = [&](int P, int Q, int t) {
        int *e = &src[((size_t)P * nb + Q) * 2];
        if (e[0] < 0) e[0] = t;
        else if (e[1] < 0 && e[0] != t) e[1] = t;
    };
    for (int t = 0; t < (int)tiles.size(); ++t) {
        const int P = tiles[t].x * bm / 256, Q = tiles[t].y;
        add(P, Q, t);
        if (P != Q) add(Q, P, t);
    }
}

// Operand storage of an adjoint whose forward chain has at most `lmax` layers:
// every X_n (lmax + 1 slots), or with checkpoint stride s the K = lmax/s + 1 kept
// X_{ks} (slot + FP32 master each) plus a ring of s - 1 slots and two FP32
// matrices for the recomputed layers.  stride -1 picks the s of least memory;
// a stride that would not save memory keeps every layer.  A slot is two 16-bit
// matrices (hi, lo), an FP32 master one 32-bit matrix: 4 bytes per element each.
void adjoint_layout(int lmax, int stride, int &slots, int &s_out, int &k_out) {
    slots = lmax + 1;
    s_out = 0;
    k_out = 0;
    auto cost = [&](int s) {  // in units of np^2 bytes: 4 per slot, 4 per FP32 master
        const int k = lmax / s + 1;
        return 4 * (k + s - 1) + 4 * k + 8;
    };
    int s = stride;
    if (stride < 0) {
        s = 0;
        for (int c = 2; c <= lmax; ++c)
            if (s == 0 || cost(c) < cost(s)) s = c;
    }
    if (s < 2 || s > lmax || cost(s) >= 4 * (lmax + 1)) return;
    s_out = s;
    k_out = lmax / s + 1;
    slots = k_out + s - 1;
}

size_t plan_bytes(const Plan &pl, std::vector<size_t> *offsets_unused = nullptr) {
    (void)offsets_unused;
    Carver c(nullptr);
    const int B = (int)pl.inst.size();
    // The upload region (the order of prepare()): what the host writes before a launch.
    c.take(64);                           // barrier, error word, dataflow layer counter
    c.take(sizeof(InstCtl) * B);          // control blocks
    c.take(sizeof(InstCtl) * B);          // their initial state, copied in before every replay
    c.take(sizeof(InstDesc) * B);
    int tiles = 0;
    for (auto &s : pl.inst) tiles += ntiles_for(pl.path, round_up(s.n, PAD), pl.cg);
    c.take(sizeof(int2) * tiles);
    c.take(sizeof(int) * (MAX_L + 1));    // forced choices
    c.take(sizeof(double) * (MAX_L + 1)); // forced expansions
    for (int i = 0; i < B; ++i) {
        const int np = round_up(pl.inst[i].n, PAD);
        if (pl.dataflow) {
            c.take(sizeof(unsigned int) * ntiles_for(pl.path, np, pl.cg));      // tile completions
            c.take(sizeof(int) * 2 * (size_t)flow_nblk(np) * flow_nblk(np));  // block sources
        }
        if (pl.path == PATH_TC) {
            c.take((size_t)pl.slots[i] * MAPS_PER_SLOT * sizeof(CUtensorMap));
            if (pl.mode == MODE_RESPONSE || pl.mode == MODE_ADJOINT) c.take(2 * MAPS_PER_SLOT * sizeof(CUtensorMap));
        }
    }
    const int initb = init_blocks_host(pl.max_np);
    for (int i = 0; i < B; ++i) {
        const int np = round_up(pl.inst[i].n, PAD);
        const size_t mat = (size_t)np * np;
        const int cap = std::max(parts_for(pl.path, np, pl.cg), initb);
        c.take(sizeof(Part) * cap);
        c.take(sizeof(Part) * cap);
        c.take(sizeof(Part) * cap);
        c.take(sizeof(double2) * FIN_BLOCKS_MAX);
        c.take(mat * 4);
        c.take(mat * 4);
        if (pl.path == PATH_TC) {
            c.take((size_t)pl.slots[i] * 2 * mat * 2);
            if (pl.ckpt_s[i] > 0) {
                c.take((size_t)pl.ckpt_k[i] * mat * 4);
                c.take(mat * 4);
                c.take(mat * 4);
            }
            if (pl.mode == MODE_RESPONSE || pl.mode == MODE_ADJOINT) {
                c.take(mat * 4);
                c.take(mat * 4);
                c.take(2 * 2 * mat * 2);
            }
        }
    }
    return c.off + 256;
}

void fill_stats(sp2_stats *st, const InstCtl &ctl) {
    if (!st) return;
    st->layers = ctl.layers;
    st->stop_reason = ctl.stop_reason;
    st->eps_min = ctl.eps_min;
    st->eps_max = ctl.eps_max;
    st->band_energy = ctl.band_energy;
    st->trace_D = ctl.trace_D;
    if (st->layer && st->layer_cap > 0) {
        const int cnt = std::min(ctl.layers + 1, st->layer_cap);
        for (int k = 0; k < cnt; ++k) {
            st->layer[k].trace = ctl.stat[k].trace;
            st->layer[k].trace_sq = ctl.stat[k].trace_sq;
            st->layer[k].idem = ctl.stat[k].idem;
            st->layer[k].choice = ctl.stat[k].choice;
            st->layer[k].reserved = 0;
            st->layer[k].alpha = ctl.stat[k].alpha;
        }
    }
}

void fill_trivial_stats(sp2_stats *st, int n, double n_occ) {
    if (!st) return;
    st->layers = 0;
    st->stop_reason = SP2_STOP_TRIVIAL;
    st->eps_min = st->eps_max = 0.0;
    st->band_energy = 0.0;  // filled by the caller when H is at hand
    st->trace_D = n_occ;
    (void)n;
    if (st->layer && st->layer_cap > 0) {
        st->layer[0].trace = n_occ;
        st->layer[0].trace_sq = n_occ;
        st->layer[0].idem = 0.0;
        st->layer[0].choice = SP2_CHOICE_INPUT;
        st->layer[0].reserved = 0;
        st->layer[0].alpha = 1.0;
    }
}

int status_rank(int s) {
    // errors first, then NOT_CONVERGED, then OK
    if (s == SP2_OK) return 0;
    if (s == SP2_ERR_NOT_CONVERGED) return 1;
    return 2;
}

#define CK(x)                                  \
    do {                                       \
        cudaError_t e_ = (x);                  \
        if (e_ != cudaSuccess) {               \
            cudaGetLastError();                \
            return SP2_ERR_CUDA;               \
        }                                      \
    } while (0)

// Everything one launch of the path needs, laid out in device memory.  prepare()
// builds and uploads it, enqueue() puts one solve on a stream (device work only:
// control-block reset, barrier reset, kernels -- so it can be captured in a CUDA
// graph and replayed), collect() reads the control blocks back.
struct Prepared {
    Plan pl;
    sp2_opts o;
    double tol = 0.0;
    int grid = 0;
    bool user_bounds = false;
    InstDesc *d_inst = nullptr;
    int2 *d_tiles = nullptr;
    uint8_t *d_sync = nullptr;       // grid barrier counter, error word, dataflow layer counter
    unsigned int *d_tile_done = nullptr;   // dataflow: per-tile completion counters
    int *d_blk_src = nullptr;              // dataflow: block sources
    int flow_tiles = 0, flow_nb = 0;
    int fin_blocks = 0;              // output kernel blocks per instance
    InstCtl *d_ctl = nullptr;        // B live control blocks
    InstCtl *d_ctl_init = nullptr;   // B initial control blocks
    std::vector<InstCtl> h_ctl;
    std::vector<uint8_t> h_upload;   // host image of the upload region
    std::vector<uint8_t> h_back;     // barrier and error words and control blocks, read back
    std::vector<std::pair<float *, float *>> copy_back;  // (host, device staging)
    std::vector<size_t> copy_back_n;
};

// Tensor-core tile shape and persistent grid for the plan: CTA pairs (M = 256)
// when the device can co-schedule them, else single CTAs; `want` forces one.
// Per device: its attributes and the persistent grid of each tile shape, queried
// once per process (the occupancy queries cost more than a small solve's setup).
struct LaunchGeometry {
    bool known = false;
    DeviceInfo di;
    int grid_cg[3] = {0, 0, 0};
    int simt_per_sm = 0;
};
bool launch_geometry(LaunchGeometry &g) {
    static std::mutex mu;
    static LaunchGeometry table[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) {
        cudaGetLastError();
        return false;
    }
    std::lock_guard<std::mutex> lock(mu);
    LaunchGeometry local;
    LaunchGeometry &e = dev < 64 ? table[dev] : local;
    if (!e.known) {
        e.di = query_device();
        if (e.di.err != cudaSuccess) return false;
        if (e.di.major == 10 && e.di.minor == 3) {
            e.grid_cg[2] = tc_grid_size(2, e.di.sm);
            e.grid_cg[1] = tc_grid_size(1, e.di.sm);
            e.simt_per_sm = simt_blocks_per_sm();
        }
        e.known = true;
    }
    g = e;
    return true;
}

sp2_status choose_launch(Plan &pl, int want, int &grid) {
    LaunchGeometry geo;
    if (!launch_geometry(geo)) return SP2_ERR_CUDA;
    const DeviceInfo &di = geo.di;
    if (di.major != 10 || di.minor != 3) return SP2_ERR_UNSUPPORTED;
    if (pl.path == PATH_TC && !get_encode_fn()) return SP2_ERR_UNSUPPORTED;
    grid = 0;
    if (pl.path == PATH_TC) {
        if (want == 0 || want == 2) {
            grid = geo.grid_cg[2];
            pl.cg = 2;
        }
        if (grid <= 0) {
            if (want == 2) return SP2_ERR_UNSUPPORTED;
            grid = geo.grid_cg[1];
            pl.cg = 1;
        }
        if (grid <= 0) return SP2_ERR_UNSUPPORTED;
    } else {
        const int per_sm = geo.simt_per_sm;
        if (per_sm <= 0) return SP2_ERR_UNSUPPORTED;
        grid = per_sm * di.sm;
    }
    return SP2_OK;
}

// Lay out the workspace (`ws`, at least plan_bytes(pl) bytes), build the
// descriptors, tile tables and tensor maps and upload them with the initial
// control blocks.  Host-resident matrices are staged through device memory
// (the workspace tail, else `arena`) when `staging_ok`; otherwise they are an
// argument error.
sp2_status prepare(Prepared &P, const sp2_opts &o, double tol, void *ws, size_t ws_bytes, cudaStream_t s,
                   Arena &arena, bool staging_ok) {
    Plan &pl = P.pl;
    P.o = o;
    P.tol = tol;
    const int B = (int)pl.inst.size();
    Carver c(ws);
    // The upload region comes first and is contiguous: one host-to-device copy
    // writes all of it (the zeroed counters included).  The control blocks follow
    // the barrier and error word, so that one copy also reads both back.
    uint8_t *d_sync = (uint8_t *)c.take(64);
    InstCtl *d_ctl = (InstCtl *)c.take(sizeof(InstCtl) * B);
    InstCtl *d_ctl_init = (InstCtl *)c.take(sizeof(InstCtl) * B);
    InstDesc *d_inst = (InstDesc *)c.take(sizeof(InstDesc) * B);
    std::vector<std::vector<int2>> tiles(B);
    int total_tiles = 0;
    for (int i = 0; i < B; ++i) {
        build_tiles(pl.path, round_up(pl.inst[i].n, PAD), pl.cg, tiles[i]);
        total_tiles += (int)tiles[i].size();
    }
    int2 *d_tiles = (int2 *)c.take(sizeof(int2) * total_tiles);
    int *d_forced = (int *)c.take(sizeof(int) * (MAX_L + 1));
    double *d_forced_alpha = (double *)c.take(sizeof(double) * (MAX_L + 1));
    std::vector<CUtensorMap *> d_xmaps(B, nullptr), d_ymaps(B, nullptr);
    std::vector<int *> d_src(B, nullptr);
    for (int i = 0; i < B; ++i) {
        const int np = round_up(pl.inst[i].n, PAD);
        if (pl.dataflow) {
            P.flow_tiles = (int)tiles[i].size();
            P.flow_nb = flow_nblk(np);
            P.d_tile_done = (unsigned int *)c.take(sizeof(unsigned int) * tiles[i].size());
            d_src[i] = (int *)c.take(sizeof(int) * 2 * (size_t)P.flow_nb * P.flow_nb);
            P.d_blk_src = d_src[i];
        }
        if (pl.path == PATH_TC) {
            d_xmaps[i] = (CUtensorMap *)c.take((size_t)pl.slots[i] * MAPS_PER_SLOT * sizeof(CUtensorMap));
            if (pl.mode == MODE_RESPONSE || pl.mode == MODE_ADJOINT)
                d_ymaps[i] = (CUtensorMap *)c.take(2 * MAPS_PER_SLOT * sizeof(CUtensorMap));
        }
    }
    const size_t upload_bytes = c.off;
    std::vector<uint8_t> &blob = P.h_upload;
    blob.assign(upload_bytes, 0);
    auto put = [&](const void *dev, const void *host, size_t bytes) {
        if (bytes) memcpy(blob.data() + ((const uint8_t *)dev - (const uint8_t *)ws), host, bytes);
    };

    std::vector<InstDesc> h_inst(B);
    std::vector<InstCtl> &h_ctl = P.h_ctl;
    h_ctl.assign(B, InstCtl());
    std::vector<int2> h_tiles;
    std::vector<std::vector<CUtensorMap>> h_xmaps(B), h_ymaps(B);
    std::vector<int> forced;
    std::vector<double> forced_alpha;
    const int initb = init_blocks_host(pl.max_np);
    P.fin_blocks = finalize_blocks();
    if (P.fin_blocks < 1) return SP2_ERR_CUDA;
    bool user_bounds = o.user_bounds != 0;

    for (int i = 0; i < B; ++i) {
        InstSpec &sp = pl.inst[i];
        InstDesc &d = h_inst[i];
        memset(&d, 0, sizeof(d));
        const int n = sp.n, np = round_up(n, PAD);
        const size_t mat = (size_t)np * np;
        d.n = n;
        d.np = np;
        d.ntiles = (int)tiles[i].size();
        d.parts = d.ntiles * (pl.path == PATH_TC ? pl.cg : 1);
        // A device constant, so that an instance's tiles walk K the same way in a
        // batch as alone (the accumulation order, and so the bits, follow the tile).
        d.kwave = (pl.path == PATH_TC) ? std::max(1, P.grid / pl.cg) : 1;
        d.tile_off = (int)h_tiles.size();
        h_tiles.insert(h_tiles.end(), tiles[i].begin(), tiles[i].end());
        d.n_occ = sp.n_occ;
        d.nforced = -1;
        d.nslots_x = pl.slots[i];
        d.part_cap = std::max(d.parts, initb);
        d.fin_blocks = P.fin_blocks;
        d.ctl = d_ctl + i;
        d.part[0] = (Part *)c.take(sizeof(Part) * d.part_cap);
        d.part[1] = (Part *)c.take(sizeof(Part) * d.part_cap);
        d.part[2] = (Part *)c.take(sizeof(Part) * d.part_cap);
        if (pl.dataflow) {
            std::vector<int> src;
            build_block_sources(np, pl.cg, tiles[i], src);
            put(d_src[i], src.data(), sizeof(int) * src.size());
        }
        d.fin_part = (double2 *)c.take(sizeof(double2) * FIN_BLOCKS_MAX);
        d.xf[0] = (float *)c.take(mat * 4);
        d.xf[1] = (float *)c.take(mat * 4);
        if (pl.path == PATH_TC) {
            d.xop = (uint16_t *)c.take((size_t)d.nslots_x * 2 * mat * 2);
            d.xmap = d_xmaps[i];
            h_xmaps[i].resize((size_t)d.nslots_x * MAPS_PER_SLOT);
            // Per slot: the K segments' operands op0, op1, op2 = hi, hi, lo over the
            // slot's two matrices (hi, lo), then the epilogue's store maps of hi and lo.
            for (int sl = 0; sl < d.nslots_x; ++sl)
                if (!encode_slot_maps(&h_xmaps[i][(size_t)sl * MAPS_PER_SLOT], d.xop + (size_t)sl * 2 * mat, np,
                                      pl.precision))
                    return SP2_ERR_UNSUPPORTED;
            if (pl.ckpt_s[i] > 0) {
                d.ckpt_s = pl.ckpt_s[i];
                d.ckpt_k = pl.ckpt_k[i];
                d.ckf = (float *)c.take((size_t)d.ckpt_k * mat * 4);
                d.rf[0] = (float *)c.take(mat * 4);
                d.rf[1] = (float *)c.take(mat * 4);
            }
            if (pl.mode == MODE_RESPONSE || pl.mode == MODE_ADJOINT) {
                d.yf[0] = (float *)c.take(mat * 4);
                d.yf[1] = (float *)c.take(mat * 4);
                d.yop = (uint16_t *)c.take(2 * 2 * mat * 2);
                d.ymap = d_ymaps[i];
                h_ymaps[i].resize(2 * MAPS_PER_SLOT);
                for (int sl = 0; sl < 2; ++sl)
                    if (!encode_slot_maps(&h_ymaps[i][(size_t)sl * MAPS_PER_SLOT], d.yop + (size_t)sl * 2 * mat, np,
                                          pl.precision))
                        return SP2_ERR_UNSUPPORTED;
            }
        }
        InstCtl &ctl = h_ctl[i];
        memset(&ctl, 0, sizeof(ctl));
        ctl.emin_key = dkey(INFINITY);
        ctl.emax_key = dkey(-INFINITY);
        ctl.ymax_key = dkey(0.0);
        ctl.y_scale = 1.0;
        ctl.layers = 0;
        // Replayed layer sequence and bounds (response / adjoint following an
        // earlier forward run, or the layer-application entry point).
        if (sp.fwd) {
            user_bounds = true;
            ctl.eps_min = sp.fwd->eps_min;
            ctl.eps_max = sp.fwd->eps_max;
            forced.assign(sp.fwd->layers, 0);
            for (int k = 0; k < sp.fwd->layers; ++k) forced[k] = sp.fwd->layer[k + 1].choice;
            d.nforced = sp.fwd->layers;
            d.forced = d_forced;
            // An accelerated forward run is replayed with its own expansions.
            bool plain = true;
            forced_alpha.assign(sp.fwd->layers, 1.0);
            for (int k = 0; k < sp.fwd->layers; ++k) {
                forced_alpha[k] = sp.fwd->layer[k + 1].alpha;
                plain = plain && forced_alpha[k] == 1.0;
            }
            if (!plain) d.forced_alpha = d_forced_alpha;
            else forced_alpha.clear();
        } else if (sp.choices) {
            forced.assign(sp.choices, sp.choices + sp.nchoices);
            d.nforced = sp.nchoices;
            d.forced = d_forced;
        } else if (user_bounds) {
            ctl.eps_min = o.eps_min;
            ctl.eps_max = o.eps_max;
        }
        if (o.accelerate && !sp.fwd && !sp.choices) {
            d.accel = 1;
            d.gap_homo = o.eps_homo;
            d.gap_lumo = o.eps_lumo;
        }
        d.H = sp.H;
        d.H1 = sp.H1;
        d.out = sp.D;
        d.out1 = sp.D1;
    }

    // Host-resident inputs and outputs go through device memory: the tail of
    // the caller's workspace when it has room, else a stream-ordered allocation
    // freed before the call returns.  Page-locked host memory is used in place
    // across the host link: symmetric inputs (H, and H1 of a response) cross
    // it as their lower triangle only, and D / D1 are written to it directly
    // by the output kernel.  Pageable memory is copied whole.
    const size_t ws_end = ws_bytes;
    bool staging_err = false;
    auto staging = [&](size_t bytes) -> void * {
        const size_t start = (c.off + 255) & ~(size_t)255;
        if (ws_end && start + bytes <= ws_end) return c.take(bytes);
        return arena.get(bytes);
    };
    for (int i = 0; i < B; ++i) {
        InstSpec &sp = pl.inst[i];
        InstDesc &d = h_inst[i];
        const size_t nn = (size_t)sp.n * sp.n;
        const bool hH = sp.H && !is_device_ptr(sp.H), hH1 = sp.H1 && !is_device_ptr(sp.H1);
        const bool hX0 = sp.X0 && !is_device_ptr(sp.X0), hD = sp.D && !is_device_ptr(sp.D);
        const bool hD1 = sp.D1 && !is_device_ptr(sp.D1);
        if (!staging_ok && (hH || hH1 || hX0 || hD || hD1)) return SP2_ERR_ARG;
        auto stage_input = [&](const double *src, bool symmetric) -> double * {
            double *t = (double *)staging(nn * 8);
            if (!t) return nullptr;
            const void *m = symmetric ? mapped_host_ptr(src) : nullptr;
            const cudaError_t e = m ? launch_stage_lower((const double *)m, t, sp.n, s)
                                    : cudaMemcpyAsync(t, src, nn * 8, cudaMemcpyHostToDevice, s);
            if (e != cudaSuccess) {
                cudaGetLastError();
                staging_err = true;
            }
            return t;
        };
        if (hH) {
            d.H = stage_input(sp.H, true);
            if (!d.H) return SP2_ERR_NOMEM;
        }
        if (hH1) {  // the adjoint's weight G need not be symmetric
            d.H1 = stage_input(sp.H1, pl.mode == MODE_RESPONSE);
            if (!d.H1) return SP2_ERR_NOMEM;
        }
        if (staging_err) return SP2_ERR_CUDA;
        if (hX0) {
            float *t = (float *)staging(nn * 4);
            if (!t) return SP2_ERR_NOMEM;
            CK(cudaMemcpyAsync(t, sp.X0, nn * 4, cudaMemcpyHostToDevice, s));
            sp.X0 = t;
        }
        auto stage_output = [&](float *dst) -> float * {
            if (const void *m = mapped_host_ptr(dst)) return (float *)m;  // written across the link
            float *t = (float *)staging(nn * 4);
            if (!t) return nullptr;
            P.copy_back.push_back({dst, t});
            P.copy_back_n.push_back(nn);
            return t;
        };
        if (hD) {
            d.out = stage_output(sp.D);
            if (!d.out) return SP2_ERR_NOMEM;
        }
        if (hD1) {
            d.out1 = stage_output(sp.D1);
            if (!d.out1) return SP2_ERR_NOMEM;
        }
    }

    // Upload descriptors, tables, tensor maps and the initial control blocks (live and
    // kept) in one copy; the barrier word, error word and completion counters go up as zeros.
    put(d_inst, h_inst.data(), sizeof(InstDesc) * B);
    put(d_tiles, h_tiles.data(), sizeof(int2) * h_tiles.size());
    put(d_forced, forced.data(), sizeof(int) * forced.size());
    put(d_forced_alpha, forced_alpha.data(), sizeof(double) * forced_alpha.size());
    put(d_ctl, h_ctl.data(), sizeof(InstCtl) * B);
    put(d_ctl_init, h_ctl.data(), sizeof(InstCtl) * B);
    for (int i = 0; i < B; ++i) {
        if (d_xmaps[i]) put(d_xmaps[i], h_xmaps[i].data(), h_xmaps[i].size() * sizeof(CUtensorMap));
        if (d_ymaps[i]) put(d_ymaps[i], h_ymaps[i].data(), h_ymaps[i].size() * sizeof(CUtensorMap));
    }
    CK(cudaMemcpyAsync(ws, blob.data(), upload_bytes, cudaMemcpyHostToDevice, s));
    P.user_bounds = user_bounds;
    P.d_inst = d_inst;
    P.d_tiles = d_tiles;
    P.d_sync = d_sync;
    P.d_ctl = d_ctl;
    P.d_ctl_init = d_ctl_init;
    return SP2_OK;
}

// One solve on stream s: reset, input layer, the persistent layer kernel, the
// output.  ev (optional, 4 events) brackets the phases.  `fresh`: the upload of
// prepare() is the last write to the control state, so the reset is already done.
sp2_status enqueue(const Prepared &P, cudaStream_t s, cudaEvent_t *ev, bool fresh = false) {
    const Plan &pl = P.pl;
    const int B = (int)pl.inst.size();
    if (!fresh) {
        CK(cudaMemcpyAsync(P.d_ctl, P.d_ctl_init, sizeof(InstCtl) * B, cudaMemcpyDeviceToDevice, s));
        CK(cudaMemsetAsync(P.d_sync, 0, 64, s));
        if (pl.dataflow) CK(cudaMemsetAsync(P.d_tile_done, 0, sizeof(unsigned int) * P.flow_tiles, s));
    }
    if (ev) CK(cudaEventRecord(ev[0], s));
    if (pl.mode == MODE_APPLY) {
        CK(launch_init_x_from(P.d_inst, pl.inst[0].X0, pl.max_np, pl.path, pl.precision, s));
    } else {
        CK(launch_gershgorin(P.d_inst, B, pl.max_n, P.user_bounds, s));
        CK(launch_init_x(P.d_inst, B, pl.max_np, pl.path, pl.precision, P.user_bounds, s));
    }
    if (pl.mode == MODE_RESPONSE || pl.mode == MODE_ADJOINT) {
        CK(launch_maxabs(P.d_inst, B, pl.max_n, s));
        CK(launch_init_y(P.d_inst, pl.mode, pl.precision, s));
    }
    RunParams rp;
    memset(&rp, 0, sizeof(rp));
    rp.inst = P.d_inst;
    rp.tiles = P.d_tiles;
    rp.barrier = (unsigned int *)P.d_sync;
    rp.err = (int *)(P.d_sync + 4);
    rp.tol = P.tol;
    rp.timeout_ns = (unsigned long long)(P.o.timeout_ms * 1e6);
    rp.B = B;
    rp.mode = pl.mode;
    rp.precision = pl.precision;
    rp.max_layers = P.o.max_layers;
    // Device hook: CTA 0 withholds its first barrier arrival (test_hook 1, or 3 in a CTA-pair launch).
    rp.test_hook = (P.o.test_hook == 1 || (P.o.test_hook == 3 && pl.path == PATH_TC && pl.cg == 2)) ? 1 : 0;
    rp.publish = (pl.mode == MODE_DENSITY && pl.path == PATH_TC && !pl.dataflow) ? 1 : 0;
    if (pl.dataflow) {
        rp.dataflow = 1;
        rp.nblk = P.flow_nb;
        rp.tile_done = P.d_tile_done;
        rp.layer_done = (unsigned int *)(P.d_sync + 8);
        rp.blk_src = P.d_blk_src;
    }
    if (ev) CK(cudaEventRecord(ev[1], s));
    CK(pl.path == PATH_TC ? launch_tc_persistent(rp, pl.cg, P.grid, s) : launch_simt_persistent(rp, P.grid, s));
    if (ev) CK(cudaEventRecord(ev[2], s));
    CK(launch_finalize(P.d_inst, B, P.fin_blocks, pl.mode == MODE_APPLY ? MODE_DENSITY : pl.mode, s));
    if (ev) CK(cudaEventRecord(ev[3], s));
    return SP2_OK;
}

// Read the control blocks back (synchronises s) and fill the callers' stats.
sp2_status collect(Prepared &P, cudaStream_t s, const float *ph) {
    const Plan &pl = P.pl;
    const int B = (int)pl.inst.size();
    for (size_t k = 0; k < P.copy_back.size(); ++k)
        CK(cudaMemcpyAsync(P.copy_back[k].first, P.copy_back[k].second, P.copy_back_n[k] * 4,
                           cudaMemcpyDeviceToHost, s));
    // The error word and the control blocks in one copy (they are adjacent).
    const size_t ctl_off = (size_t)((const uint8_t *)P.d_ctl - P.d_sync);
    P.h_back.resize(ctl_off + sizeof(InstCtl) * B);
    CK(cudaMemcpyAsync(P.h_back.data(), P.d_sync, P.h_back.size(), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    int h_err = 0;
    memcpy(&h_err, P.h_back.data() + 4, sizeof(int));
    memcpy(P.h_ctl.data(), P.h_back.data() + ctl_off, sizeof(InstCtl) * B);
    if (h_err) return (sp2_status)h_err;
    int worst = SP2_OK;
    for (int i = 0; i < B; ++i) {
        fill_stats(pl.inst[i].st, P.h_ctl[i]);
        if (pl.inst[i].st) {
            for (int k = 0; k < 4; ++k) pl.inst[i].st->phase_ms[k] = ph ? ph[k] : 0.0f;
            pl.inst[i].st->cta_group = (pl.path == PATH_TC) ? pl.cg : 0;
        }
        int stt = P.h_ctl[i].status;
        if (P.h_ctl[i].nonfinite) stt = SP2_ERR_NONFINITE;
        if (status_rank(stt) > status_rank(worst)) worst = stt;
    }
    return (sp2_status)worst;
}

sp2_status run_plan_once(Plan &pl, double tol, const sp2_opts &o, void *ws, size_t ws_bytes, cudaStream_t s,
                         int *used_cg) {
    const int B = (int)pl.inst.size();
    if (B == 0) return SP2_OK;
    Prepared P;
    P.pl = pl;
    sp2_status r = choose_launch(P.pl, o.cta_group, P.grid);
    if (r != SP2_OK) return r;
    *used_cg = (P.pl.path == PATH_TC) ? P.pl.cg : 0;
    Arena arena(s);
    arena.fail = (o.test_hook == 2);
    const size_t need = plan_bytes(P.pl);
    if (ws && ws_bytes < need) return SP2_ERR_ARG;
    if (ws && ((uintptr_t)ws & 255)) return SP2_ERR_ARG;
    if (!ws) {
        ws = arena.get(need);
        if (!ws) return SP2_ERR_NOMEM;
    }
    r = prepare(P, o, tol, ws, ws_bytes, s, arena, true);
    if (r != SP2_OK) return r;
    // Optional per-phase device timing on the call's stream.
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    struct EvGuard {
        cudaEvent_t *e;
        ~EvGuard() {
            for (int k = 0; k < 4; ++k)
                if (e[k]) cudaEventDestroy(e[k]);
        }
    } ev_guard{ev};
    if (o.profile)
        for (int k = 0; k < 4; ++k) CK(cudaEventCreate(&ev[k]));
    r = enqueue(P, s, o.profile ? ev : nullptr, true);
    if (r != SP2_OK) return r;
    float ph[4] = {0.f, 0.f, 0.f, 0.f};
    r = collect(P, s, nullptr);
    if (o.profile) {
        CK(cudaEventElapsedTime(&ph[0], ev[0], ev[1]));
        CK(cudaEventElapsedTime(&ph[1], ev[1], ev[2]));
        CK(cudaEventElapsedTime(&ph[2], ev[2], ev[3]));
        CK(cudaEventElapsedTime(&ph[3], ev[0], ev[3]));
        for (int i = 0; i < B; ++i)
            if (P.pl.inst[i].st)
                for (int k = 0; k < 4; ++k) P.pl.inst[i].st->phase_ms[k] = ph[k];
    }
    return r;
}

// A CTA-pair launch relies on every pair being resident at once (it is a cluster
// launch, not a cooperative one); work running concurrently on the same GPU can
// deny that, and the waits between layers (the grid barrier, or the dataflow
// schedule's waits for the previous layer's tiles) then run out of time.  When the tile shape was
// left to the library, the call is retried once with single-CTA tiles, whose
// cooperative launch guarantees co-residency.
sp2_status run_plan(Plan &pl, double tol, const sp2_opts &o, void *ws, size_t ws_bytes, cudaStream_t s) {
    int used_cg = 0;
    sp2_status r = run_plan_once(pl, tol, o, ws, ws_bytes, s, &used_cg);
    if (r == SP2_ERR_TIMEOUT && used_cg == 2 && o.cta_group == 0 && o.test_hook != 1) {
        sp2_opts o1 = o;
        o1.cta_group = 1;
        r = run_plan_once(pl, tol, o1, ws, ws_bytes, s, &used_cg);
    }
    return r;
}

bool integral_occ(double n_occ, int n) {
    return std::isfinite(n_occ) && n_occ >= 0.0 && n_occ <= (double)n && std::floor(n_occ) == n_occ;
}

sp2_status check_opts(const sp2_opts &o) {
    if (o.precision < SP2_FP32_SIMT || o.precision > SP2_BF16_SPLIT) return SP2_ERR_ARG;
    if (o.max_layers < 1 || o.max_layers > SP2_MAX_LAYERS_LIMIT) return SP2_ERR_ARG;
    if (!(o.timeout_ms > 0.0)) return SP2_ERR_ARG;
    if (o.user_bounds && !(o.eps_max > o.eps_min)) return SP2_ERR_ARG;
    if (o.test_hook < 0 || o.test_hook > 3) return SP2_ERR_ARG;
    if (o.profile < 0 || o.profile > 1) return SP2_ERR_ARG;
    if (o.cta_group < 0 || o.cta_group > 2) return SP2_ERR_ARG;
    if (o.accelerate < 0 || o.accelerate > 1) return SP2_ERR_ARG;
    if (o.accelerate && !(std::isfinite(o.eps_homo) && std::isfinite(o.eps_lumo) && o.eps_homo < o.eps_lumo))
        return SP2_ERR_ARG;
    if (o.checkpoint_stride < -1 || o.checkpoint_stride > SP2_MAX_LAYERS_LIMIT) return SP2_ERR_ARG;
    return SP2_OK;
}

// Trivial occupations: D = 0 or I, response and gradient 0.
sp2_status run_trivial(const InstSpec &sp, cudaStream_t s) {
    const size_t nn = (size_t)sp.n * sp.n;
    const float diag = (sp.n_occ == 0.0) ? 0.0f : 1.0f;
    auto fill = [&](float *p, float dv) -> sp2_status {
        if (!p) return SP2_OK;
        if (is_device_ptr(p)) {
            if (launch_fill_trivial(p, sp.n, dv, s) != cudaSuccess) return SP2_ERR_CUDA;
        } else {
            if (cudaStreamSynchronize(s) != cudaSuccess) return SP2_ERR_CUDA;
            for (size_t k = 0; k < nn; ++k) p[k] = ((k / sp.n) == (k % sp.n)) ? dv : 0.0f;
        }
        return SP2_OK;
    };
    sp2_status r = fill(sp.D, diag);
    if (r != SP2_OK) return r;
    r = fill(sp.D1, 0.0f);
    if (r != SP2_OK) return r;
    if (cudaStreamSynchronize(s) != cudaSuccess) return SP2_ERR_CUDA;
    fill_trivial_stats(sp.st, sp.n, sp.n_occ);
    if (sp.st && sp.H && sp.n_occ > 0.0) {
        // Tr[I H] = sum of the diagonal, in FP64.
        std::vector<double> diagv(sp.n);
        double e = 0.0;
        if (is_device_ptr(sp.H)) {
            for (int i = 0; i < sp.n; ++i) {
                if (cudaMemcpy(&diagv[i], sp.H + (size_t)i * sp.n + i, 8, cudaMemcpyDeviceToHost) != cudaSuccess)
                    return SP2_ERR_CUDA;
            }
        } else {
            for (int i = 0; i < sp.n; ++i) diagv[i] = sp.H[(size_t)i * sp.n + i];
        }
        for (int i = 0; i < sp.n; ++i) e += diagv[i];
        sp.st->band_energy = e;
    }
    return SP2_OK;
}

sp2_status run_instances(int mode, std::vector<InstSpec> &specs, double tol, const sp2_opts *opts, void *ws,
                         size_t ws_bytes, void *stream) {
    const sp2_opts o = resolve_opts(opts);
    sp2_status r = check_opts(o);
    if (r != SP2_OK) return r;
    if (!(tol >= 0.0)) return SP2_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    Plan pl;
    pl.mode = mode;
    pl.precision = o.precision;
    pl.path = (o.precision == SP2_FP32_SIMT) ? PATH_SIMT : PATH_TC;
    if ((mode == MODE_RESPONSE || mode == MODE_ADJOINT) && pl.path == PATH_SIMT) return SP2_ERR_UNSUPPORTED;
    if ((int)specs.size() > MAX_BATCH) return SP2_ERR_ARG;
    int worst = SP2_OK;
    std::vector<int> order;
    for (size_t k = 0; k < specs.size(); ++k) {
        InstSpec &sp = specs[k];
        if (sp.n < 1 || sp.n > 65536) return SP2_ERR_ARG;
        if (!integral_occ(sp.n_occ, sp.n)) return SP2_ERR_ARG;
        if (mode != MODE_APPLY && !sp.H) return SP2_ERR_ARG;
        if ((mode == MODE_DENSITY || mode == MODE_APPLY) && !sp.D) return SP2_ERR_ARG;
        if ((mode == MODE_RESPONSE || mode == MODE_ADJOINT) && (!sp.H1 || !sp.D1)) return SP2_ERR_ARG;
        if (sp.fwd && (!sp.fwd->layer || sp.fwd->layer_cap < sp.fwd->layers + 1 || sp.fwd->layers < 0 ||
                       sp.fwd->layers > SP2_MAX_LAYERS_LIMIT))
            return SP2_ERR_ARG;
        const bool trivial = (mode != MODE_APPLY) && (sp.n_occ == 0.0 || sp.n_occ == (double)sp.n);
        if (trivial) {
            sp2_status t = run_trivial(sp, s);
            if (t != SP2_OK) return t;
            continue;
        }
        order.push_back((int)k);
    }
    // Largest instances first: the static round-robin tile schedule then mixes
    // long and short tiles across CTAs.
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return specs[a].n > specs[b].n; });
    for (int k : order) {
        const InstSpec &sp = specs[k];
        pl.inst.push_back(sp);
        int slots = 2, cs = 0, ck = 0;
        if (mode == MODE_ADJOINT)
            adjoint_layout(sp.fwd ? sp.fwd->layers : o.max_layers, o.checkpoint_stride, slots, cs, ck);
        pl.slots.push_back(slots);
        pl.ckpt_s.push_back(cs);
        pl.ckpt_k.push_back(ck);
        pl.max_n = std::max(pl.max_n, sp.n);
        pl.max_np = std::max(pl.max_np, round_up(sp.n, PAD));
    }
    set_flow(pl);
    r = run_plan(pl, tol, o, ws, ws_bytes, s);
    if (status_rank(r) > status_rank(worst)) worst = r;
    return (sp2_status)worst;
}

size_t bytes_for(int mode, const std::vector<int> &ns, int layers, const sp2_opts *opts) {
    const sp2_opts o = resolve_opts(opts);
    Plan pl;
    pl.mode = mode;
    pl.precision = o.precision;
    pl.path = (o.precision == SP2_FP32_SIMT) ? PATH_SIMT : PATH_TC;
    for (int n : ns) {
        if (n < 1) continue;
        InstSpec sp;
        sp.n = n;
        pl.inst.push_back(sp);
        int slots = 2, cs = 0, ck = 0;
        if (mode == MODE_ADJOINT) adjoint_layout(layers > 0 ? layers : o.max_layers, o.checkpoint_stride, slots, cs, ck);
        pl.slots.push_back(slots);
        pl.ckpt_s.push_back(cs);
        pl.ckpt_k.push_back(ck);
        pl.max_n = std::max(pl.max_n, n);
        pl.max_np = std::max(pl.max_np, round_up(n, PAD));
    }
    if (pl.inst.empty()) return 0;
    set_flow(pl);
    pl.cg = 1;
    const size_t b1 = plan_bytes(pl);
    pl.cg = 2;
    const size_t b2 = plan_bytes(pl);
    return b1 > b2 ? b1 : b2;  // the tile shape is chosen per device at run time
}

// Tile shape chosen by timing, per (precision, sorted sizes); process-wide.
std::mutex g_tune_mu;
std::vector<std::pair<std::string, int>> g_tune;

std::string tune_key(const Plan &pl) {
    std::vector<int> ns;
    for (auto &sp : pl.inst) ns.push_back(sp.n);
    std::sort(ns.begin(), ns.end());
    std::string k = std::to_string(pl.precision) + ":" + std::to_string(pl.mode);
    for (int n : ns) k += "," + std::to_string(n);
    return k;
}

}  // namespace

struct sp2_batch_plan {
    Prepared P;                        // non-trivial instances, in launch order
    std::vector<int> order;            // P.pl.inst[i] is the caller's instance order[i]
    std::vector<InstSpec> trivial;     // n_occ = 0 or N: D = 0 or I
    std::vector<int> trivial_index;
    int B = 0;
    void *ws = nullptr;                // plan-owned workspace
    ~sp2_batch_plan() {
        if (ws) cudaFree(ws);
    }
};

extern "C" {

void sp2_default_opts(sp2_opts *o) {
    if (!o) return;
    memset(o, 0, sizeof(*o));
    o->precision = SP2_FP16_SPLIT;
    o->max_layers = 100;
    o->timeout_ms = 2000.0;
    o->user_bounds = 0;
}

const char *sp2_status_string(sp2_status s) {
    switch (s) {
        case SP2_OK: return "ok";
        case SP2_ERR_ARG: return "invalid argument";
        case SP2_ERR_NONFINITE: return "non-finite input";
        case SP2_ERR_NOT_CONVERGED: return "not converged within max_layers";
        case SP2_ERR_TIMEOUT: return "device wait timed out";
        case SP2_ERR_CUDA: return "CUDA error";
        case SP2_ERR_NOMEM: return "out of memory";
        case SP2_ERR_UNSUPPORTED: return "unsupported device or configuration";
    }
    return "unknown status";
}

sp2_status sp2_device_info(int *sm_count, int *cc_major, int *cc_minor) {
    DeviceInfo di = query_device();
    if (di.err != cudaSuccess) return SP2_ERR_CUDA;
    if (sm_count) *sm_count = di.sm;
    if (cc_major) *cc_major = di.major;
    if (cc_minor) *cc_minor = di.minor;
    return (di.major == 10 && di.minor == 3) ? SP2_OK : SP2_ERR_UNSUPPORTED;
}

size_t sp2_density_workspace_bytes(int N, const sp2_opts *o) { return bytes_for(MODE_DENSITY, {N}, 0, o); }

size_t sp2_response_workspace_bytes(int N, const sp2_opts *o) { return bytes_for(MODE_RESPONSE, {N}, 0, o); }

size_t sp2_adjoint_workspace_bytes(int N, int layers, const sp2_opts *o) {
    return bytes_for(MODE_ADJOINT, {N}, layers, o);
}

sp2_status sp2_batch_plan_create(int B, const double *const *H, const int *N, const double *n_occ, double tol,
                                 float *const *D, const sp2_opts *opts, int autotune, void *stream,
                                 sp2_batch_plan **plan) {
    if (!plan) return SP2_ERR_ARG;
    *plan = nullptr;
    if (B < 1 || B > MAX_BATCH || !H || !N || !n_occ || !D || !(tol >= 0.0)) return SP2_ERR_ARG;
    if (autotune < 0 || autotune > 1) return SP2_ERR_ARG;
    const sp2_opts o = resolve_opts(opts);
    sp2_status r = check_opts(o);
    if (r != SP2_OK) return r;
    if (o.accelerate || o.profile || o.test_hook) return SP2_ERR_ARG;
    for (int b = 0; b < B; ++b) {
        if (N[b] < 1 || N[b] > 65536 || !integral_occ(n_occ[b], N[b]) || !H[b] || !D[b]) return SP2_ERR_ARG;
    }
    for (int b = 0; b < B; ++b)
        if (!is_device_ptr(H[b]) || !is_device_ptr(D[b])) return SP2_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    std::unique_ptr<sp2_batch_plan> pb(new sp2_batch_plan());
    pb->B = B;
    Plan pl;
    pl.mode = MODE_DENSITY;
    pl.precision = o.precision;
    pl.path = (o.precision == SP2_FP32_SIMT) ? PATH_SIMT : PATH_TC;
    std::vector<int> order;
    for (int b = 0; b < B; ++b) {
        InstSpec sp;
        sp.n = N[b];
        sp.n_occ = n_occ[b];
        sp.H = H[b];
        sp.D = D[b];
        if (sp.n_occ == 0.0 || sp.n_occ == (double)sp.n) {
            pb->trivial.push_back(sp);
            pb->trivial_index.push_back(b);
        } else {
            order.push_back(b);
        }
    }
    std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return N[a] > N[c]; });
    for (int b : order) {
        InstSpec sp;
        sp.n = N[b];
        sp.n_occ = n_occ[b];
        sp.H = H[b];
        sp.D = D[b];
        pl.inst.push_back(sp);
        pl.slots.push_back(2);
        pl.ckpt_s.push_back(0);
        pl.ckpt_k.push_back(0);
        pl.max_n = std::max(pl.max_n, sp.n);
        pl.max_np = std::max(pl.max_np, round_up(sp.n, PAD));
    }
    set_flow(pl);
    pb->order = order;
    if (!pl.inst.empty()) {
        // Workspace for either tile shape, owned by the plan.
        const size_t need = bytes_for(MODE_DENSITY, [&] {
            std::vector<int> ns;
            for (auto &sp : pl.inst) ns.push_back(sp.n);
            return ns;
        }(), 0, &o);
        if (cudaMalloc(&pb->ws, need) != cudaSuccess) {
            cudaGetLastError();
            return SP2_ERR_NOMEM;
        }
        Arena arena(s);  // unused: every matrix is device-resident
        int want = o.cta_group;
        if (pl.path == PATH_TC && want == 0) {
            const std::string key = tune_key(pl);
            {
                std::lock_guard<std::mutex> g(g_tune_mu);
                for (auto &kv : g_tune)
                    if (kv.first == key) want = kv.second;
            }
            if (want == 0 && autotune) {
                // Time one solve per tile shape on these inputs (after one warm-up).
                float best = 0.0f;
                int best_cg = 0;
                cudaEvent_t e0 = nullptr, e1 = nullptr;
                if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
                    if (e0) cudaEventDestroy(e0);
                    cudaGetLastError();
                    return SP2_ERR_CUDA;
                }
                for (int cg = 2; cg >= 1; --cg) {
                    Prepared T;
                    T.pl = pl;
                    if (choose_launch(T.pl, cg, T.grid) != SP2_OK) continue;
                    if (prepare(T, o, tol, pb->ws, need, s, arena, false) != SP2_OK) continue;
                    if (enqueue(T, s, nullptr) != SP2_OK) continue;
                    cudaEventRecord(e0, s);
                    if (enqueue(T, s, nullptr) != SP2_OK) continue;
                    cudaEventRecord(e1, s);
                    if (status_rank(collect(T, s, nullptr)) > 1) continue;  // an error, not a slow chain
                    float ms = 0.0f;
                    cudaEventElapsedTime(&ms, e0, e1);
                    if (best_cg == 0 || ms < best) {
                        best = ms;
                        best_cg = cg;
                    }
                }
                cudaEventDestroy(e0);
                cudaEventDestroy(e1);
                cudaGetLastError();
                if (best_cg == 0) return SP2_ERR_UNSUPPORTED;
                want = best_cg;
                std::lock_guard<std::mutex> g(g_tune_mu);
                g_tune.push_back({key, best_cg});
            }
        }
        pb->P.pl = pl;
        r = choose_launch(pb->P.pl, want, pb->P.grid);
        if (r != SP2_OK) return r;
        r = prepare(pb->P, o, tol, pb->ws, need, s, arena, false);
        if (r != SP2_OK) return r;
        if (cudaStreamSynchronize(s) != cudaSuccess) {
            cudaGetLastError();
            return SP2_ERR_CUDA;
        }
    } else {
        pb->P.pl = pl;
        pb->P.o = o;
    }
    *plan = pb.release();
    return SP2_OK;
}

sp2_status sp2_batch_plan_launch(sp2_batch_plan *plan, void *stream) {
    if (!plan) return SP2_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    for (auto &sp : plan->trivial)
        if (launch_fill_trivial(sp.D, sp.n, sp.n_occ == 0.0 ? 0.0f : 1.0f, s) != cudaSuccess) {
            cudaGetLastError();
            return SP2_ERR_CUDA;
        }
    if (plan->P.pl.inst.empty()) return SP2_OK;
    return enqueue(plan->P, s, nullptr);
}

sp2_status sp2_batch_plan_stats(sp2_batch_plan *plan, sp2_stats *st, void *stream) {
    if (!plan) return SP2_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    sp2_status worst = SP2_OK;
    if (!plan->P.pl.inst.empty()) {
        for (size_t i = 0; i < plan->P.pl.inst.size(); ++i)
            plan->P.pl.inst[i].st = st ? &st[plan->order[i]] : nullptr;
        worst = collect(plan->P, s, nullptr);
    } else if (cudaStreamSynchronize(s) != cudaSuccess) {
        cudaGetLastError();
        return SP2_ERR_CUDA;
    }
    for (size_t k = 0; k < plan->trivial.size(); ++k) {
        InstSpec sp = plan->trivial[k];
        sp.D = nullptr;  // already written by the launch
        sp.st = st ? &st[plan->trivial_index[k]] : nullptr;
        sp2_status t = run_trivial(sp, s);
        if (status_rank(t) > status_rank(worst)) worst = t;
    }
    return worst;
}

int sp2_batch_plan_cta_group(const sp2_batch_plan *plan) {
    if (!plan || plan->P.pl.path != PATH_TC || plan->P.pl.inst.empty()) return 0;
    return plan->P.pl.cg;
}

void sp2_batch_plan_destroy(sp2_batch_plan *plan) { delete plan; }

size_t sp2_density_batched_workspace_bytes(int B, const int *N, const sp2_opts *o) {
    if (B < 1 || !N) return 0;
    return bytes_for(MODE_DENSITY, std::vector<int>(N, N + B), 0, o);
}

sp2_status sp2_density(const double *H, int N, double n_occ, double tol, float *D, sp2_stats *st, const sp2_opts *o,
                       void *workspace, size_t ws_bytes, void *stream) {
    std::vector<InstSpec> v(1);
    v[0].n = N;
    v[0].n_occ = n_occ;
    v[0].H = H;
    v[0].D = D;
    v[0].st = st;
    return run_instances(MODE_DENSITY, v, tol, o, workspace, ws_bytes, stream);
}

sp2_status sp2_response(const double *H, const double *H1, int N, double n_occ, double tol, const sp2_stats *fwd,
                        float *D, float *D1, sp2_stats *st, const sp2_opts *o, void *workspace, size_t ws_bytes,
                        void *stream) {
    std::vector<InstSpec> v(1);
    v[0].n = N;
    v[0].n_occ = n_occ;
    v[0].H = H;
    v[0].H1 = H1;
    v[0].D = D;
    v[0].D1 = D1;
    v[0].st = st;
    v[0].fwd = fwd;
    return run_instances(MODE_RESPONSE, v, tol, o, workspace, ws_bytes, stream);
}

sp2_status sp2_adjoint(const double *H, const double *G, int N, double n_occ, double tol, const sp2_stats *fwd,
                       float *D, float *dH, sp2_stats *st, const sp2_opts *o, void *workspace, size_t ws_bytes,
                       void *stream) {
    std::vector<InstSpec> v(1);
    v[0].n = N;
    v[0].n_occ = n_occ;
    v[0].H = H;
    v[0].H1 = G;
    v[0].D = D;
    v[0].D1 = dH;
    v[0].st = st;
    v[0].fwd = fwd;
    return run_instances(MODE_ADJOINT, v, tol, o, workspace, ws_bytes, stream);
}

sp2_status sp2_density_batched(int B, const double *const *H, const int *N, const double *n_occ, double tol,
                               float *const *D, sp2_stats *st, const sp2_opts *o, void *workspace, size_t ws_bytes,
                               void *stream) {
    if (B < 1 || !H || !N || !n_occ || !D) return SP2_ERR_ARG;
    if (o && o->accelerate) return SP2_ERR_ARG;  // one interval cannot serve every instance
    std::vector<InstSpec> v(B);
    for (int b = 0; b < B; ++b) {
        v[b].n = N[b];
        v[b].n_occ = n_occ[b];
        v[b].H = H[b];
        v[b].D = D[b];
        v[b].st = st ? &st[b] : nullptr;
    }
    return run_instances(MODE_DENSITY, v, tol, o, workspace, ws_bytes, stream);
}

sp2_status sp2_apply_layers(const float *X0, int N, const int *choices, int n_layers, float *X, sp2_stats *st,
                            const sp2_opts *o, void *stream) {
    if (!X0 || !X || n_layers < 0 || n_layers > SP2_MAX_LAYERS_LIMIT || (n_layers > 0 && !choices))
        return SP2_ERR_ARG;
    for (int k = 0; k < n_layers; ++k)
        if (choices[k] != SP2_CHOICE_SQUARE && choices[k] != SP2_CHOICE_FLIP) return SP2_ERR_ARG;
    if (o && o->accelerate) return SP2_ERR_ARG;  // the layers applied here are the plain ones
    std::vector<InstSpec> v(1);
    v[0].n = N;
    v[0].n_occ = 0.0;
    v[0].X0 = X0;
    v[0].D = X;
    v[0].st = st;
    v[0].choices = choices;
    v[0].nchoices = n_layers;
    return run_instances(MODE_APPLY, v, 1e300, o, nullptr, 0, stream);
}

}  // extern "C"
