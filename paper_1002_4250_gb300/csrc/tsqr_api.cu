// The C ABI of libtsqr (include/tsqr.h): argument checks, plan selection, workspace and
// launches.  Every step of the computation runs in the kernels; this file only plans and
// enqueues.
#include <algorithm>
#include <cstring>
#include <map>
#include <mutex>
#include <numeric>
#include <utility>
#include <vector>
#include <cmath>

#include "tsqr.h"
#include "tsqr_internal.h"
#include "tsqr_qr.cuh"

namespace tsqr {
// Q^T B and the triangular solve of tsqr_lstsq (tsqr_qr.cu)
size_t qt_smem_bytes(int n, int k, int ldS, int warps);
cudaError_t qt_prepare(size_t smem_bytes);
cudaError_t qt_launch(const QtArgs &a, int blk, int warps, size_t smem_bytes, cudaStream_t stream);
size_t wy_smem_bytes(int n, int ldX);
cudaError_t wy_launch(const WyArgs &a, size_t smem_bytes, int grid, cudaStream_t stream);
size_t qt_wy_smem_bytes(int n, int kc, int ldS, bool fused = false);
size_t q_leaf_wy_smem_bytes(int n, int qn, int ldS, bool fused);
cudaError_t q_leaf_wy_launch(const QLeafArgs &a, size_t smem_bytes, cudaStream_t stream);
cudaError_t qt_wy_launch(const QtArgs &a, size_t smem_bytes, cudaStream_t stream);
cudaError_t trsm_launch(const double *R, int64_t ldr, const double *C, int64_t ldc, double *X,
                        int64_t ldx, int n, int k, int *status, cudaStream_t stream);
}  // namespace tsqr

using namespace tsqr;

namespace {

thread_local int g_last_launches = 0;
thread_local tsqr_plan_t g_last_plan{};  // the plan of the last call's (first) factorization
thread_local tsqr_batch_plan_t g_last_batch_plan{};  // the knobs of the last batched call

struct Workspace {
    void *base = nullptr;   // counters + slots (grown on demand)
    size_t bytes = 0;
    int *status = nullptr;  // device status word (lives as long as the workspace entry)
    // batched calls: the problem table and work items last copied to base + table_off
    std::vector<char> table;
    size_t table_off = 0;
};

std::mutex g_mu;
std::map<std::pair<int, cudaStream_t>, Workspace> g_ws;

struct DeviceInfo {
    int sms = 0;
    size_t smem_block_optin = 0;
    size_t smem_sm = 0;
};

DeviceInfo device_info(int dev) {
    static std::mutex mu;
    static std::map<int, DeviceInfo> cache;
    std::lock_guard<std::mutex> lk(mu);
    auto it = cache.find(dev);
    if (it != cache.end()) return it->second;
    DeviceInfo d;
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess) d.sms = v;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) == cudaSuccess)
        d.smem_block_optin = (size_t)v;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) == cudaSuccess)
        d.smem_sm = (size_t)v;
    cache[dev] = d;
    return d;
}

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }
inline int64_t round_up(int64_t x, int64_t a) { return (x + a - 1) / a * a; }

struct F64Plan {
    int tree = TSQR_TREE_HYBRID;
    int leaf = 0;                  // mixed path: TSQR_LEAF_FOLD or TSQR_LEAF_PANELS
    int warps = 4;
    int64_t unit = 0, nunits = 0;  // rows per work unit (tile or slab) and their count
    int h = 0, hs = 0, ldS = 0;    // chunk rows, shared-memory rows, leading dimension
    int blk = 1, vec = 1;          // inner-loop block and vector width of the leaf fold
    int arity = 2;                 // children per tree node
    int ldSd = 0, s_doubles = 0;   // FP64 view of the S region for the tree operator
    int nleaves = 0;
    size_t smem = 0;
    TreeShape shape{};
    int64_t nodes = 0;
};

// Arguments of the Q^T apply for a factorization with storage `q` under plan p: B (m x ktot,
// leading dimension ldb) in groups of k columns; the apply's counters, slots, outputs and S
// factors are the caller's to set.  Every other field is zero.
QtArgs qt_args(const F64Plan &p, const QStore &q, int64_t m, int n, const double *B,
               int64_t ldb, int k, int ktot) {
    QtArgs t;
    std::memset(&t, 0, sizeof(t));
    t.V = q.V;
    t.ldv = q.ldv;
    t.B = B;
    t.m = m;
    t.ldb = ldb;
    t.n = n;
    t.k = k;
    t.ktot = ktot;
    t.unit = p.unit;
    t.nunits = p.nunits;
    t.nleaves = p.nleaves;
    t.h = p.h;
    t.hs = p.hs;
    t.ldS = p.ldS;
    t.arity = p.arity;
    t.chunk_sc = q.chunk_sc;
    t.node_V = q.node_V;
    t.node_sc = q.node_sc;
    t.signs = q.signs;
    t.nodes = p.nodes;
    return t;
}

// Arguments of the compact WY factor kernel for the chunks of a factorization with storage q.
WyArgs wy_args(const F64Plan &p, const QStore &q, int64_t m, int n, int ldX, double *S) {
    WyArgs w;
    w.V = q.V;
    w.ldv = q.ldv;
    w.m = m;
    w.n = n;
    w.h = p.h;
    w.ldX = ldX;
    w.nchunks = (m + p.h - 1) / p.h;
    w.chunk_sc = q.chunk_sc;
    w.S = S;
    return w;
}

// The public form of a plan: passed back as a plan it gives the same partition and kernels.
tsqr_plan_t public_plan(const F64Plan &p) {
    tsqr_plan_t o;
    o.tree = p.tree;
    o.tile_rows = (int32_t)p.unit;
    o.ctas = p.nleaves;
    o.warps = p.warps;
    o.arity = p.arity;
    o.leaf = p.leaf;
    return o;
}

// Kernel arguments for a plan: A (leading dimension lda), m, n and the plan's shape; the
// workspace, R and status pointers are the caller's to set.  Every other field is zero.
F64Args plan_args(const F64Plan &p, const double *A, int64_t m, int64_t n, int64_t lda) {
    F64Args a;
    std::memset(&a, 0, sizeof(a));
    a.A = A;
    a.m = m;
    a.lda = lda;
    a.n = (int)n;
    a.unit = p.unit;
    a.nunits = p.nunits;
    a.nleaves = p.nleaves;
    a.arity = p.arity;
    a.h = p.h;
    a.hs = p.hs;
    a.blk = p.blk;
    a.vec = p.vec;
    a.ldS = p.ldS;
    return a;
}

tsqr_status_t build_tree(int64_t leaves, int arity, TreeShape *t, int64_t *nodes) {
    std::memset(t, 0, sizeof(*t));
    int64_t c = leaves, off = 0;
    int l = 0;
    for (;;) {
        if (l >= kMaxLevels) return TSQR_ERR_UNSUPPORTED;
        t->count[l] = (int)c;
        t->offset[l] = (int)off;
        off += c;
        ++l;
        if (c == 1) break;
        c = (c + arity - 1) / arity;
    }
    t->levels = l;
    *nodes = off;
    return TSQR_SUCCESS;
}

// Leading dimension of the chunk in shared memory for accesses of `vec` elements: a multiple of
// vec whose quotient by vec is odd, so that the lanes' accesses into different columns at the
// same row fall into different banks.
int ld_for(int hs, int vec = 1) {
    const int q = (hs + vec - 1) / vec;
    return vec * ((q % 2 == 0) ? q + 1 : q);
}


// Rows per lane whose inner loop blocks well: a multiple of 4 or 3 when r >= 3.
int good_r(int r) {
    if (r < 3) return r;
    while (r % 4 && r % 3) --r;
    return r;
}

// Inner-loop block (rows, a divisor of the rows per lane r) and vector width (elements per
// shared-memory access) of the leaf fold; the pairs are those the kernels are instantiated for.
void block_for(int r, bool fp32, int *blk, int *vec) {
    if (fp32) {
        if (r % 8 == 0) { *blk = 8; *vec = 4; }
        else if (r % 4 == 0) { *blk = 4; *vec = 4; }
        else if (r % 6 == 0) { *blk = 6; *vec = 2; }
        else if (r % 3 == 0) { *blk = 3; *vec = 1; }
        else if (r % 2 == 0) { *blk = 2; *vec = 2; }
        else { *blk = 1; *vec = 1; }
    } else {
        *blk = (r % 4 == 0) ? 4 : (r % 3 == 0) ? 3 : (r % 2 == 0) ? 2 : 1;
        *vec = 1;
    }
}

// Plan for the FP64 path (mixed == false) or the mixed path (FP32 chunk in shared memory).
tsqr_status_t plan_leaf(int64_t m, int n, const tsqr_plan_t *over, bool mixed, F64Plan *p);

tsqr_status_t plan_f64(int64_t m, int n, const tsqr_plan_t *over, F64Plan *p) {
    return plan_leaf(m, n, over, false, p);
}

tsqr_status_t plan_store(int64_t m, int n, const tsqr_plan_t *over, F64Plan *p);

// Shared memory of a leaf CTA holding an hs-row chunk with leading dimension ld.
size_t leaf_smem_bytes(int n, int hs, int ld, int warps, bool mixed) {
    return mixed ? mixed_smem_bytes(n, ld, warps) : f64_smem_bytes(n, hs, ld, warps);
}

// Largest r (rows per lane) whose shared memory, with hs = 32 r warps rows and the leading
// dimension its inner-loop vector width implies, fits `budget`.
int max_rows_per_lane_p(int n, int warps, size_t budget, bool mixed) {
    int best = 0;
    for (int r = 1; r <= 256; ++r) {
        int blk = 1, vec = 1;
        block_for(r, mixed, &blk, &vec);
        const int hs = 32 * warps * r;
        if (leaf_smem_bytes(n, hs, ld_for(hs, vec), warps, mixed) > budget) break;
        best = r;
    }
    return best;
}

// Plans chosen by tsqr_autotune, per (device, n, leaf precision, floor(log2 m)); the AUTO plan
// of a problem in a tuned bucket is the tuned plan.
struct TuneKey {
    int dev, n, mixed, mlog;
    bool operator<(const TuneKey &o) const {
        if (dev != o.dev) return dev < o.dev;
        if (n != o.n) return n < o.n;
        if (mixed != o.mixed) return mixed < o.mixed;
        return mlog < o.mlog;
    }
};
std::mutex g_tune_mu;
std::map<TuneKey, tsqr_plan_t> g_tuned;

int floor_log2(int64_t m) {
    int l = 0;
    while (l < 62 && ((int64_t)1 << (l + 1)) <= m) ++l;
    return l;
}

bool plan_is_auto(const tsqr_plan_t *p) {
    return !p || (p->tree == 0 && p->tile_rows == 0 && p->ctas == 0 && p->warps == 0 &&
                  p->arity == 0 && p->leaf == 0);
}

bool tuned_plan(int dev, int64_t m, int n, bool mixed, tsqr_plan_t *out) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tuned.find(TuneKey{dev, n, mixed ? 1 : 0, floor_log2(std::max<int64_t>(m, 1))});
    if (it == g_tuned.end()) return false;
    *out = it->second;
    return true;
}

// The rest of plan_leaf once the rows per lane that fit (r_fit) are chosen.
tsqr_status_t plan_with_r(int64_t m, int n, const tsqr_plan_t *over, bool mixed, int r_fit,
                          const DeviceInfo &di, F64Plan *p) {
    const int W = p->warps;
    if (r_fit < 1 || 32 * W * r_fit < n) return TSQR_ERR_UNSUPPORTED;
    r_fit = good_r(r_fit);
    const int64_t mm = std::max<int64_t>(m, 1);
    const bool tiled = (p->tree == TSQR_TREE_BINARY) || (over && over->tile_rows > 0);
    int r;
    if (tiled) {
        // work unit = one tile of b rows; a tile taller than fits on chip is folded in chunks
        p->unit = (over && over->tile_rows > 0) ? over->tile_rows : 256;
        r = (int)std::min<int64_t>(r_fit, (std::max<int64_t>(std::min<int64_t>(p->unit, mm), n) +
                                           32 * W - 1) / (32 * W));
        p->hs = 32 * W * r;
        p->h = (int)std::min<int64_t>(p->unit, p->hs);
    } else {
        // work unit = one slab as tall as fits (a slab taller than A only multiplies zeros)
        r = (int)std::min<int64_t>(r_fit, (std::max<int64_t>(mm, n) + 32 * W - 1) / (32 * W));
        p->hs = 32 * W * r;
        p->h = p->hs;
        p->unit = p->h;
    }
    if (p->hs < n) return TSQR_ERR_UNSUPPORTED;
    block_for(r, mixed, &p->blk, &p->vec);
    p->ldS = ld_for(p->hs, p->vec);
    p->smem = leaf_smem_bytes(n, p->hs, p->ldS, W, mixed);
    if (p->smem > di.smem_block_optin) return TSQR_ERR_UNSUPPORTED;
    p->nunits = (mm + p->unit - 1) / p->unit;
    int64_t leaves;
    if (p->tree == TSQR_TREE_FLAT) {
        leaves = 1;
    } else if (p->tree == TSQR_TREE_BINARY) {
        leaves = p->nunits;
    } else if (over && over->ctas > 0) {
        leaves = over->ctas;
    } else {
        if ((mixed ? mixed_prepare(p->smem) : f64_prepare(p->smem)) != cudaSuccess)
            return TSQR_ERR_CUDA;
        const int per_sm = std::max(1, mixed ? mixed_blocks_per_sm(W, p->smem)
                                             : f64_blocks_per_sm(W, p->smem));
        leaves = (int64_t)di.sms * per_sm;
    }
    leaves = std::min<int64_t>(leaves, p->nunits);
    if (leaves < 1 || leaves > 0x7fffffffLL) return TSQR_ERR_UNSUPPORTED;
    p->nleaves = (int)leaves;
    // tree arity: 2 (the paper's binary operator) for the BINARY tree, else as many stacked
    // triangles as the S region holds (at most 8), unless the plan says otherwise
    const int s_avail = mixed ? mixed_s_doubles(n, p->ldS) : p->ldS * n;
    if (p->tree == TSQR_TREE_BINARY) {
        p->arity = 2;
    } else if (over && over->arity > 0) {
        if (over->arity < 2 || over->arity > 8) return TSQR_ERR_INVALID_ARG;
        p->arity = over->arity;
        if (tree_ldsd(n, p->arity) * n > s_avail) return TSQR_ERR_UNSUPPORTED;
    } else {
        p->arity = arity_for(n, s_avail);
    }
    p->ldSd = mixed ? tree_ldsd(n, p->arity) : p->ldS;
    p->s_doubles = mixed ? mixed_s_doubles_of(n, p->ldS, p->arity) : p->ldS * n;
    if (!mixed && tree_ldsd(n, p->arity) > p->ldS) return TSQR_ERR_UNSUPPORTED;
    return build_tree(leaves, p->arity, &p->shape, &p->nodes);
}

// FP64 bulk warps of the AUTO plan past 55 columns (one reduction of a matrix too short for
// the PANELS tree): from a sweep of every n = 2 .. 128 at 4,194,304 rows with 4, 8 and 12 bulk
// warps, 8 or 12 where that was at least 2% faster than 4 (80-90: +40% with 8, where four
// warps drop to one CTA per SM; 56-64 with 12: +4-5%).
int f64_auto_warps_wide(int n) {
    if (n >= 80 && n <= 90) return 8;
    if (n >= 56 && n <= 64) return 12;
    return 4;
}

// FP64 AUTO leaf shape for n <= 55: bulk warps W and resident CTAs per SM k (the chunk as tall
// as k CTAs per SM allow).  From sweeps of every W = 3 .. 12 and k = 1 .. 3 (with chunks of 1 to
// 12 rows per lane) for each n = 1 .. 55 at 4,194,304 rows: a width keeps (4, 2) unless a
// setting was at least 1% faster (ms, (4, 2) against the table's): n = 9: 0.985 / 0.914 (5, 3);
// 13: 2.00 / 1.85 (5, 2); 18: 3.76 / 3.28 (8, 1); 20: 4.46 / 4.14 (7, 1) (2^24 rows: 17.24 /
// 15.73); 22: 5.16 / 4.91 (4, 3); 27: 7.60 / 7.23 (5, 2); 36: 14.06 / 13.27 (5, 2) (2^24 rows:
// 54.70 / 50.76); 40: 16.88 / 16.27 (7, 1); 44: 20.12 / 19.77 (9, 1); 52: 29.55 / 28.19 (6, 2).
struct LeafShape {
    int W, k;
};
LeafShape f64_auto_shape(int n) {
    struct Entry {
        int lo, hi, W, k;
    };
    static const Entry kTable[] = {
        {5, 5, 8, 2},   {7, 7, 9, 2},   {8, 8, 8, 2},   {9, 9, 5, 3},   {13, 14, 5, 2},
        {18, 18, 8, 1}, {19, 20, 7, 1}, {21, 22, 4, 3}, {23, 23, 6, 2}, {24, 25, 5, 3},
        {26, 27, 5, 2}, {35, 35, 8, 1}, {36, 39, 5, 2}, {40, 40, 7, 1}, {41, 41, 3, 3},
        {42, 46, 9, 1}, {49, 51, 8, 1}, {52, 55, 6, 2}};
    for (const Entry &e : kTable)
        if (n >= e.lo && n <= e.hi) return LeafShape{e.W, e.k};
    if (n > 55) return LeafShape{f64_auto_warps_wide(n), 2};
    return LeafShape{4, 2};
}

tsqr_status_t plan_leaf(int64_t m, int n, const tsqr_plan_t *over, bool mixed, F64Plan *p) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return TSQR_ERR_CUDA;
    const DeviceInfo di = device_info(dev);
    if (di.sms <= 0) return TSQR_ERR_CUDA;
    tsqr_plan_t tuned;
    if (plan_is_auto(over) && tuned_plan(dev, m, n, mixed, &tuned) &&
        tuned.tree != TSQR_TREE_PANELS)
        over = &tuned;
    p->tree = (over && over->tree) ? over->tree : TSQR_TREE_HYBRID;
    if (p->tree < TSQR_TREE_BINARY || p->tree > TSQR_TREE_HYBRID) return TSQR_ERR_INVALID_ARG;
    if (over && over->leaf != 0 && (!mixed || over->leaf != TSQR_LEAF_FOLD))
        return TSQR_ERR_INVALID_ARG;
    p->leaf = mixed ? TSQR_LEAF_FOLD : 0;
    // bulk warps: 8 for the mixed path from n = 48 on, whose latency-bound FP32 sweep gains
    // from two warps per sub-partition (2^24 x 64 FP32: 47.2 against 52.1 ms with 4, 52.1 with
    // 12), and 12 from n = 96 on where they fit (2^24 x 96: FP32 143.6 against 177.4 ms, BF16
    // 156.5 against 197.7); FP64 by width
    const LeafShape shape = f64_auto_shape(n);
    p->warps = mixed ? (n >= 96 ? 12 : n >= 48 ? 8 : 4) : shape.W;
    if (over && over->warps) {
        if (over->warps < 1 || over->warps > 12) return TSQR_ERR_INVALID_ARG;
        p->warps = over->warps;
    }
    if (over && (over->tile_rows < 0 || over->ctas < 0 || over->arity < 0))
        return TSQR_ERR_INVALID_ARG;
    int W = p->warps;
    const size_t reserve = 1024;
    const size_t three_per_sm = (di.smem_sm > 3 * reserve) ? (di.smem_sm - 3 * reserve) / 3 : 0;
    const size_t two_per_sm = (di.smem_sm > 2 * reserve) ? (di.smem_sm - 2 * reserve) / 2 : 0;
    const size_t one_per_sm = std::min(di.smem_block_optin, di.smem_sm - reserve);
    int r2 = max_rows_per_lane_p(n, W, two_per_sm, mixed);
    int r1 = max_rows_per_lane_p(n, W, one_per_sm, mixed);
    if (mixed && W == 12 && !(over && over->warps) && r1 < 1) {  // 12 warps do not fit: 8
        W = 8;
        p->warps = 8;
        r2 = max_rows_per_lane_p(n, W, two_per_sm, mixed);
        r1 = max_rows_per_lane_p(n, W, one_per_sm, mixed);
    }
    // FP64: two CTAs per SM hide each other's per-column serial work (the reflector chain,
    // the barriers), which pays even at one row per lane (measured at n = 16, 32, 64).
    // Mixed: the FP32 bulk is cheap, so what counts is the number of rows sharing each
    // reflector's serial FP64 work, i.e. the rows held on chip per SM (ties go to two CTAs).
    // FP64 AUTO widths (n <= 55, bulk warps not given) take the table's CTAs per SM: k = 1 one,
    // k = 3 three where their chunk holds a row per lane, else two.
    const bool auto_shape = !mixed && n <= 55 && !(over && over->warps);
    const bool two = mixed ? (r2 >= 1 && 2 * good_r(r2) >= good_r(r1))
                           : (r2 >= 1 && !(auto_shape && shape.k == 1));
    const int r3 = (auto_shape && shape.k == 3) ? max_rows_per_lane_p(n, W, three_per_sm, mixed) : 0;
    // explicit tile rows are honoured up to what one CTA per SM holds
    const bool tile_given = over && over->tile_rows > 0;
    const int r_auto = r3 >= 1 ? r3 : two ? r2 : r1;
    tsqr_status_t st = plan_with_r(m, n, over, mixed, tile_given ? r1 : r_auto, di, p);
    // an explicit arity whose stacked triangles need a taller S region than two CTAs per SM
    // leave room for: one CTA per SM
    if (st == TSQR_ERR_UNSUPPORTED && two && over && over->arity > 0)
        st = plan_with_r(m, n, over, mixed, r1, di, p);
    return st;
}

// Workspace for (current device, stream): at least `bytes` bytes plus a status word.
tsqr_status_t get_workspace(cudaStream_t stream, size_t bytes, Workspace **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return TSQR_ERR_CUDA;
    std::lock_guard<std::mutex> lk(g_mu);
    Workspace &w = g_ws[{dev, stream}];
    if (!w.status) {
        if (cudaMallocAsync((void **)&w.status, 256, stream) != cudaSuccess) return TSQR_ERR_ALLOC;
        if (cudaMemsetAsync(w.status, 0, sizeof(int), stream) != cudaSuccess) return TSQR_ERR_CUDA;
    }
    if (bytes > w.bytes) {
        if (w.base) cudaFreeAsync(w.base, stream);
        w.base = nullptr;
        w.bytes = 0;
        w.table.clear();
        const size_t nb = align_up(bytes, 1 << 20);
        if (cudaMallocAsync(&w.base, nb, stream) != cudaSuccess) return TSQR_ERR_ALLOC;
        w.bytes = nb;
    }
    *out = &w;
    return TSQR_SUCCESS;
}

tsqr_status_t zero_r(double *R, int64_t n, int64_t ldr, cudaStream_t stream) {
    if (cudaMemset2DAsync(R, (size_t)ldr * sizeof(double), 0, (size_t)n * sizeof(double),
                          (size_t)n, stream) != cudaSuccess)
        return TSQR_ERR_CUDA;
    return TSQR_SUCCESS;
}

tsqr_status_t run_caqr(const double *A, int64_t m, int64_t N, int64_t lda, double *R,
                       int64_t ldr, int64_t nb, const tsqr_plan_t *over, cudaStream_t stream);

// Panels (TSQR_TREE_PANELS): the AUTO plan of a tall FP64 matrix from n = 56 on, where the one
// reduction's leaves hold one CTA per SM and n reflectors per chunk, while panels of 16 columns
// (each a TSQR reduction of its own, then Q^T applied to the columns right of it) keep the
// leaves small and the updates blocked: 4,194,304 rows, n = 56 / 64 / 96 / 128: 775 / 828 /
// 863 / 887 against 727 / 750 / 555 / 586 GFLOP/s (n = 48: 802 against 826, so one reduction
// below 56).  Returns the panel width, or 0 for one reduction.
constexpr int kPanelsMinN = 56;
constexpr int kPanelsWidth = 16;

int64_t panels_width(int64_t m, int64_t n, const tsqr_plan_t *over, int dev) {
    tsqr_plan_t tuned;
    if (plan_is_auto(over) && tuned_plan(dev, m, (int)n, false, &tuned)) over = &tuned;
    if (over && over->tree == TSQR_TREE_PANELS)
        return over->tile_rows > 0 ? over->tile_rows : kPanelsWidth;
    if (plan_is_auto(over) && (n > TSQR_MAX_N || (n >= kPanelsMinN && m >= 8 * n)))
        return kPanelsWidth;  // past TSQR_MAX_N only panels run
    return 0;
}

tsqr_status_t run_f64(const double *A, int64_t m, int64_t n, int64_t lda, double *R, int64_t ldr,
                      const tsqr_plan_t *over, cudaStream_t stream) {
    g_last_launches = 0;
    g_last_plan = tsqr_plan_t{};
    if (n == 0) return TSQR_SUCCESS;
    if (m == 0) return zero_r(R, n, ldr, stream);
    {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess) return TSQR_ERR_CUDA;
        const int64_t nb = panels_width(m, n, over, dev);
        if (nb > 0) {
            if (nb > TSQR_MAX_N) return TSQR_ERR_INVALID_ARG;
            if (m < n) return n > TSQR_MAX_N ? TSQR_ERR_UNSUPPORTED : TSQR_ERR_INVALID_ARG;
            const tsqr_status_t st = run_caqr(A, m, n, lda, R, ldr, nb, nullptr, stream);
            g_last_plan = tsqr_plan_t{};
            if (st == TSQR_SUCCESS) {
                g_last_plan.tree = TSQR_TREE_PANELS;
                g_last_plan.tile_rows = (int32_t)nb;
            }
            return st;
        }
    }
    if (n > TSQR_MAX_N) return TSQR_ERR_UNSUPPORTED;
    F64Plan p;
    tsqr_status_t st = plan_f64(m, (int)n, over, &p);
    if (st != TSQR_SUCCESS) return st;
    g_last_plan = public_plan(p);
    if (f64_prepare(p.smem) != cudaSuccess) return TSQR_ERR_CUDA;
    const size_t cnt_bytes = align_up((size_t)p.nodes * sizeof(unsigned int), 256);
    const size_t slot_bytes = (size_t)p.nodes * (size_t)n * (size_t)n * sizeof(double);
    Workspace *ws = nullptr;
    st = get_workspace(stream, cnt_bytes + slot_bytes, &ws);
    if (st != TSQR_SUCCESS) return st;
    F64Args a = plan_args(p, A, m, n, lda);
    a.counters = (unsigned int *)ws->base;
    a.slots = (double *)((char *)ws->base + cnt_bytes);
    a.R = R;
    a.ldr = ldr;
    a.status = ws->status;
    if (cudaMemsetAsync(a.counters, 0, (size_t)p.nodes * sizeof(unsigned int), stream) != cudaSuccess)
        return TSQR_ERR_CUDA;
    if (f64_launch(a, p.warps, p.smem, stream) != cudaSuccess) return TSQR_ERR_CUDA;
    g_last_launches = 1;
    return TSQR_SUCCESS;
}

// Thin QR: the FP64 factorization with its reflectors kept, then the Q passes (tsqr_qr.cu).
// Workspace: counters | tree slots | chunk scalars | node tails | node scalars | node blocks |
// signs.
tsqr_status_t run_qr(const double *A, int64_t m, int64_t n, int64_t lda, double *Q, int64_t ldq,
                     double *R, int64_t ldr, const tsqr_plan_t *over, cudaStream_t stream) {
    g_last_launches = 0;
    g_last_plan = tsqr_plan_t{};
    F64Plan p;
    tsqr_status_t st = plan_store(m, (int)n, over, &p);
    if (st != TSQR_SUCCESS) return st;
    g_last_plan = public_plan(p);
    if (p.unit % p.h != 0) return TSQR_ERR_UNSUPPORTED;  // chunk ids = first row / h
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return TSQR_ERR_CUDA;
    const DeviceInfo di = device_info(dev);
    // the leaf pass has no serial reflector chain, so more, shorter warps hide its latency:
    // 12 or 8 bulk warps (three or two per sub-partition) where they divide the chunk
    int qwarps = p.warps;
    for (int c : {12, 8})
        if (c > qwarps && p.hs % (32 * c) == 0) {
            qwarps = c;
            break;
        }
    const int qr_rows = p.hs / (32 * qwarps);
    int qblk = 1;
    for (int c = 4; c >= 1; --c)
        if (qr_rows % c == 0) {
            qblk = c;
            break;
        }
    // column groups: Q's columns (and the carried blocks') are independent, so the leaf pass
    // takes them qn at a time and the tree pass qg at a time where all n do not fit
    int qn = (int)n, qg = (int)n;
    // the blocked leaf pass (compact WY factors per chunk) where a chunk's tails and two n x n
    // blocks fit one CTA, else the sweep
    const int ldX = p.h | 1;
    const size_t wy_smem = wy_smem_bytes((int)n, ldX);
    bool wyq = wy_smem <= di.smem_block_optin;
    if (wyq) {
        while (qn > 8 && q_leaf_wy_smem_bytes((int)n, qn, p.ldS, false) > di.smem_block_optin)
            qn = (qn + 1) / 2;
        wyq = q_leaf_wy_smem_bytes((int)n, qn, p.ldS, false) <= di.smem_block_optin;
        if (!wyq) qn = (int)n;
    }
    if (!wyq)
        while (qn > 8 && q_leaf_smem_bytes((int)n, qn, p.ldS, qwarps) > di.smem_block_optin)
            qn = (qn + 1) / 2;
    while (qg > 8 && q_tree_smem_bytes((int)n, p.arity, qg) > di.smem_block_optin)
        qg = (qg + 1) / 2;
    // one column group: the leaf pass forms each chunk's S itself from the tails it loads anyway
    const bool fuse = wyq && qn == n &&
                      q_leaf_wy_smem_bytes((int)n, qn, p.ldS, true) <= di.smem_block_optin;
    const size_t leaf_smem = wyq ? q_leaf_wy_smem_bytes((int)n, qn, p.ldS, fuse)
                                 : q_leaf_smem_bytes((int)n, qn, p.ldS, qwarps);
    const size_t tree_smem = q_tree_smem_bytes((int)n, p.arity, qg);
    if (leaf_smem > di.smem_block_optin || tree_smem > di.smem_block_optin)
        return TSQR_ERR_UNSUPPORTED;
    const bool grouped = qn < n;  // then the tails cannot live in Q: later groups still read them
    if (qr_prepare(p.smem, wyq ? 0 : leaf_smem, tree_smem) != cudaSuccess) return TSQR_ERR_CUDA;
    const int64_t nchunks = (m + p.h - 1) / p.h;
    const size_t nn = (size_t)n * (size_t)n;
    const size_t wys_bytes =
        (wyq && !fuse) ? align_up((size_t)nchunks * nn * sizeof(double), 256) : 0;
    const size_t cnt_bytes = align_up((size_t)p.nodes * sizeof(unsigned int), 256);
    const size_t slot_bytes = align_up((size_t)p.nodes * nn * sizeof(double), 256);
    const size_t csc_bytes = align_up((size_t)nchunks * 2 * n * sizeof(double), 256);
    const size_t nv_bytes = align_up((size_t)p.nodes * (p.arity - 1) * nn * sizeof(double), 256);
    const size_t nsc_bytes = align_up((size_t)p.nodes * 2 * n * sizeof(double), 256);
    const size_t blk_bytes = align_up((size_t)p.nodes * nn * sizeof(double), 256);
    const size_t sgn_bytes = align_up((size_t)n * sizeof(double), 256);
    const size_t v_bytes = grouped ? align_up((size_t)m * (size_t)n * sizeof(double), 256) : 0;
    Workspace *ws = nullptr;
    st = get_workspace(stream, cnt_bytes + slot_bytes + csc_bytes + nv_bytes + nsc_bytes +
                                   blk_bytes + sgn_bytes + v_bytes + wys_bytes, &ws);
    if (st != TSQR_SUCCESS) return st;
    char *base = (char *)ws->base;
    F64Args a = plan_args(p, A, m, n, lda);
    a.counters = (unsigned int *)base;
    a.slots = (double *)(base + cnt_bytes);
    a.R = R;
    a.ldr = ldr;
    a.status = ws->status;
    size_t o = cnt_bytes + slot_bytes;
    a.q.V = Q;
    a.q.ldv = ldq;
    a.q.chunk_sc = (double *)(base + o);
    o += csc_bytes;
    a.q.node_V = (double *)(base + o);
    o += nv_bytes;
    a.q.node_sc = (double *)(base + o);
    o += nsc_bytes;
    double *blocks = (double *)(base + o);
    o += blk_bytes;
    a.q.signs = (double *)(base + o);
    o += sgn_bytes;
    if (grouped) {
        a.q.V = (double *)(base + o);
        a.q.ldv = m;
    }
    o += v_bytes;
    double *wyS = (double *)(base + o);
    if (cudaMemsetAsync(a.counters, 0, (size_t)p.nodes * sizeof(unsigned int), stream) !=
        cudaSuccess)
        return TSQR_ERR_CUDA;
    if (qr_factor_launch(a, p.warps, p.smem, stream) != cudaSuccess) return TSQR_ERR_CUDA;
    int launches = 1;
    if (wyq && !fuse) {
        const WyArgs wa = wy_args(p, a.q, m, (int)n, ldX, wyS);
        const int grid = (int)std::min<int64_t>(nchunks, 4LL * di.sms);
        if (wy_launch(wa, wy_smem, grid, stream) != cudaSuccess) return TSQR_ERR_CUDA;
        ++launches;
    }
    // tree pass, from the root's level down to level 1 (whose children are the leaves)
    const TreeShape &sh = p.shape;
    for (int L = sh.levels - 1; L >= 1; --L) {
        QTreeArgs t;
        t.n = (int)n;
        t.arity = p.arity;
        t.level_off = sh.offset[L];
        t.child_cnt = sh.count[L - 1];
        t.child_off = sh.offset[L - 1];
        t.is_root = (L == sh.levels - 1) ? 1 : 0;
        t.node_V = a.q.node_V;
        t.node_sc = a.q.node_sc;
        t.signs = a.q.signs;
        t.B = blocks;
        t.qg = qg;
        if (q_tree_launch(t, sh.count[L], tree_smem, stream) != cudaSuccess) return TSQR_ERR_CUDA;
        ++launches;
    }
    QLeafArgs l;
    l.Q = Q;
    l.m = m;
    l.ldq = ldq;
    l.n = (int)n;
    l.unit = p.unit;
    l.nunits = p.nunits;
    l.nleaves = p.nleaves;
    l.h = p.h;
    l.hs = p.hs;
    l.ldS = p.ldS;
    l.chunk_sc = a.q.chunk_sc;
    l.B = blocks;
    l.signs = a.q.signs;
    l.single = (sh.levels == 1) ? 1 : 0;
    l.V = a.q.V;
    l.ldv = a.q.ldv;
    l.wyS = fuse ? nullptr : wyS;
    for (int q0 = 0; q0 < n; q0 += qn) {
        l.q0 = q0;
        l.qn = (int)std::min<int64_t>(qn, n - q0);
        if ((wyq ? q_leaf_wy_launch(l, leaf_smem, stream)
                 : q_leaf_launch(l, qblk, qwarps, leaf_smem, stream)) != cudaSuccess)
            return TSQR_ERR_CUDA;
        ++launches;
    }
    g_last_launches = launches;
    return TSQR_SUCCESS;
}

// Host-input FP64 call: A and R in host memory.
// Host input where the AUTO plan runs by panels (n >= 56, tall): A copied whole into a buffer
// of this call (stream-ordered; the panels take the stream's pooled workspace themselves), the
// panels, and R copied back.  The panels' updates read every column more than once, so A is
// brought to HBM first.
tsqr_status_t run_host_panels(const double *A, int64_t m, int64_t n, int64_t lda, double *R,
                              int64_t ldr, int64_t nb, cudaStream_t stream) {
    double *Ad = nullptr, *Rd = nullptr;
    if (cudaMallocAsync((void **)&Ad, (size_t)m * n * sizeof(double), stream) != cudaSuccess)
        return TSQR_ERR_ALLOC;
    if (cudaMallocAsync((void **)&Rd, (size_t)n * n * sizeof(double), stream) != cudaSuccess) {
        cudaFreeAsync(Ad, stream);
        return TSQR_ERR_ALLOC;
    }
    tsqr_status_t st = TSQR_SUCCESS;
    if (cudaMemcpy2DAsync(Ad, (size_t)m * sizeof(double), A, (size_t)lda * sizeof(double),
                          (size_t)m * sizeof(double), (size_t)n, cudaMemcpyHostToDevice,
                          stream) != cudaSuccess)
        st = TSQR_ERR_CUDA;
    int launches = 0;
    if (st == TSQR_SUCCESS) {
        st = run_caqr(Ad, m, n, m, Rd, n, nb, nullptr, stream);
        launches = g_last_launches;
    }
    if (st == TSQR_SUCCESS &&
        cudaMemcpy2DAsync(R, (size_t)ldr * sizeof(double), Rd, (size_t)n * sizeof(double),
                          (size_t)n * sizeof(double), (size_t)n, cudaMemcpyDeviceToHost,
                          stream) != cudaSuccess)
        st = TSQR_ERR_CUDA;
    cudaFreeAsync(Ad, stream);
    cudaFreeAsync(Rd, stream);
    g_last_launches = st == TSQR_SUCCESS ? launches : 0;
    g_last_plan = tsqr_plan_t{};
    if (st == TSQR_SUCCESS) {
        g_last_plan.tree = TSQR_TREE_PANELS;
        g_last_plan.tile_rows = (int32_t)nb;
    }
    return st;
}

// The device address of page-locked host memory, or null for memory the device cannot address
// in place (pageable memory, or a registration without a device mapping).
const double *mapped_device_ptr(const double *A) {
    cudaPointerAttributes attr;
    const double *d = nullptr;
    if (cudaPointerGetAttributes(&attr, A) == cudaSuccess && attr.type == cudaMemoryTypeHost)
        d = static_cast<const double *>(attr.devicePointer);
    cudaGetLastError();  // an unregistered pointer may leave an error behind
    return d;
}

// One reduction (the AUTO plan, as tsqr_r) on host A.  Page-locked A is read in place: the
// leaves' cp.async loads go through the device mapping of A's pages (NVLink-C2C on a Grace
// host), so the transfer of A is spread over the whole factorization and overlaps it without a
// second stream, flags or waits; the kernel is tsqr_r's, with tsqr_r's plan, so R is tsqr_r's
// bit for bit.  Other host memory is copied whole to a device buffer of the workspace first.
// Workspace: counters | tree slots | R (ld n) | [A (ld m), when staged].
tsqr_status_t run_f64_host(const double *A, int64_t m, int64_t n, int64_t lda, double *R,
                           int64_t ldr, cudaStream_t stream) {
    g_last_launches = 0;
    g_last_plan = tsqr_plan_t{};
    if (n == 0) return TSQR_SUCCESS;
    if (m == 0) {
        for (int64_t c = 0; c < n; ++c)
            for (int64_t i = 0; i < n; ++i) R[i + c * ldr] = 0.0;
        return TSQR_SUCCESS;
    }
    {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess) return TSQR_ERR_CUDA;
        const int64_t nb = panels_width(m, n, nullptr, dev);
        if (nb > 0) return run_host_panels(A, m, n, lda, R, ldr, nb, stream);
    }
    const double *Amapped = mapped_device_ptr(A);
    F64Plan p;
    tsqr_status_t st = plan_f64(m, (int)n, nullptr, &p);
    if (st != TSQR_SUCCESS) return st;
    g_last_plan = public_plan(p);
    if (f64_prepare(p.smem) != cudaSuccess) return TSQR_ERR_CUDA;
    const size_t cnt_bytes = align_up((size_t)p.nodes * sizeof(unsigned int), 256);
    const size_t slot_bytes = align_up((size_t)p.nodes * (size_t)n * (size_t)n * sizeof(double), 256);
    const size_t r_bytes = align_up((size_t)n * (size_t)n * sizeof(double), 256);
    const size_t a_bytes = Amapped ? 0 : (size_t)m * (size_t)n * sizeof(double);
    Workspace *ws = nullptr;
    st = get_workspace(stream, cnt_bytes + slot_bytes + r_bytes + a_bytes, &ws);
    if (st != TSQR_SUCCESS) return st;
    char *base = (char *)ws->base;
    double *Rd = (double *)(base + cnt_bytes + slot_bytes);
    const double *Ain = Amapped;
    int64_t ld_in = lda;
    if (!Amapped) {
        double *Ad = (double *)(base + cnt_bytes + slot_bytes + r_bytes);
        if (cudaMemcpy2DAsync(Ad, (size_t)m * sizeof(double), A, (size_t)lda * sizeof(double),
                              (size_t)m * sizeof(double), (size_t)n, cudaMemcpyHostToDevice,
                              stream) != cudaSuccess)
            return TSQR_ERR_CUDA;
        Ain = Ad;
        ld_in = m;
    }
    F64Args a = plan_args(p, Ain, m, n, ld_in);
    a.counters = (unsigned int *)base;
    a.slots = (double *)(base + cnt_bytes);
    a.R = Rd;
    a.ldr = n;
    a.status = ws->status;
    if (cudaMemsetAsync(a.counters, 0, (size_t)p.nodes * sizeof(unsigned int), stream) !=
            cudaSuccess ||
        f64_launch(a, p.warps, p.smem, stream) != cudaSuccess)
        return TSQR_ERR_CUDA;
    if (cudaMemcpy2DAsync(R, (size_t)ldr * sizeof(double), Rd, (size_t)n * sizeof(double),
                          (size_t)n * sizeof(double), (size_t)n, cudaMemcpyDeviceToHost,
                          stream) != cudaSuccess)
        return TSQR_ERR_CUDA;
    g_last_launches = 1;
    return TSQR_SUCCESS;
}

// Least squares with few right-hand sides (k <= max(1, n / 4), n + k <= TSQR_MAX_N): the R factor of the augmented
// matrix [A | B] holds R in its leading n x n block and (Q^T B)(0:n, :) beside it (the first n
// reflectors are A's own; the sign convention negates whole rows, which keeps R X = C), so one
// factorization of [A | B] and one triangular solve give X.  Workspace: counters | slots |
// [A | B] (ld m) | R of [A | B].
tsqr_status_t run_lstsq_augmented(const double *A, int64_t m, int64_t n, int64_t lda,
                                  const double *B, int64_t ldb, int64_t k, double *X, int64_t ldx,
                                  double *R, int64_t ldr, const tsqr_plan_t *over,
                                  cudaStream_t stream) {
    const int64_t na = n + k;
    F64Plan p;
    tsqr_status_t st = plan_f64(m, (int)na, over, &p);
    if (st != TSQR_SUCCESS) return st;
    g_last_plan = public_plan(p);
    if (f64_prepare(p.smem) != cudaSuccess) return TSQR_ERR_CUDA;
    const size_t cnt_bytes = align_up((size_t)p.nodes * sizeof(unsigned int), 256);
    const size_t slot_bytes = align_up((size_t)p.nodes * (size_t)na * na * sizeof(double), 256);
    const size_t aug_bytes = align_up((size_t)m * (size_t)na * sizeof(double), 256);
    const size_t ra_bytes = (size_t)na * na * sizeof(double);
    Workspace *ws = nullptr;
    st = get_workspace(stream, cnt_bytes + slot_bytes + aug_bytes + ra_bytes, &ws);
    if (st != TSQR_SUCCESS) return st;
    char *base = (char *)ws->base;
    double *aug = (double *)(base + cnt_bytes + slot_bytes);
    double *Ra = (double *)(base + cnt_bytes + slot_bytes + aug_bytes);
    if (cudaMemcpy2DAsync(aug, (size_t)m * sizeof(double), A, (size_t)lda * sizeof(double),
                          (size_t)m * sizeof(double), (size_t)n, cudaMemcpyDeviceToDevice,
                          stream) != cudaSuccess ||
        cudaMemcpy2DAsync(aug + n * m, (size_t)m * sizeof(double), B, (size_t)ldb * sizeof(double),
                          (size_t)m * sizeof(double), (size_t)k, cudaMemcpyDeviceToDevice,
                          stream) != cudaSuccess ||
        cudaMemsetAsync(base, 0, (size_t)p.nodes * sizeof(unsigned int), stream) != cudaSuccess)
        return TSQR_ERR_CUDA;
    F64Args a = plan_args(p, aug, m, na, m);
    a.counters = (unsigned int *)base;
    a.slots = (double *)(base + cnt_bytes);
    a.R = Ra;
    a.ldr = na;
    a.status = ws->status;
    if (f64_launch(a, p.warps, p.smem, stream) != cudaSuccess) return TSQR_ERR_CUDA;
    if (R && cudaMemcpy2DAsync(R, (size_t)ldr * sizeof(double), Ra, (size_t)na * sizeof(double),
                               (size_t)n * sizeof(double), (size_t)n, cudaMemcpyDeviceToDevice,
                               stream) != cudaSuccess)
        return TSQR_ERR_CUDA;
    if (trsm_launch(Ra, na, Ra + n * na, na, X, ldx, (int)n, (int)k, ws->status, stream) !=
        cudaSuccess)
        return TSQR_ERR_CUDA;
    g_last_launches = 2;
    return TSQR_SUCCESS;
}

// Compact WY factors fit when a chunk's scaled tails and two n x n blocks fit one CTA; the
// blocked apply then takes as many update columns per CTA as fit beside the chunk.
bool plan_wy(int w, const F64Plan &p, const DeviceInfo &di, int *ldX, size_t *wy_smem, int *kc,
             size_t *qt_smem) {
    *ldX = p.h | 1;
    *wy_smem = wy_smem_bytes(w, *ldX);
    if (*wy_smem > di.smem_block_optin) return false;
    int k = w;
    while (k > 8 && qt_wy_smem_bytes(w, k, p.ldS) > di.smem_block_optin) k = (k + 1) / 2;
    *kc = k;
    *qt_smem = qt_wy_smem_bytes(w, k, p.ldS);
    return *qt_smem <= di.smem_block_optin;
}

// The plan of a factorization whose reflectors the Q and Q^T passes apply: tsqr_r's, unless
// that is the AUTO plan and its chunks are too tall for the blocked passes' buffers (some wide
// n where the AUTO plan takes 8 or 12 bulk warps); then the four-warp plan.  tsqr_last_plan
// reports which.
tsqr_status_t plan_store(int64_t m, int n, const tsqr_plan_t *over, F64Plan *p) {
    // the passes that keep and apply the reflectors run 4, 8 or 12 bulk warps
    if (over && over->warps % 4 != 0) return TSQR_ERR_INVALID_ARG;
    tsqr_status_t st = plan_f64(m, n, over, p);
    if (st != TSQR_SUCCESS || p->warps == 4) return st;
    if (p->warps % 4 == 0) {
        if (!plan_is_auto(over)) return st;
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess) return TSQR_ERR_CUDA;
        const DeviceInfo di = device_info(dev);
        int ldX = 0, kc = 0;
        size_t wy = 0, qt = 0;
        if (plan_wy(n, *p, di, &ldX, &wy, &kc, &qt) &&
            q_leaf_wy_smem_bytes(n, std::min(n, 8), p->ldS, false) <= di.smem_block_optin)
            return st;
    }
    // an AUTO (or tuned) width with other warp counts, or 8 / 12 whose blocked Q pass does not
    // fit: four bulk warps, the plan's other fields kept
    tsqr_plan_t w4 = plan_is_auto(over) ? tsqr_plan_t{} : *over;
    w4.warps = 4;
    return plan_f64(m, n, &w4, p);
}

// tsqr_lstsq's stored-reflector path with each chunk's reflectors applied as one compact WY
// block: the factorization, the chunks' S factors, one apply launch over every column of B
// (groups of kg on the grid; only T is kept, so the chunk's rows of Q^T B are never formed)
// and one triangular solve.
tsqr_status_t run_lstsq_wy(const double *A, int64_t m, int64_t n, int64_t lda, const double *B,
                           int64_t ldb, int64_t k, double *X, int64_t ldx, double *R, int64_t ldr,
                           const F64Plan &p, int ldX, size_t wy_smem, int kg, size_t qtw_smem,
                           const DeviceInfo &di, cudaStream_t stream) {
    if (qr_prepare(p.smem, 0, 0) != cudaSuccess) return TSQR_ERR_CUDA;
    const int64_t nchunks = (m + p.h - 1) / p.h;
    const int64_t groups = k > 0 ? (k + kg - 1) / kg : 0;
    if (groups > 65535) return TSQR_ERR_UNSUPPORTED;  // one grid row per column group
    const size_t nn = (size_t)n * (size_t)n;
    const size_t sizes[] = {
        (size_t)p.nodes * sizeof(unsigned int),                    // factorization counters
        (size_t)p.nodes * nn * sizeof(double),                     // factorization slots
        (size_t)m * (size_t)n * sizeof(double),                    // chunk tails
        (size_t)nchunks * 2 * n * sizeof(double),                  // chunk tau, c
        (size_t)p.nodes * (p.arity - 1) * nn * sizeof(double),     // node tails
        (size_t)p.nodes * 2 * n * sizeof(double),                  // node tau, c
        (size_t)n * sizeof(double),                                // root signs
        (size_t)groups * p.nodes * sizeof(unsigned int),           // apply counters
        (size_t)groups * p.nodes * n * kg * sizeof(double),        // apply slots
        (size_t)n * (size_t)k * sizeof(double),                    // (Q^T B)(0:n, :)
        (size_t)nchunks * nn * sizeof(double),                     // S per chunk
        R ? (size_t)0 : nn * sizeof(double)};                      // R when the caller has none
    constexpr int kBufs = sizeof(sizes) / sizeof(sizes[0]);
    size_t total = 0;
    for (size_t b : sizes) total += align_up(b, 256);
    Workspace *ws = nullptr;
    tsqr_status_t st = get_workspace(stream, total, &ws);
    if (st != TSQR_SUCCESS) return st;
    char *bufs[kBufs];
    size_t o = 0;
    for (int i = 0; i < kBufs; ++i) {
        bufs[i] = (char *)ws->base + o;
        o += align_up(sizes[i], 256);
    }
    if (!R) {
        R = (double *)bufs[11];
        ldr = n;
    }
    F64Args a = plan_args(p, A, m, n, lda);
    a.counters = (unsigned int *)bufs[0];
    a.slots = (double *)bufs[1];
    a.R = R;
    a.ldr = ldr;
    a.status = ws->status;
    a.q.V = (double *)bufs[2];
    a.q.ldv = m;
    a.q.chunk_sc = (double *)bufs[3];
    a.q.node_V = (double *)bufs[4];
    a.q.node_sc = (double *)bufs[5];
    a.q.signs = (double *)bufs[6];
    const WyArgs wa = wy_args(p, a.q, m, (int)n, ldX, (double *)bufs[10]);
    QtArgs t = qt_args(p, a.q, m, (int)n, B, ldb, kg, (int)k);
    t.counters = (unsigned int *)bufs[7];
    t.slots = (double *)bufs[8];
    t.C = (double *)bufs[9];
    t.ldc = n;
    t.wyS = wa.S;
    const int grid = (int)std::min<int64_t>(nchunks, 4LL * di.sms);
    // one column group: the apply forms each chunk's S itself from the tails it loads anyway
    const bool fuse = groups == 1 && qt_wy_smem_bytes((int)n, kg, p.ldS, true) <= di.smem_block_optin;
    if (fuse) {
        t.wyS = nullptr;
        qtw_smem = qt_wy_smem_bytes((int)n, kg, p.ldS, true);
    }
    if (cudaMemsetAsync(a.counters, 0, (size_t)p.nodes * sizeof(unsigned int), stream) !=
        cudaSuccess)
        return TSQR_ERR_CUDA;
    if (k == 0) {  // R alone
        if (qr_factor_launch(a, p.warps, p.smem, stream) != cudaSuccess) return TSQR_ERR_CUDA;
        g_last_launches = 1;
        return TSQR_SUCCESS;
    }
    if (cudaMemsetAsync(t.counters, 0, (size_t)groups * p.nodes * sizeof(unsigned int),
                        stream) != cudaSuccess ||
        qr_factor_launch(a, p.warps, p.smem, stream) != cudaSuccess ||
        (!fuse && wy_launch(wa, wy_smem, grid, stream) != cudaSuccess) ||
        qt_wy_launch(t, qtw_smem, stream) != cudaSuccess ||
        trsm_launch(R, ldr, t.C, n, X, ldx, (int)n, (int)k, ws->status, stream) != cudaSuccess)
        return TSQR_ERR_CUDA;
    g_last_launches = fuse ? 3 : 4;
    return TSQR_SUCCESS;
}

// Least squares: the factorization with its reflectors kept (as tsqr_qr's, with the tails in
// the workspace), then Q^T B's first n rows and R X = those rows: with the blocked apply, one
// launch over every column of B (run_lstsq_wy); otherwise per group of at most n columns of B,
// two launches.  With k <= max(1, n / 4) and n + k <= TSQR_MAX_N the augmented factorization
// above is used, and above TSQR_MAX_N columns the panels of run_lstsq_panels.
tsqr_status_t run_lstsq(const double *A, int64_t m, int64_t n, int64_t lda, const double *B,
                        int64_t ldb, int64_t k, double *X, int64_t ldx, double *R, int64_t ldr,
                        const tsqr_plan_t *over, cudaStream_t stream) {
    g_last_launches = 0;
    g_last_plan = tsqr_plan_t{};
    // the augmented factorization costs ~(n + k)^2 per row against n^2 plus the apply pass:
    // cheaper up to k ~ n / 4 (4,194,304 x 32: k = 1 11.3 against 15.2 ms, k = 32 49.0 against
    // 41.1 ms)
    if (k > 0 && k <= std::max<int64_t>(1, n / 4) && n + k <= TSQR_MAX_N)
        return run_lstsq_augmented(A, m, n, lda, B, ldb, k, X, ldx, R, ldr, over, stream);
    F64Plan p;
    tsqr_status_t st = plan_store(m, (int)n, over, &p);
    if (st != TSQR_SUCCESS) return st;
    g_last_plan = public_plan(p);
    if (p.unit % p.h != 0) return TSQR_ERR_UNSUPPORTED;  // chunk ids = first row / h
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return TSQR_ERR_CUDA;
    const DeviceInfo di = device_info(dev);
    const int kg = (int)std::min<int64_t>(k, n);  // columns of B per apply launch
    // the apply pass has no serial reflector chain: more, shorter warps (as the Q leaf pass)
    int qwarps = p.warps;
    for (int c : {12, 8})
        if (c > qwarps && p.hs % (32 * c) == 0) {
            qwarps = c;
            break;
        }
    int qblk = 1;
    for (int c = 4; c >= 1; --c)
        if ((p.hs / (32 * qwarps)) % c == 0) {
            qblk = c;
            break;
        }
    int ldX = 0, kw = 0;
    size_t wy_smem = 0, qtw_smem = 0;
    const bool wy = plan_wy((int)n, p, di, &ldX, &wy_smem, &kw, &qtw_smem);
    if (wy) return run_lstsq_wy(A, m, n, lda, B, ldb, k, X, ldx, R, ldr, p, ldX, wy_smem,
                                (int)std::max<int64_t>(1, std::min<int64_t>(k, kw)), qtw_smem,
                                di, stream);
    const size_t qt_smem = qt_smem_bytes((int)n, kg, p.ldS, qwarps);
    if (qt_smem > di.smem_block_optin) return TSQR_ERR_UNSUPPORTED;
    if (qr_prepare(p.smem, 0, 0) != cudaSuccess ||
        qt_prepare(qt_smem) != cudaSuccess)
        return TSQR_ERR_CUDA;
    const int64_t nchunks = (m + p.h - 1) / p.h;
    const size_t nn = (size_t)n * (size_t)n;
    const size_t cnt_bytes = align_up((size_t)p.nodes * sizeof(unsigned int), 256);
    const size_t slot_bytes = align_up((size_t)p.nodes * nn * sizeof(double), 256);
    const size_t v_bytes = align_up((size_t)m * (size_t)n * sizeof(double), 256);
    const size_t csc_bytes = align_up((size_t)nchunks * 2 * n * sizeof(double), 256);
    const size_t nv_bytes = align_up((size_t)p.nodes * (p.arity - 1) * nn * sizeof(double), 256);
    const size_t nsc_bytes = align_up((size_t)p.nodes * 2 * n * sizeof(double), 256);
    const size_t sgn_bytes = align_up((size_t)n * sizeof(double), 256);
    const size_t qslot_bytes = align_up((size_t)p.nodes * (size_t)n * kg * sizeof(double), 256);
    const size_t c_bytes = align_up((size_t)n * kg * sizeof(double), 256);
    const size_t r_bytes = R ? 0 : nn * sizeof(double);
    Workspace *ws = nullptr;
    st = get_workspace(stream, 2 * cnt_bytes + slot_bytes + v_bytes + csc_bytes + nv_bytes +
                                   nsc_bytes + sgn_bytes + qslot_bytes + c_bytes + r_bytes, &ws);
    if (st != TSQR_SUCCESS) return st;
    char *base = (char *)ws->base;
    size_t o = 0;
    unsigned int *counters = (unsigned int *)(base + o);
    o += cnt_bytes;
    double *slots = (double *)(base + o);
    o += slot_bytes;
    double *V = (double *)(base + o);
    o += v_bytes;
    double *csc = (double *)(base + o);
    o += csc_bytes;
    double *nV = (double *)(base + o);
    o += nv_bytes;
    double *nsc = (double *)(base + o);
    o += nsc_bytes;
    double *signs = (double *)(base + o);
    o += sgn_bytes;
    unsigned int *qcounters = (unsigned int *)(base + o);
    o += cnt_bytes;
    double *qslots = (double *)(base + o);
    o += qslot_bytes;
    double *C = (double *)(base + o);
    o += c_bytes;
    if (!R) {
        R = (double *)(base + o);
        ldr = n;
    }
    F64Args a = plan_args(p, A, m, n, lda);
    a.counters = counters;
    a.slots = slots;
    a.R = R;
    a.ldr = ldr;
    a.status = ws->status;
    a.q.V = V;
    a.q.ldv = m;
    a.q.chunk_sc = csc;
    a.q.node_V = nV;
    a.q.node_sc = nsc;
    a.q.signs = signs;
    if (cudaMemsetAsync(counters, 0, (size_t)p.nodes * sizeof(unsigned int), stream) !=
            cudaSuccess ||
        qr_factor_launch(a, p.warps, p.smem, stream) != cudaSuccess)
        return TSQR_ERR_CUDA;
    int launches = 1;
    for (int64_t q0 = 0; q0 < k; q0 += kg) {
        const int kc = (int)std::min<int64_t>(kg, k - q0);
        QtArgs t = qt_args(p, a.q, m, (int)n, B + q0 * ldb, ldb, kc, kc);
        t.slots = qslots;
        t.counters = qcounters;
        t.C = C;
        t.ldc = n;
        if (cudaMemsetAsync(qcounters, 0, (size_t)p.nodes * sizeof(unsigned int), stream) !=
                cudaSuccess ||
            qt_launch(t, qblk, qwarps, qt_smem, stream) != cudaSuccess ||
            trsm_launch(R, ldr, C, n, X + q0 * ldx, ldx, (int)n, kc, ws->status, stream) !=
                cudaSuccess)
            return TSQR_ERR_CUDA;
        launches += 2;
    }
    g_last_launches = launches;
    return TSQR_SUCCESS;
}

// Communication-avoiding QR of a general m x N matrix (Section 5): panels of nb columns, each
// factorized by the TSQR factorization with its reflectors kept, then Q^T applied to the
// columns right of it.  The rows that update leaves behind form the next panel's matrix: every
// row of the old one (its chunks' rows of Q^T B, in place) and the n-row blocks its tree nodes
// left behind (appended below), so a panel on L leaves adds (L - 1) nb rows.
constexpr int64_t kCaqrPanel = 16;  // the default panel width (measured: 16 >= 24, 32, 48)

struct CaqrPanel {
    F64Plan p;
    int64_t j0, M;  // first column, rows of the panel's matrix
    int w, kc;      // panel width, trailing columns per update CTA (kc <= w)
    int qwarps, qblk;
    size_t qt_smem;
    bool wy;        // the update applies each chunk's reflectors as one compact WY block
    size_t wy_smem;
    int ldX;
};


tsqr_status_t run_caqr(const double *A, int64_t m, int64_t N, int64_t lda, double *R,
                       int64_t ldr, int64_t nb, const tsqr_plan_t *over, cudaStream_t stream) {
    g_last_launches = 0;
    g_last_plan = tsqr_plan_t{};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return TSQR_ERR_CUDA;
    const DeviceInfo di = device_info(dev);
    std::vector<CaqrPanel> panels;
    int64_t M = m;
    size_t max_fsmem = 0, max_qt = 0;
    size_t cnt_max = 0, slot_max = 0, v_max = 0, csc_max = 0, nv_max = 0, nsc_max = 0;
    size_t qcnt_max = 0, qslot_max = 0, wys_max = 0;
    for (int64_t j0 = 0; j0 < N; j0 += nb) {
        CaqrPanel c;
        c.j0 = j0;
        c.M = M;
        c.w = (int)std::min<int64_t>(nb, N - j0);
        tsqr_status_t st = plan_store(M, c.w, over, &c.p);
        if (st != TSQR_SUCCESS) return st;
        const int64_t trail = N - j0 - c.w;
        if (plan_is_auto(over) && trail > 0) {
            // Fewer leaves than the AUTO plan's: the panel's factorization runs on fewer CTAs
            // (its time ~ 2 M w^2 (2 SMs) / (L P) at a GPU rate P), but every later panel's
            // matrix has (L - 1) w rows more (their cost ~ w sum_{q > p} 4 w trail_q / P ~
            // 2 w trail^2 / P per leaf).  The two balance at L = sqrt(2 SMs M w) / trail.
            const double best = std::sqrt(2.0 * di.sms * (double)M * c.w) / (double)trail;
            const int leaves = (int)std::max(1.0, std::ceil(best));
            if (leaves < c.p.nleaves) {
                tsqr_plan_t o;
                std::memset(&o, 0, sizeof(o));
                o.tree = TSQR_TREE_HYBRID;
                o.ctas = leaves;
                o.warps = c.p.warps;
                st = plan_f64(M, c.w, &o, &c.p);
                if (st != TSQR_SUCCESS) return st;
            }
        }
        if (c.p.unit % c.p.h != 0) return TSQR_ERR_UNSUPPORTED;  // chunk ids = first row / h
        c.qwarps = c.p.warps;
        for (int w : {12, 8})
            if (w > c.qwarps && c.p.hs % (32 * w) == 0) {
                c.qwarps = w;
                break;
            }
        c.qblk = 1;
        for (int b = 4; b >= 1; --b)
            if ((c.p.hs / (32 * c.qwarps)) % b == 0) {
                c.qblk = b;
                break;
            }
        c.wy = plan_wy(c.w, c.p, di, &c.ldX, &c.wy_smem, &c.kc, &c.qt_smem);
        if (plan_is_auto(over) && trail > 0 && c.wy) {
            // The update's grid is L x G CTAs of equal work (G column groups), whole waves of
            // SMs x (CTAs per SM) at a time: a leaf count within 15% of L that fills the last
            // wave better wins (262,144 x 512: 2,288 CTAs in 15.05 waves of 152 left the
            // sixteenth wave almost empty).
            const int64_t G = (trail + c.kc - 1) / c.kc;
            const int64_t slots =
                (int64_t)di.sms * std::max<int64_t>(1, (int64_t)(di.smem_sm / (c.qt_smem + 1024)));
            const int L = c.p.nleaves;
            auto eff = [&](int64_t l) {
                const int64_t ctas = l * G;
                return (double)ctas / (double)(((ctas + slots - 1) / slots) * slots);
            };
            int bestL = L;
            const int lo = std::max(1, (int)(0.85 * L)), hi = (int)std::min<int64_t>(
                                                             c.p.nunits, (int64_t)(1.15 * L) + 1);
            for (int l = lo; l <= hi; ++l)
                if (eff(l) > eff(bestL) + 1e-9 ||
                    (eff(l) > eff(bestL) - 1e-9 && std::abs(l - L) < std::abs(bestL - L)))
                    bestL = l;
            if (bestL != L) {
                tsqr_plan_t o;
                std::memset(&o, 0, sizeof(o));
                o.tree = TSQR_TREE_HYBRID;
                o.ctas = bestL;
                o.warps = c.p.warps;
                st = plan_f64(M, c.w, &o, &c.p);
                if (st != TSQR_SUCCESS) return st;
                if (c.p.unit % c.p.h != 0) return TSQR_ERR_UNSUPPORTED;
                c.wy = plan_wy(c.w, c.p, di, &c.ldX, &c.wy_smem, &c.kc, &c.qt_smem);
            }
        }
        if (!c.wy) {
            // the reflector-by-reflector update; its columns are independent too: as many per
            // CTA as fit beside the chunk
            c.kc = c.w;
            while (c.kc > 8 && qt_smem_bytes(c.w, c.kc, c.p.ldS, c.qwarps) > di.smem_block_optin)
                c.kc = (c.kc + 1) / 2;
            c.qt_smem = qt_smem_bytes(c.w, c.kc, c.p.ldS, c.qwarps);
        }
        if (c.qt_smem > di.smem_block_optin) return TSQR_ERR_UNSUPPORTED;
        const size_t ww = (size_t)c.w * c.w, nodes = (size_t)c.p.nodes;
        const size_t groups = trail > 0 ? (size_t)((trail + c.kc - 1) / c.kc) : 0;
        if (groups > 65535) return TSQR_ERR_UNSUPPORTED;  // one grid row per column group
        max_fsmem = std::max(max_fsmem, c.p.smem);
        max_qt = std::max(max_qt, c.qt_smem);
        cnt_max = std::max(cnt_max, nodes * sizeof(unsigned int));
        slot_max = std::max(slot_max, nodes * ww * sizeof(double));
        v_max = std::max(v_max, (size_t)M * c.w * sizeof(double));
        csc_max = std::max(csc_max, (size_t)((M + c.p.h - 1) / c.p.h) * 2 * c.w * sizeof(double));
        nv_max = std::max(nv_max, nodes * (c.p.arity - 1) * ww * sizeof(double));
        nsc_max = std::max(nsc_max, nodes * 2 * c.w * sizeof(double));
        if (c.wy) wys_max = std::max(wys_max, (size_t)((M + c.p.h - 1) / c.p.h) * ww * sizeof(double));
        qcnt_max = std::max(qcnt_max, groups * nodes * sizeof(unsigned int));
        qslot_max = std::max(qslot_max, groups * nodes * c.w * c.kc * sizeof(double));
        if (panels.empty()) g_last_plan = public_plan(c.p);
        panels.push_back(c);
        M += (int64_t)(c.p.nleaves - 1) * c.w;
    }
    const int64_t w0 = panels[0].w;
    const int64_t ldC = (M + 3) / 4 * 4;  // the last panel's rows, rounded to 32 bytes
    const size_t c_bytes = (size_t)ldC * (size_t)(N - w0) * sizeof(double);
    if (qr_prepare(max_fsmem, 0, 0) != cudaSuccess || qt_prepare(max_qt) != cudaSuccess)
        return TSQR_ERR_CUDA;
    const size_t sizes[] = {cnt_max, slot_max,  v_max,    csc_max, nv_max,  nsc_max,
                            (size_t)nb * sizeof(double), qcnt_max, qslot_max, c_bytes, wys_max};
    constexpr int kBufs = sizeof(sizes) / sizeof(sizes[0]);
    size_t total = 0;
    for (size_t b : sizes) total += align_up(b, 256);
    Workspace *ws = nullptr;
    tsqr_status_t st = get_workspace(stream, total, &ws);
    if (st != TSQR_SUCCESS) return st;
    char *base = (char *)ws->base;
    void *bufs[kBufs];
    size_t o = 0;
    for (int i = 0; i < kBufs; ++i) {
        bufs[i] = base + o;
        o += align_up(sizes[i], 256);
    }
    unsigned int *counters = (unsigned int *)bufs[0];
    double *slots = (double *)bufs[1], *V = (double *)bufs[2], *csc = (double *)bufs[3];
    double *nV = (double *)bufs[4], *nsc = (double *)bufs[5], *signs = (double *)bufs[6];
    unsigned int *qcounters = (unsigned int *)bufs[7];
    double *qslots = (double *)bufs[8], *C = (double *)bufs[9], *wyS = (double *)bufs[10];
    // R's rows below each diagonal block stay zero; the kernels write the rest
    if (cudaMemset2DAsync(R, (size_t)ldr * sizeof(double), 0, (size_t)N * sizeof(double),
                          (size_t)N, stream) != cudaSuccess)
        return TSQR_ERR_CUDA;
    int launches = 0;
    for (size_t pi = 0; pi < panels.size(); ++pi) {
        const CaqrPanel &c = panels[pi];
        // the panel's matrix: A itself for the first panel, then C (column j of the matrix is
        // column j - w0 of C)
        const double *src = pi == 0 ? A : C + (c.j0 - w0) * ldC;
        const int64_t lds = pi == 0 ? lda : ldC;
        F64Args a = plan_args(c.p, src, c.M, c.w, lds);
        a.counters = counters;
        a.slots = slots;
        a.R = R + c.j0 + c.j0 * ldr;
        a.ldr = ldr;
        a.status = ws->status;
        a.q.V = V;
        a.q.ldv = c.M;
        a.q.chunk_sc = csc;
        a.q.node_V = nV;
        a.q.node_sc = nsc;
        a.q.signs = signs;
        if (cudaMemsetAsync(counters, 0, (size_t)c.p.nodes * sizeof(unsigned int), stream) !=
                cudaSuccess ||
            qr_factor_launch(a, c.p.warps, c.p.smem, stream) != cudaSuccess)
            return TSQR_ERR_CUDA;
        ++launches;
        const int64_t trail = N - c.j0 - c.w;
        if (trail == 0) break;
        QtArgs t = qt_args(c.p, a.q, c.M, c.w, src + c.w * lds, lds, c.kc, (int)trail);
        t.slots = qslots;
        t.counters = qcounters;
        t.C = R + c.j0 + (c.j0 + c.w) * ldr;
        t.ldc = ldr;
        t.Cout = C + (c.j0 + c.w - w0) * ldC;
        t.ldco = ldC;
        t.grow0 = c.M;
        const size_t groups = (size_t)((trail + c.kc - 1) / c.kc);
        if (cudaMemsetAsync(qcounters, 0, groups * (size_t)c.p.nodes * sizeof(unsigned int),
                            stream) != cudaSuccess)
            return TSQR_ERR_CUDA;
        if (c.wy) {
            const WyArgs wa = wy_args(c.p, a.q, c.M, c.w, c.ldX, wyS);
            t.wyS = wyS;
            const int grid = (int)std::min<int64_t>(wa.nchunks, 4LL * di.sms);
            if (wy_launch(wa, c.wy_smem, grid, stream) != cudaSuccess ||
                qt_wy_launch(t, c.qt_smem, stream) != cudaSuccess)
                return TSQR_ERR_CUDA;
            launches += 2;
        } else {
            if (qt_launch(t, c.qblk, c.qwarps, c.qt_smem, stream) != cudaSuccess)
                return TSQR_ERR_CUDA;
            ++launches;
        }
    }
    g_last_launches = launches;
    return TSQR_SUCCESS;
}

// Least squares above TSQR_MAX_N columns: [A | B] (copied to a buffer of this call) by panels,
// as tsqr_caqr_r; its R holds R and (Q^T B)(0:n, :) side by side (the sign convention negates
// whole rows, which keeps R X = C), then R X = C.  The copy and the augmented R are allocated
// stream-ordered for the call, since the panels take the stream's pooled workspace themselves.
tsqr_status_t run_lstsq_panels(const double *A, int64_t m, int64_t n, int64_t lda,
                               const double *B, int64_t ldb, int64_t k, double *X, int64_t ldx,
                               double *R, int64_t ldr, cudaStream_t stream) {
    const int64_t na = n + k;
    double *aug = nullptr, *Ra = nullptr;
    if (cudaMallocAsync((void **)&aug, (size_t)m * na * sizeof(double), stream) != cudaSuccess)
        return TSQR_ERR_ALLOC;
    if (cudaMallocAsync((void **)&Ra, (size_t)na * na * sizeof(double), stream) != cudaSuccess) {
        cudaFreeAsync(aug, stream);
        return TSQR_ERR_ALLOC;
    }
    tsqr_status_t st = TSQR_SUCCESS;
    if (cudaMemcpy2DAsync(aug, (size_t)m * sizeof(double), A, (size_t)lda * sizeof(double),
                          (size_t)m * sizeof(double), (size_t)n, cudaMemcpyDeviceToDevice,
                          stream) != cudaSuccess ||
        (k > 0 && cudaMemcpy2DAsync(aug + n * m, (size_t)m * sizeof(double), B,
                                    (size_t)ldb * sizeof(double), (size_t)m * sizeof(double),
                                    (size_t)k, cudaMemcpyDeviceToDevice, stream) != cudaSuccess))
        st = TSQR_ERR_CUDA;
    int launches = 0;
    if (st == TSQR_SUCCESS) {
        st = run_caqr(aug, m, na, m, Ra, na, kCaqrPanel, nullptr, stream);
        launches = g_last_launches;
    }
    Workspace *ws = nullptr;
    if (st == TSQR_SUCCESS) st = get_workspace(stream, 0, &ws);
    if (st == TSQR_SUCCESS &&
        ((R && cudaMemcpy2DAsync(R, (size_t)ldr * sizeof(double), Ra, (size_t)na * sizeof(double),
                                 (size_t)n * sizeof(double), (size_t)n, cudaMemcpyDeviceToDevice,
                                 stream) != cudaSuccess) ||
         (k > 0 && trsm_launch(Ra, na, Ra + n * na, na, X, ldx, (int)n, (int)k, ws->status,
                               stream) != cudaSuccess)))
        st = TSQR_ERR_CUDA;
    cudaFreeAsync(aug, stream);
    cudaFreeAsync(Ra, stream);
    g_last_launches = st == TSQR_SUCCESS ? launches + (k > 0 ? 1 : 0) : 0;
    return st;
}

// Plan of the blocked mixed leaf (TSQR_LEAF_PANELS): chunks of h rows, one of kMixedWyHeights
// (AUTO: the tallest that the width's shared and tensor memory hold), work units of one chunk
// (HYBRID, FLAT) or one tile (BINARY), the largest tree arity whose stacked FP64 triangles fit
// the chunk region.
tsqr_status_t plan_mixed_wy(int64_t m, int n, const tsqr_plan_t *over, F64Plan *p) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return TSQR_ERR_CUDA;
    const DeviceInfo di = device_info(dev);
    if (di.sms <= 0) return TSQR_ERR_CUDA;
    if (n < 1 || n > kMixedWyMaxN) return TSQR_ERR_UNSUPPORTED;
    p->leaf = TSQR_LEAF_PANELS;
    p->tree = (over && over->tree) ? over->tree : TSQR_TREE_HYBRID;
    if (p->tree < TSQR_TREE_BINARY || p->tree > TSQR_TREE_HYBRID) return TSQR_ERR_INVALID_ARG;
    if (over && (over->warps != 0 && over->warps != 8)) return TSQR_ERR_INVALID_ARG;
    if (over && (over->tile_rows < 0 || over->ctas < 0 || over->arity < 0))
        return TSQR_ERR_INVALID_ARG;
    p->warps = 8;
    const int64_t mm = std::max<int64_t>(m, 1);
    const size_t reserve = 1024;
    // AUTO chunk height: the tallest of 1024, 768, 640, 512 rows that fits one CTA's shared
    // memory and the SM's tensor memory (fewer reflector chains per row of A: 2^24 x 64 FP32
    // with 512-row chunks 24.3 ms, with 256-row chunks (two CTAs per SM) 49 ms)
    auto fits = [&](int hh) {
        return mixed_wy_smem_bytes(n, hh) + reserve <= di.smem_block_optin && mixed_wy_tmem_fits(n, hh);
    };
    int h_auto = 256;
    for (int hh : kMixedWyHeights)
        if (fits(hh)) {
            h_auto = hh;
            break;
        }
    int h;
    if (p->tree == TSQR_TREE_BINARY) {
        p->unit = (over && over->tile_rows > 0) ? over->tile_rows : 256;
        h = 256;
        for (int hh : kMixedWyHeights)
            if (hh <= h_auto && p->unit % hh == 0) {
                h = hh;
                break;
            }
    } else if (over && over->tile_rows > 0) {
        bool known = false;
        for (int hh : kMixedWyHeights) known |= (over->tile_rows == hh);
        if (!known || !fits(over->tile_rows)) return TSQR_ERR_INVALID_ARG;
        h = over->tile_rows;
        p->unit = h;
    } else {
        h = h_auto;
        p->unit = h;
    }
    p->h = h;
    p->hs = h;
    p->ldS = 0;
    p->blk = h / 128;
    (void)reserve;
    p->vec = 1;
    p->smem = mixed_wy_smem_bytes(n, h);
    if (p->smem > di.smem_block_optin) return TSQR_ERR_UNSUPPORTED;
    p->nunits = (mm + p->unit - 1) / p->unit;
    int64_t leaves;
    if (p->tree == TSQR_TREE_FLAT) {
        leaves = 1;
    } else if (p->tree == TSQR_TREE_BINARY) {
        leaves = p->nunits;
    } else if (over && over->ctas > 0) {
        leaves = over->ctas;
    } else {
        if (mixed_wy_prepare(p->smem) != cudaSuccess) return TSQR_ERR_CUDA;
        leaves = (int64_t)di.sms * std::max(1, mixed_wy_blocks_per_sm(h, p->smem));
    }
    leaves = std::min<int64_t>(leaves, p->nunits);
    if (leaves < 1 || leaves > 0x7fffffffLL) return TSQR_ERR_UNSUPPORTED;
    p->nleaves = (int)leaves;
    if (p->tree == TSQR_TREE_BINARY) {
        p->arity = 2;
    } else if (over && over->arity > 0) {
        if (over->arity < 2 || over->arity > 8) return TSQR_ERR_INVALID_ARG;
        p->arity = over->arity;
    } else {
        p->arity = mixed_wy_arity(n, h);
    }
    if (!mixed_wy_tree_fits(n, h, p->arity)) return TSQR_ERR_UNSUPPORTED;
    p->ldSd = tree_ldsd(n, p->arity);
    p->s_doubles = 0;
    return build_tree(leaves, p->arity, &p->shape, &p->nodes);
}

// The mixed path's plan: the tuned plan of the bucket for AUTO calls, then the blocked leaf
// where it applies (TSQR_LEAF_PANELS requested, or AUTO where it measured faster, see wy_auto
// below; up to kMixedWyMaxN columns), else the fold.
tsqr_status_t plan_mixed(int64_t m, int n, bool bf16, const tsqr_plan_t *over, F64Plan *p) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return TSQR_ERR_CUDA;
    tsqr_plan_t tuned;
    if (plan_is_auto(over) && tuned_plan(dev, m, n, true, &tuned)) over = &tuned;
    const int leaf = over ? over->leaf : 0;
    // AUTO leaf: the panels where they apply and the plan's knobs are theirs (8 or 0 warps;
    // chunks of 256 or 512 rows unless the tree is BINARY); else the fold
    const bool wy_knobs =
        !over || ((over->warps == 0 || over->warps == 8) &&
                  (over->tree == TSQR_TREE_BINARY || over->tile_rows == 0 ||
                   over->tile_rows == 256 || over->tile_rows == 512));
    // measured at 2^24 rows: the fold wins up to n = 8 for FP32 (n = 8: 0.80 against 0.82 ms;
    // n = 9: 1.31 against 0.90; n = 7 alone goes the other way, 0.85 against 0.75) and at
    // n <= 2 for BF16 (n = 2: 0.34 against 0.44 ms; n = 3: 0.84 against 0.53), the blocked leaf
    // from there to 112 columns (FP32, fold against panels: n = 65: 48.8 against 25.7 ms;
    // n = 96: 143.8 against 45.2; n = 112: 226.8 against 73.2; BF16 alike)
    const bool wy_auto = n <= kMixedWyMaxN && n > (bf16 ? 2 : 8);
    if (leaf == TSQR_LEAF_PANELS || (leaf == 0 && wy_auto && wy_knobs)) {
        tsqr_plan_t o = over ? *over : tsqr_plan_t{};
        o.leaf = TSQR_LEAF_PANELS;
        return plan_mixed_wy(m, n, &o, p);
    }
    if (leaf != 0 && leaf != TSQR_LEAF_FOLD) return TSQR_ERR_INVALID_ARG;
    tsqr_plan_t o = over ? *over : tsqr_plan_t{};
    o.leaf = 0;
    return plan_leaf(m, n, plan_is_auto(&o) ? nullptr : &o, true, p);
}

tsqr_status_t run_mixed(const void *A, bool bf16, int64_t m, int64_t n, int64_t lda, double *R,
                        int64_t ldr, const tsqr_plan_t *over, cudaStream_t stream) {
    g_last_launches = 0;
    g_last_plan = tsqr_plan_t{};
    if (n == 0) return TSQR_SUCCESS;
    if (m == 0) return zero_r(R, n, ldr, stream);
    F64Plan p;
    tsqr_status_t st = plan_mixed(m, (int)n, bf16, over, &p);
    if (st != TSQR_SUCCESS) return st;
    const bool wy = p.leaf == TSQR_LEAF_PANELS;
    if ((wy ? mixed_wy_prepare(p.smem) : mixed_prepare(p.smem)) != cudaSuccess)
        return TSQR_ERR_CUDA;
    const size_t cnt_bytes = align_up((size_t)p.nodes * sizeof(unsigned int), 256);
    const size_t slot_bytes = (size_t)p.nodes * (size_t)n * (size_t)n * sizeof(double);
    Workspace *ws = nullptr;
    st = get_workspace(stream, cnt_bytes + slot_bytes, &ws);
    if (st != TSQR_SUCCESS) return st;
    F64Args base = plan_args(p, nullptr, m, n, lda);
    base.counters = (unsigned int *)ws->base;
    base.slots = (double *)((char *)ws->base + cnt_bytes);
    base.R = R;
    base.ldr = ldr;
    base.status = ws->status;
    if (cudaMemsetAsync(base.counters, 0, (size_t)p.nodes * sizeof(unsigned int), stream) !=
        cudaSuccess)
        return TSQR_ERR_CUDA;
    if (wy) {
        if (mixed_wy_launch(base, A, bf16, p.ldSd, p.smem, stream) != cudaSuccess)
            return TSQR_ERR_CUDA;
    } else {
        MixedArgs a;
        std::memset(&a, 0, sizeof(a));
        a.base = base;
        a.A = A;
        a.ldSd = p.ldSd;
        a.s_doubles = p.s_doubles;
        if (mixed_launch(a, bf16, p.warps, p.smem, stream) != cudaSuccess) return TSQR_ERR_CUDA;
    }
    g_last_plan = public_plan(p);
    g_last_launches = 1;
    return TSQR_SUCCESS;
}

// ------------------------------------------------------------------------------------------
// Varlen batch.  One CTA size and shared-memory budget for the whole batch (set by its widest
// problem); per width n the tallest chunk that fits; per problem leaves of a few chunks sized
// so that the batch has several leaves per CTA; work items (problem, leaf) ordered by work,
// largest first, for the persistent kernel's queue.
// ------------------------------------------------------------------------------------------
// Width bucket of a batched problem: n <= 8, <= 16, <= 32, > 32.
int width_bucket(int n) { return n <= 8 ? 0 : n <= 16 ? 1 : n <= 32 ? 2 : 3; }

// Batch plans chosen by tsqr_autotune_batched, per batch shape bucket: device, input type,
// the width buckets present, floor(log2 count) and floor(log2 of the work sum max(m, 1) n^2).
struct BatchKey {
    int dev, dt, widths, clog, wlog;
    bool operator<(const BatchKey &o) const {
        if (dev != o.dev) return dev < o.dev;
        if (dt != o.dt) return dt < o.dt;
        if (widths != o.widths) return widths < o.widths;
        if (clog != o.clog) return clog < o.clog;
        return wlog < o.wlog;
    }
};
std::map<BatchKey, tsqr_batch_plan_t> g_batch_tuned;  // guarded by g_tune_mu

BatchKey batch_key(int dev, int dt, const int64_t *ms, const int32_t *ns, int32_t count) {
    int widths = 0;
    double work = 0.0;
    for (int32_t i = 0; i < count; ++i) {
        widths |= 1 << width_bucket(ns[i]);
        work += (double)std::max<int64_t>(ms[i], 1) * ns[i] * ns[i];
    }
    int wlog = 0;
    while (wlog < 120 && std::ldexp(1.0, wlog + 1) <= work) ++wlog;
    return BatchKey{dev, dt, widths, floor_log2(std::max(count, 1)), wlog};
}

bool batch_plan_is_auto(const tsqr_batch_plan_t *p) {
    return !p || (p->warps == 0 && p->ctas_per_sm == 0 && p->leaves_per_cta == 0 &&
                  p->arity[0] == 0 && p->arity[1] == 0 && p->arity[2] == 0 && p->arity[3] == 0 &&
                  p->leaf == 0);
}

tsqr_status_t run_batched(const void *const *ptrs, const int64_t *ms, const int32_t *ns,
                          const int64_t *offsets, int32_t count, double *R_packed, int dt,
                          const tsqr_batch_plan_t *bp_in, cudaStream_t stream) {
    g_last_launches = 0;
    g_last_plan = tsqr_plan_t{};
    g_last_batch_plan = tsqr_batch_plan_t{};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return TSQR_ERR_CUDA;
    const DeviceInfo di = device_info(dev);
    if (di.sms <= 0) return TSQR_ERR_CUDA;
    tsqr_batch_plan_t bp{};
    if (!batch_plan_is_auto(bp_in)) {
        bp = *bp_in;
    } else {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_batch_tuned.find(batch_key(dev, dt, ms, ns, count));
        if (it != g_batch_tuned.end()) bp = it->second;
    }
    if (bp.warps < 0 || bp.warps > 12 ||
        bp.ctas_per_sm < 0 || bp.ctas_per_sm > 2 || bp.leaves_per_cta < 0 ||
        bp.leaves_per_cta > 64)
        return TSQR_ERR_INVALID_ARG;
    for (int b = 0; b < 4; ++b)
        if (bp.arity[b] != 0 && (bp.arity[b] < 2 || bp.arity[b] > 8)) return TSQR_ERR_INVALID_ARG;
    if (bp.leaf != 0 && bp.leaf != TSQR_LEAF_FOLD && bp.leaf != TSQR_LEAF_PANELS)
        return TSQR_ERR_INVALID_ARG;
    const bool mixed = dt != 0;
    int nmax = 1;
    for (int32_t i = 0; i < count; ++i) nmax = std::max(nmax, (int)ns[i]);
    if (bp.leaf == TSQR_LEAF_PANELS && (!mixed || nmax > kMixedWyMaxN)) return TSQR_ERR_UNSUPPORTED;
    // mixed batches up to 112 columns take the blocked leaf unless the plan says fold
    // (4096-problem varlen batch, FP32: 181 ms with the fold and its tuned knobs against 81)
    const bool wy = mixed && nmax <= kMixedWyMaxN && bp.leaf != TSQR_LEAF_FOLD;
    int wy_h = 0, wy_tcols = 0;
    if (wy) {
        for (int hh : kMixedWyHeights)
            if (mixed_wy_smem_bytes(nmax, hh) <= di.smem_block_optin && mixed_wy_tmem_fits(nmax, hh)) {
                wy_h = hh;
                break;
            }
        if (!wy_h) return TSQR_ERR_UNSUPPORTED;
        wy_tcols = batched_wy_tmem_cols(nmax, wy_h);
    }
    const size_t reserve = 1024 + 256;  // per-CTA reserve plus the kernel's static shared memory
    const size_t two_per_sm = (di.smem_sm > 2 * reserve) ? (di.smem_sm - 2 * reserve) / 2 : 0;
    const size_t one_per_sm = std::min(di.smem_block_optin - 256, di.smem_sm - reserve);
    // bulk warps (AUTO): 4, or 12 for a batch with widths from 48 on whose widest chunk fits
    // with 12 warps: it runs one CTA per SM and hides the wide problems' reflector chains
    // behind more warps (the varlen batch of 4096 problems with widths up to 64: FP64 716 ms
    // with 4, 640 with 8, 626 with 12; mixed FP32 304 ms with 4, 224 with 12)
    const int W = wy ? 8
                     : bp.warps ? bp.warps
                     : (nmax >= 48 && max_rows_per_lane_p(nmax, 12, one_per_sm, mixed) >= 1) ? 12
                                                                                            : 4;
    // CTAs per SM (AUTO): two when the widest problem's chunk fits at two rows per lane (one
    // CTA per SM with taller chunks measured faster on the varlen batch otherwise: 717
    // against 1010 ms for FP64 with widths up to 64)
    size_t budget = two_per_sm;
    if (bp.ctas_per_sm == 1 ||
        (bp.ctas_per_sm == 0 && good_r(max_rows_per_lane_p(nmax, W, two_per_sm, mixed)) < 2))
        budget = one_per_sm;
    // per width: chunk rows
    std::vector<int> hs_of(TSQR_MAX_N + 1, 0), blk_of(TSQR_MAX_N + 1, 1), vec_of(TSQR_MAX_N + 1, 1);
    size_t smem = 0;
    for (int32_t i = 0; i < count && wy; ++i) {
        const int n = ns[i];
        if (hs_of[n]) continue;
        hs_of[n] = wy_h;
        smem = std::max(smem, mixed_wy_smem_bytes(n, wy_h));
    }
    // the blocked leaf's CTAs hold their tensor memory for the whole launch: one CTA per SM
    // (more than half an SM's shared memory), so that no CTA's allocation waits for another's
    if (wy) smem = std::max(smem, di.smem_sm / 2 + 1024);
    for (int32_t i = 0; i < count && !wy; ++i) {
        const int n = ns[i];
        if (hs_of[n]) continue;
        int r = good_r(max_rows_per_lane_p(n, W, budget, mixed));
        // the batched mixed kernels are instantiated for blocks (4,4), (2,2) and (1,1)
        if (mixed && r >= 4) r -= r % 4;
        if (r < 1 || 32 * W * r < n) return TSQR_ERR_UNSUPPORTED;
        hs_of[n] = 32 * W * r;
        block_for(r, mixed, &blk_of[n], &vec_of[n]);
        if (mixed && blk_of[n] * 10 + vec_of[n] != 44 && blk_of[n] * 10 + vec_of[n] != 22) {
            blk_of[n] = (r % 4 == 0) ? 4 : (r % 2 == 0) ? 2 : 1;
            vec_of[n] = blk_of[n];
        }
        smem = std::max(smem, leaf_smem_bytes(n, hs_of[n], ld_for(hs_of[n], vec_of[n]), W,
                                              mixed));
    }
    const int kdt = (W > 7) ? dt + 3 : dt;  // the kernels for up to 12 bulk warps
    if ((wy ? batched_wy_prepare(dt == 2, wy_h, smem) : batched_prepare(kdt, smem)) != cudaSuccess)
        return TSQR_ERR_CUDA;
    const int per_sm = std::max(1, wy ? batched_wy_blocks_per_sm(dt == 2, wy_h, smem)
                                      : batched_blocks_per_sm(kdt, W, smem));
    const int64_t ctas = (int64_t)di.sms * per_sm;
    // leaf size: about 6 leaves per CTA over the whole batch (AUTO)
    const int lpc = bp.leaves_per_cta ? bp.leaves_per_cta : 6;
    double work = 0.0;
    for (int32_t i = 0; i < count; ++i) work += (double)std::max<int64_t>(ms[i], 1) * ns[i] * ns[i];
    const double target = work / (double)(ctas * lpc);

    std::vector<BatchProblem> probs(count);
    std::vector<std::pair<double, int2>> items;
    int64_t slot_doubles = 0, nodes_total = 0;
    for (int32_t i = 0; i < count; ++i) {
        const int n = ns[i];
        const int64_t m = std::max<int64_t>(ms[i], 1);
        BatchProblem &P = probs[i];
        P.A = ptrs[i];
        P.m = ms[i];
        P.lda = std::max<int64_t>(ms[i], 1);
        P.R = R_packed + offsets[i];
        P.n = n;
        P.hs = hs_of[n];
        P.blk = blk_of[n];
        P.vec = vec_of[n];
        P.ldS = ld_for(P.hs, P.vec);
        const int64_t chunks = std::max<int64_t>(1, (int64_t)(target / ((double)n * n * P.hs)));
        P.unit = chunks * P.hs;
        P.h = P.hs;
        P.nunits = (m + P.unit - 1) / P.unit;
        if (P.nunits > (1 << 24)) return TSQR_ERR_UNSUPPORTED;
        P.nleaves = (int)P.nunits;
        // arity: the largest that the width's shared memory holds, or the plan's, lowered to fit
        const int amax = wy ? mixed_wy_arity(n, wy_h)
                            : arity_for(n, mixed ? mixed_s_doubles(n, P.ldS) : P.ldS * n);
        const int areq = bp.arity[width_bucket(n)];
        P.arity = areq ? std::min(areq, amax) : amax;
        if (wy)
            while (P.arity > 2 && !mixed_wy_tree_fits(n, wy_h, P.arity)) --P.arity;
        else if (!mixed)
            while (P.arity > 2 && tree_ldsd(n, P.arity) > P.ldS) --P.arity;
        TreeShape shape;
        int64_t nodes = 0;
        if (build_tree(P.nleaves, P.arity, &shape, &nodes) != TSQR_SUCCESS) return TSQR_ERR_UNSUPPORTED;
        P.slot_off = slot_doubles;
        P.cnt_off = nodes_total;
        slot_doubles += nodes * (int64_t)n * n;
        nodes_total += nodes;
        for (int l = 0; l < P.nleaves; ++l) {
            const int64_t rows = std::min<int64_t>(P.unit, m - (int64_t)l * P.unit);
            items.push_back({(double)rows * n * n, make_int2(i, l)});
        }
    }
    std::stable_sort(items.begin(), items.end(),
                     [](const std::pair<double, int2> &a, const std::pair<double, int2> &b) {
                         return a.first > b.first;
                     });
    if (items.size() > (size_t)0x7fffffff) return TSQR_ERR_UNSUPPORTED;
    // table: problems then items, copied once and reused while the batch is unchanged
    std::vector<char> table(sizeof(BatchProblem) * probs.size() + sizeof(int2) * items.size());
    std::memcpy(table.data(), probs.data(), sizeof(BatchProblem) * probs.size());
    int2 *it_host = reinterpret_cast<int2 *>(table.data() + sizeof(BatchProblem) * probs.size());
    for (size_t k = 0; k < items.size(); ++k) it_host[k] = items[k].second;

    const size_t head_bytes = align_up((size_t)(1 + nodes_total) * sizeof(unsigned int), 256);
    const size_t slots_bytes = align_up((size_t)slot_doubles * sizeof(double), 256);
    Workspace *ws = nullptr;
    tsqr_status_t st = get_workspace(stream, head_bytes + slots_bytes + table.size(), &ws);
    if (st != TSQR_SUCCESS) return st;
    const size_t table_off = head_bytes + slots_bytes;
    char *base = (char *)ws->base;
    if (ws->table != table || ws->table_off != table_off) {
        if (cudaMemcpyAsync(base + table_off, table.data(), table.size(), cudaMemcpyHostToDevice,
                            stream) != cudaSuccess)
            return TSQR_ERR_CUDA;
        ws->table = table;
        ws->table_off = table_off;
    }
    BatchArgs b;
    b.probs = reinterpret_cast<const BatchProblem *>(base + table_off);
    b.items = reinterpret_cast<const int2 *>(base + table_off + sizeof(BatchProblem) * probs.size());
    b.nitems = (int)items.size();
    b.queue = reinterpret_cast<unsigned int *>(base);
    b.counters = b.queue + 1;
    b.slots = reinterpret_cast<double *>(base + head_bytes);
    b.status = ws->status;
    if (cudaMemsetAsync(base, 0, (size_t)(1 + nodes_total) * sizeof(unsigned int), stream) !=
        cudaSuccess)
        return TSQR_ERR_CUDA;
    const int grid = (int)std::min<int64_t>(ctas, (int64_t)items.size());
    if ((wy ? batched_wy_launch(b, grid, dt == 2, wy_h, wy_tcols, smem, stream)
            : batched_launch(kdt, b, grid, W, smem, stream)) != cudaSuccess)
        return TSQR_ERR_CUDA;
    g_last_launches = 1;
    tsqr_batch_plan_t used{};
    used.warps = W;
    used.ctas_per_sm = wy ? 1 : budget == one_per_sm ? 1 : 2;
    used.leaves_per_cta = lpc;
    for (int b2 = 0; b2 < 4; ++b2) used.arity[b2] = bp.arity[b2];
    used.leaf = mixed ? (wy ? TSQR_LEAF_PANELS : TSQR_LEAF_FOLD) : 0;
    g_last_batch_plan = used;
    return TSQR_SUCCESS;
}

bool bad_dims(int64_t m, int64_t n, int64_t lda, int64_t ldr) {
    return m < 0 || n < 0 || lda < std::max<int64_t>(1, m) || ldr < std::max<int64_t>(1, n);
}

}  // namespace

namespace tsqr {

// The AUTO plan of tsqr_r expressed as kernel arguments (A, R, workspace and status left for
// the caller to fill), for entry points that bring their own workspace.
tsqr_status_t f64_auto_args(int64_t m, int n, F64Args *a, int *warps, size_t *smem,
                            int64_t *nodes, tsqr_plan_t *plan) {
    F64Plan p;
    const tsqr_status_t st = plan_f64(m, n, nullptr, &p);
    if (st != TSQR_SUCCESS) return st;
    *a = plan_args(p, nullptr, m, n, 0);
    *warps = p.warps;
    *smem = p.smem;
    *nodes = p.nodes;
    *plan = public_plan(p);
    return TSQR_SUCCESS;
}

void set_last_call(int launches, const tsqr_plan_t &plan) {
    g_last_launches = launches;
    g_last_plan = plan;
}

}  // namespace tsqr

extern "C" {

const char *tsqr_status_string(int32_t s) {
    switch (s) {
        case TSQR_SUCCESS: return "success";
        case TSQR_ERR_INVALID_ARG: return "invalid argument";
        case TSQR_ERR_UNSUPPORTED: return "unsupported size or configuration";
        case TSQR_ERR_CUDA: return "CUDA runtime error";
        case TSQR_ERR_ALLOC: return "workspace allocation failed";
        case TSQR_ERR_TIMEOUT: return "bounded device wait timed out";
        case TSQR_STATUS_NONFINITE: return "R holds NaN or Inf";
        default: return "unknown status";
    }
}

int32_t tsqr_last_launch_count(void) { return g_last_launches; }

tsqr_status_t tsqr_r(const double *A, int64_t m, int64_t n, int64_t lda, double *R, int64_t ldr,
                     tsqr_stream_t stream) {
    g_last_launches = 0;
    g_last_plan = tsqr_plan_t{};
    if (bad_dims(m, n, lda, ldr)) return TSQR_ERR_INVALID_ARG;
    if (n > TSQR_MAX_N && (m < n || n > 0x7fffffffLL)) return TSQR_ERR_UNSUPPORTED;
    if (n > 0 && (!R || (m > 0 && !A))) return TSQR_ERR_INVALID_ARG;
    return run_f64(A, m, n, lda, R, ldr, nullptr, (cudaStream_t)stream);
}

tsqr_status_t tsqr_r_ex(const void *A, int32_t dtype, int32_t prec, int64_t m, int64_t n,
                        int64_t lda, double *R, int64_t ldr, const tsqr_plan_t *plan,
                        tsqr_stream_t stream) {
    g_last_launches = 0;
    g_last_plan = tsqr_plan_t{};
    if (bad_dims(m, n, lda, ldr)) return TSQR_ERR_INVALID_ARG;
    if (dtype < TSQR_F64 || dtype > TSQR_BF16 || prec < TSQR_PREC_F64 || prec > TSQR_PREC_MIXED)
        return TSQR_ERR_INVALID_ARG;
    const bool f64 = dtype == TSQR_F64 && prec == TSQR_PREC_F64;
    if (n > TSQR_MAX_N && (!f64 || m < n || n > 0x7fffffffLL)) return TSQR_ERR_UNSUPPORTED;
    if (n > 0 && (!R || (m > 0 && !A))) return TSQR_ERR_INVALID_ARG;
    if (f64) return run_f64((const double *)A, m, n, lda, R, ldr, plan, (cudaStream_t)stream);
    if (dtype == TSQR_F64 || prec == TSQR_PREC_F64) return TSQR_ERR_INVALID_ARG;
    return run_mixed(A, dtype == TSQR_BF16, m, n, lda, R, ldr, plan, (cudaStream_t)stream);
}

tsqr_status_t tsqr_lstsq(const double *A, int64_t m, int64_t n, int64_t lda, const double *B,
                         int64_t ldb, int64_t k, double *X, int64_t ldx, double *R, int64_t ldr,
                         const tsqr_plan_t *plan, tsqr_stream_t stream) {
    g_last_launches = 0;
    g_last_plan = tsqr_plan_t{};
    if (bad_dims(m, n, lda, std::max<int64_t>(ldr, n)) || n < 1 || m < n || k < 0 ||
        ldb < std::max<int64_t>(1, m) || ldx < n || (R && ldr < n))
        return TSQR_ERR_INVALID_ARG;
    if (!A || (k > 0 && (!B || !X))) return TSQR_ERR_INVALID_ARG;
    if (plan && plan->warps % 4 != 0) return TSQR_ERR_INVALID_ARG;  // as for tsqr_qr
    if (n > TSQR_MAX_N) {
        if (!plan_is_auto(plan) || n + k > 0x7fffffffLL) return TSQR_ERR_UNSUPPORTED;
        return run_lstsq_panels(A, m, n, lda, B, ldb, k, X, ldx, R, ldr, (cudaStream_t)stream);
    }
    return run_lstsq(A, m, n, lda, B, ldb, k, X, ldx, R, ldr, plan, (cudaStream_t)stream);
}

tsqr_status_t tsqr_caqr_r(const double *A, int64_t m, int64_t n, int64_t lda, double *R,
                          int64_t ldr, int64_t panel, const tsqr_plan_t *plan,
                          tsqr_stream_t stream) {
    g_last_launches = 0;
    g_last_plan = tsqr_plan_t{};
    if (bad_dims(m, n, lda, ldr) || n < 1 || m < n || panel < 0 || !A || !R)
        return TSQR_ERR_INVALID_ARG;
    if (panel > TSQR_MAX_N || n > 0x7fffffffLL) return TSQR_ERR_UNSUPPORTED;
    if (plan && plan->warps % 4 != 0) return TSQR_ERR_INVALID_ARG;  // as for tsqr_qr
    const int64_t nb = panel > 0 ? panel : std::min<int64_t>(n, kCaqrPanel);
    return run_caqr(A, m, n, lda, R, ldr, nb, plan, (cudaStream_t)stream);
}

tsqr_status_t tsqr_r_host(const double *A, int64_t m, int64_t n, int64_t lda, double *R,
                          int64_t ldr, tsqr_stream_t stream) {
    g_last_launches = 0;
    g_last_plan = tsqr_plan_t{};
    if (bad_dims(m, n, lda, ldr)) return TSQR_ERR_INVALID_ARG;
    if (n > TSQR_MAX_N && (m < n || n > 0x7fffffffLL)) return TSQR_ERR_UNSUPPORTED;
    if (n > 0 && (!R || (m > 0 && !A))) return TSQR_ERR_INVALID_ARG;
    return run_f64_host(A, m, n, lda, R, ldr, (cudaStream_t)stream);
}

tsqr_status_t tsqr_qr(const double *A, int64_t m, int64_t n, int64_t lda, double *Q,
                      int64_t ldq, double *R, int64_t ldr, const tsqr_plan_t *plan,
                      tsqr_stream_t stream) {
    g_last_launches = 0;
    g_last_plan = tsqr_plan_t{};
    if (bad_dims(m, n, lda, ldr) || n < 1 || m < n || ldq < m) return TSQR_ERR_INVALID_ARG;
    if (!A || !Q || !R) return TSQR_ERR_INVALID_ARG;
    if (n > TSQR_MAX_N) return TSQR_ERR_UNSUPPORTED;
    return run_qr(A, m, n, lda, Q, ldq, R, ldr, plan, (cudaStream_t)stream);
}

tsqr_status_t tsqr_qr_uppers(int64_t n, const double *R1, int64_t ld1, const double *R2,
                             int64_t ld2, double *R, int64_t ldr, int32_t normalize,
                             tsqr_stream_t stream) {
    g_last_launches = 0;
    g_last_plan = tsqr_plan_t{};
    if (n < 0 || ld1 < std::max<int64_t>(1, n) || ld2 < std::max<int64_t>(1, n) ||
        ldr < std::max<int64_t>(1, n))
        return TSQR_ERR_INVALID_ARG;
    if (n == 0) return TSQR_SUCCESS;
    if (n > TSQR_MAX_N) return TSQR_ERR_UNSUPPORTED;
    if (!R1 || !R2 || !R) return TSQR_ERR_INVALID_ARG;
    const int W = (n <= 64) ? 4 : 8;
    const int hs = (int)round_up(n, W);
    const int ldS = ld_for(hs);
    const size_t smem = f64_smem_bytes((int)n, hs, ldS, W);
    if (f64_prepare(smem) != cudaSuccess) return TSQR_ERR_CUDA;
    Workspace *ws = nullptr;
    tsqr_status_t st = get_workspace((cudaStream_t)stream, 0, &ws);
    if (st != TSQR_SUCCESS) return st;
    if (f64_combine_launch((int)n, R1, ld1, R2, ld2, R, ldr, normalize ? 1 : 0, W, ldS, hs, smem,
                           ws->status, (cudaStream_t)stream) != cudaSuccess)
        return TSQR_ERR_CUDA;
    g_last_launches = 1;
    return TSQR_SUCCESS;
}

}  // extern "C"

namespace {
// Argument checks shared by the batched entry points; *dt receives the kernels' input type
// (0 FP64, 1 FP32, 2 BF16).  count == 0 is valid (nothing to do).
tsqr_status_t check_batch(const void *const *ptrs, const int64_t *ms, const int32_t *ns,
                          const int64_t *offsets, int32_t count, double *R_packed, int32_t dtype,
                          int32_t prec, int *dt) {
    if (count < 0) return TSQR_ERR_INVALID_ARG;
    const bool f64 = (dtype == TSQR_F64 && prec == TSQR_PREC_F64);
    const bool mixed = (dtype == TSQR_F32 || dtype == TSQR_BF16) && prec == TSQR_PREC_MIXED;
    if (!f64 && !mixed) return TSQR_ERR_INVALID_ARG;
    *dt = f64 ? 0 : (dtype == TSQR_F32 ? 1 : 2);
    if (count == 0) return TSQR_SUCCESS;
    if (!ptrs || !ms || !ns || !offsets || !R_packed) return TSQR_ERR_INVALID_ARG;
    for (int32_t i = 0; i < count; ++i) {
        if (ms[i] < 0 || ns[i] < 1 || offsets[i] < 0) return TSQR_ERR_INVALID_ARG;
        if (ns[i] > TSQR_MAX_N) return TSQR_ERR_UNSUPPORTED;
        if (offsets[i + 1] - offsets[i] < (int64_t)ns[i] * ns[i]) return TSQR_ERR_INVALID_ARG;
        if (ms[i] > 0 && !ptrs[i]) return TSQR_ERR_INVALID_ARG;
    }
    return TSQR_SUCCESS;
}
}  // namespace

extern "C" {

tsqr_status_t tsqr_r_batched(const void *const *ptrs, const int64_t *ms, const int32_t *ns,
                             const int64_t *offsets, int32_t count, double *R_packed,
                             int32_t dtype, int32_t prec, tsqr_stream_t stream) {
    return tsqr_r_batched_ex(ptrs, ms, ns, offsets, count, R_packed, dtype, prec, nullptr, stream);
}

tsqr_status_t tsqr_r_batched_ex(const void *const *ptrs, const int64_t *ms, const int32_t *ns,
                                const int64_t *offsets, int32_t count, double *R_packed,
                                int32_t dtype, int32_t prec, const tsqr_batch_plan_t *plan,
                                tsqr_stream_t stream) {
    g_last_launches = 0;
    g_last_plan = tsqr_plan_t{};
    g_last_batch_plan = tsqr_batch_plan_t{};
    int dt = 0;
    const tsqr_status_t st = check_batch(ptrs, ms, ns, offsets, count, R_packed, dtype, prec, &dt);
    if (st != TSQR_SUCCESS || count == 0) return st;
    return run_batched(ptrs, ms, ns, offsets, count, R_packed, dt, plan, (cudaStream_t)stream);
}

tsqr_status_t tsqr_last_batch_plan(tsqr_batch_plan_t *out) {
    if (!out) return TSQR_ERR_INVALID_ARG;
    *out = g_last_batch_plan;
    return TSQR_SUCCESS;
}

tsqr_status_t tsqr_autotune_batched(const void *const *ptrs, const int64_t *ms, const int32_t *ns,
                                    const int64_t *offsets, int32_t count, double *R_packed,
                                    int32_t dtype, int32_t prec, tsqr_batch_plan_t *best,
                                    tsqr_stream_t stream) {
    g_last_launches = 0;
    g_last_plan = tsqr_plan_t{};
    g_last_batch_plan = tsqr_batch_plan_t{};
    int dt = 0;
    tsqr_status_t st = check_batch(ptrs, ms, ns, offsets, count, R_packed, dtype, prec, &dt);
    if (st != TSQR_SUCCESS) return st;
    if (count == 0) return TSQR_ERR_INVALID_ARG;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return TSQR_ERR_CUDA;
    {
        // the search starts from the built-in rules, which an all-zero plan means once the
        // bucket has no tuned plan
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_batch_tuned.erase(batch_key(dev, dt, ms, ns, count));
    }
    const cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return TSQR_ERR_CUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return TSQR_ERR_CUDA;
    }
    // time of one plan: one call to warm up (workspace, table upload), then one timed call; a
    // plan run_batched refuses scores -1
    auto time_plan = [&](const tsqr_batch_plan_t &c, float *ms_out) -> tsqr_status_t {
        *ms_out = -1.0f;
        if (run_batched(ptrs, ms, ns, offsets, count, R_packed, dt, &c, s) != TSQR_SUCCESS)
            return TSQR_SUCCESS;
        if (cudaEventRecord(e0, s) != cudaSuccess) return TSQR_ERR_CUDA;
        const tsqr_status_t r = run_batched(ptrs, ms, ns, offsets, count, R_packed, dt, &c, s);
        if (r != TSQR_SUCCESS) return r;
        if (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
            cudaEventElapsedTime(ms_out, e0, e1) != cudaSuccess)
            return TSQR_ERR_CUDA;
        return TSQR_SUCCESS;
    };
    // coordinate search from the built-in rules (all fields 0): bulk warps x CTAs per SM, then
    // leaves per CTA, then the tree arity of each width bucket present
    tsqr_batch_plan_t cur{};
    float cur_ms = -1.0f;
    auto consider = [&](const tsqr_batch_plan_t &c) -> tsqr_status_t {
        float t = 0.0f;
        const tsqr_status_t r = time_plan(c, &t);
        if (r != TSQR_SUCCESS) return r;
        if (t >= 0.0f && (cur_ms < 0.0f || t < cur_ms)) {
            cur_ms = t;
            cur = c;
        }
        return TSQR_SUCCESS;
    };
    int present = 0, nmax = 1;
    for (int32_t i = 0; i < count; ++i) {
        present |= 1 << width_bucket(ns[i]);
        nmax = std::max(nmax, (int)ns[i]);
    }
    st = consider(tsqr_batch_plan_t{});
    // mixed batches up to 112 columns: the fold leaf against the blocked one first; the warps
    // and chunk-height knobs are the fold's
    if (dt != 0 && nmax <= kMixedWyMaxN)
        for (int lf : {TSQR_LEAF_FOLD, TSQR_LEAF_PANELS}) {
            if (st != TSQR_SUCCESS) break;
            tsqr_batch_plan_t c{};
            c.leaf = lf;
            st = consider(c);
        }
    const bool fold_knobs = !(dt != 0 && nmax <= kMixedWyMaxN && cur.leaf != TSQR_LEAF_FOLD);
    for (int w : {4, 6, 8, 12})
        for (int k : {1, 2}) {
            if (st != TSQR_SUCCESS || !fold_knobs) break;
            tsqr_batch_plan_t c = cur;
            c.warps = w;
            c.ctas_per_sm = k;
            st = consider(c);
        }
    for (int l : {2, 3, 4, 6, 10, 16}) {
        if (st != TSQR_SUCCESS) break;
        tsqr_batch_plan_t c = cur;
        c.leaves_per_cta = l;
        st = consider(c);
    }
    for (int b = 0; b < 4; ++b) {
        if (!((present >> b) & 1)) continue;
        for (int a : {2, 4, 8}) {
            if (st != TSQR_SUCCESS) break;
            tsqr_batch_plan_t c = cur;
            c.arity[b] = a;
            st = consider(c);
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    g_last_launches = 0;
    g_last_plan = tsqr_plan_t{};
    g_last_batch_plan = tsqr_batch_plan_t{};
    if (st != TSQR_SUCCESS) return st;
    if (cur_ms < 0.0f) return TSQR_ERR_UNSUPPORTED;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_batch_tuned[batch_key(dev, dt, ms, ns, count)] = cur;
    }
    if (best) *best = cur;
    return TSQR_SUCCESS;
}

// Test hook (not part of the C ABI in include/tsqr.h): a bounded device wait on an mbarrier,
// completed (arrive != 0) or left to run out after `limit` polls, which then sets the timeout
// bit of the stream's status word (read back by tsqr_get_device_status as TSQR_ERR_TIMEOUT).
// result: device int, 1 if the wait succeeded.
extern "C" int tsqr_internal_wait_selftest(int64_t limit, int32_t arrive, int32_t *result,
                                           tsqr_stream_t stream) {
    if (limit < 1 || limit > (1LL << 20) || !result) return TSQR_ERR_INVALID_ARG;
    Workspace *ws = nullptr;
    const tsqr_status_t st = get_workspace((cudaStream_t)stream, 0, &ws);
    if (st != TSQR_SUCCESS) return st;
    return tsqr::wait_selftest_launch(limit, arrive, ws->status, result, (cudaStream_t)stream) == 0
               ? TSQR_SUCCESS
               : TSQR_ERR_CUDA;
}

tsqr_status_t tsqr_get_device_status(tsqr_stream_t stream) {
    cudaStream_t s = (cudaStream_t)stream;
    if (cudaStreamSynchronize(s) != cudaSuccess) return TSQR_ERR_CUDA;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return TSQR_ERR_CUDA;
    int flags = 0;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        auto it = g_ws.find({dev, s});
        if (it == g_ws.end() || !it->second.status) return TSQR_SUCCESS;
        if (cudaMemcpy(&flags, it->second.status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
            return TSQR_ERR_CUDA;
        if (cudaMemset(it->second.status, 0, sizeof(int)) != cudaSuccess) return TSQR_ERR_CUDA;
    }
    if (flags & kStatusTimeoutBit) return TSQR_ERR_TIMEOUT;
    return (flags & kStatusNonfiniteBit) ? TSQR_STATUS_NONFINITE : TSQR_SUCCESS;
}

void tsqr_release_workspace(void) {
    std::lock_guard<std::mutex> lk(g_mu);
    int cur = 0;
    cudaGetDevice(&cur);
    for (auto &kv : g_ws) {
        cudaSetDevice(kv.first.first);
        cudaDeviceSynchronize();
        if (kv.second.base) cudaFree(kv.second.base);
        if (kv.second.status) cudaFree(kv.second.status);
    }
    g_ws.clear();
    cudaSetDevice(cur);
}

tsqr_status_t tsqr_last_plan(tsqr_plan_t *out) {
    if (!out) return TSQR_ERR_INVALID_ARG;
    *out = g_last_plan;
    return TSQR_SUCCESS;
}

tsqr_status_t tsqr_resolve_plan(int64_t m, int64_t n, int32_t dtype, int32_t prec,
                                const tsqr_plan_t *plan, tsqr_plan_t *out) {
    if (!out || m < 0 || n < 1) return TSQR_ERR_INVALID_ARG;
    const bool f64 = (dtype == TSQR_F64 && prec == TSQR_PREC_F64);
    if (n > TSQR_MAX_N && (!f64 || m < n)) return TSQR_ERR_UNSUPPORTED;
    const bool mixed = (dtype == TSQR_F32 || dtype == TSQR_BF16) && prec == TSQR_PREC_MIXED;
    if (!f64 && !mixed) return TSQR_ERR_INVALID_ARG;
    if (f64 && m > 0) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess) return TSQR_ERR_CUDA;
        const int64_t nb = panels_width(m, n, plan, dev);
        if (nb > 0) {
            *out = tsqr_plan_t{};
            out->tree = TSQR_TREE_PANELS;
            out->tile_rows = (int32_t)nb;
            return TSQR_SUCCESS;
        }
    }
    F64Plan p;
    tsqr_status_t st = mixed ? plan_mixed(m, (int)n, dtype == TSQR_BF16, plan, &p)
                             : plan_leaf(m, (int)n, plan, false, &p);
    if (st != TSQR_SUCCESS) return st;
    *out = public_plan(p);
    return TSQR_SUCCESS;
}

tsqr_status_t tsqr_autotune(const void *A, int32_t dtype, int32_t prec, int64_t m, int64_t n,
                            int64_t lda, double *R, int64_t ldr, tsqr_plan_t *best,
                            tsqr_stream_t stream) {
    g_last_launches = 0;
    g_last_plan = tsqr_plan_t{};
    if (bad_dims(m, n, lda, ldr) || n < 1 || m < 1 || !A || !R) return TSQR_ERR_INVALID_ARG;
    if (n > TSQR_MAX_N) return TSQR_ERR_UNSUPPORTED;
    const bool f64 = (dtype == TSQR_F64 && prec == TSQR_PREC_F64);
    const bool mixed = (dtype == TSQR_F32 || dtype == TSQR_BF16) && prec == TSQR_PREC_MIXED;
    if (!f64 && !mixed) return TSQR_ERR_INVALID_ARG;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return TSQR_ERR_CUDA;
    const DeviceInfo di = device_info(dev);
    if (di.sms <= 0) return TSQR_ERR_CUDA;
    const cudaStream_t s = (cudaStream_t)stream;
    // candidates: HYBRID slabs as tall as fit k CTAs per SM (k = 1, 2, 3), and half as tall,
    // with 4, 12 or 8 bulk warps; k CTAs per SM on every SM
    std::vector<tsqr_plan_t> cands;
    const int warps_opts[5] = {4, 12, 8, 6, 5};
    for (int wi = 0; wi < 5; ++wi) {
        const int W = warps_opts[wi];
        for (int k = 1; k <= 3; ++k) {
            const size_t reserve = 1024;
            if (di.smem_sm <= k * reserve) continue;
            const size_t budget = std::min(di.smem_block_optin, (di.smem_sm - k * reserve) / k);
            const int rmax = good_r(max_rows_per_lane_p((int)n, W, budget, mixed));
            if (rmax < 1) continue;
            for (int r : {rmax, good_r(std::max(1, rmax / 2))}) {
                const int64_t tile = 32LL * W * r;
                if (tile < n) continue;
                const int64_t units = (m + tile - 1) / tile;
                tsqr_plan_t c{TSQR_TREE_HYBRID, (int32_t)tile,
                              (int32_t)std::min<int64_t>((int64_t)di.sms * k, units), W, 0,
                              mixed ? TSQR_LEAF_FOLD : 0};
                bool dup = false;
                for (const auto &o : cands)
                    dup |= (o.tile_rows == c.tile_rows && o.ctas == c.ctas && o.warps == c.warps);
                if (!dup) cands.push_back(c);
            }
        }
    }
    if (f64 && n >= 48 && m >= 8 * n)
        for (int32_t nb : {16, 32}) cands.push_back(tsqr_plan_t{TSQR_TREE_PANELS, nb, 0, 0, 0, 0});
    // the blocked mixed leaf: every chunk height the width's shared and tensor memory hold, with
    // 1 .. as many CTAs as fit on every SM
    if (mixed && n <= kMixedWyMaxN)
        for (int32_t hh : kMixedWyHeights) {
            const size_t sm_b = mixed_wy_smem_bytes((int)n, hh);
            if (sm_b + 1024 > di.smem_block_optin || !mixed_wy_tmem_fits((int)n, hh) ||
                mixed_wy_prepare(sm_b) != cudaSuccess)
                continue;
            const int per_sm = std::max(1, mixed_wy_blocks_per_sm(hh, sm_b));
            const int64_t units = (m + hh - 1) / hh;
            for (int k = 1; k <= per_sm; ++k)
                cands.push_back(tsqr_plan_t{TSQR_TREE_HYBRID, hh,
                                            (int32_t)std::min<int64_t>((int64_t)di.sms * k, units),
                                            8, 0, TSQR_LEAF_PANELS});
        }
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return TSQR_ERR_CUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return TSQR_ERR_CUDA;
    }
    float best_ms = -1.0f;
    tsqr_plan_t best_plan{};
    tsqr_status_t st = TSQR_SUCCESS;
    for (const auto &c : cands) {
        auto call = [&]() {
            return f64 ? run_f64((const double *)A, m, n, lda, R, ldr, &c, s)
                       : run_mixed(A, dtype == TSQR_BF16, m, n, lda, R, ldr, &c, s);
        };
        if (call() != TSQR_SUCCESS) continue;  // a candidate the planner rejects is skipped
        float ms = 0.0f;
        if (cudaEventRecord(e0, s) != cudaSuccess) { st = TSQR_ERR_CUDA; break; }
        bool ok = true;
        for (int rep = 0; rep < 3 && ok; ++rep) ok = (call() == TSQR_SUCCESS);
        if (!ok || cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
            cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
            st = TSQR_ERR_CUDA;
            break;
        }
        if (best_ms < 0.0f || ms < best_ms) {
            best_ms = ms;
            best_plan = c;
        }
    }
    // then the tree arity of the fastest one-reduction plan: 2 (the paper's binary tree) to 8
    if (st == TSQR_SUCCESS && best_ms >= 0.0f && best_plan.tree == TSQR_TREE_HYBRID) {
        const tsqr_plan_t base = best_plan;
        for (int32_t k : {2, 3, 4, 6, 8}) {
            tsqr_plan_t c = base;
            c.arity = k;
            auto call = [&]() {
                return f64 ? run_f64((const double *)A, m, n, lda, R, ldr, &c, s)
                           : run_mixed(A, dtype == TSQR_BF16, m, n, lda, R, ldr, &c, s);
            };
            if (call() != TSQR_SUCCESS) continue;  // an arity the width's memory cannot hold
            float ms = 0.0f;
            if (cudaEventRecord(e0, s) != cudaSuccess) { st = TSQR_ERR_CUDA; break; }
            bool ok = true;
            for (int rep = 0; rep < 3 && ok; ++rep) ok = (call() == TSQR_SUCCESS);
            if (!ok || cudaEventRecord(e1, s) != cudaSuccess ||
                cudaEventSynchronize(e1) != cudaSuccess ||
                cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
                st = TSQR_ERR_CUDA;
                break;
            }
            if (ms < best_ms) {
                best_ms = ms;
                best_plan = c;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    g_last_launches = 0;
    g_last_plan = tsqr_plan_t{};
    if (st != TSQR_SUCCESS) return st;
    if (best_ms < 0.0f) return TSQR_ERR_UNSUPPORTED;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tuned[TuneKey{dev, (int)n, mixed ? 1 : 0, floor_log2(m)}] = best_plan;
    }
    if (best) *best = best_plan;
    return TSQR_SUCCESS;
}

void tsqr_autotune_reset(void) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tuned.clear();
    g_batch_tuned.clear();
}

}  // extern "C"
