// FP64 TSQR device code: the shared-memory fold R <- R([R; S]) that serves both as the leaf
// (S = a row slab of A, Section 2 step 1 fused with a flat tree, Section 1) and as the tree
// operator qr(R1, R2) (S = R2, an upper triangle; Section 2, Table 3), plus the cross-CTA
// binary reduction tree (Fig. 1) with the "last child to arrive combines" rule.
//
// Cost model this is written for (measured on GB300): one warp-wide FP64 instruction occupies a
// sub-partition's FP64 unit for ~64 cycles whether 1 or 32 lanes are active, FP64 latency is
// ~65 cycles, sqrt ~620 and divide ~375 cycles; everything that is not FP64 (shared-memory
// traffic, integer work, shuffles, barriers) is nearly free by comparison.  Hence:
//   * the bulk pass spreads its (row, column) items evenly over all 32 lanes, whatever the
//     shrinking width of the trailing triangle, and fuses the update by reflector j with the
//     dot products for reflector j+1 (one sweep, two FMAs per item);
//   * partial dot products are summed along fixed, index-determined orders (bit-reproducible);
//   * the per-column scalar work (norm, sqrt, divides) is done once per CTA by one warp.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace tsqr {

constexpr int kMaxN = 128;
constexpr int kMaxLevels = 48;
// Partial-sum slots per warp for width n: one per lane plus one per column boundary a lane's
// run can cross (a slot index is lane + column offset < 32 + n).
__host__ __device__ inline int seg_stride(int n) { return 32 + n; }

// Binary reduction tree over `count[0]` leaves (host side): level l has count[l] nodes; node t
// of level l+1 has children 2t and 2t+1 of level l (an odd last child is promoted unchanged).
// Node (l, t) has the global id offset[l] + t; the kernels walk the same levels incrementally.
struct TreeShape {
    int levels;
    int count[kMaxLevels];
    int offset[kMaxLevels];
};

// Where the factorization behind tsqr_qr keeps its reflectors for forming Q (all null for the
// R-only kernels).  Reflector J of a chunk or node is H = I - tau v v^T with v = [e_J; c x],
// x its stored tail; (tau, c) = (0, 0) for an identity reflector.
struct QStore {
    double *V;         // m x n, leading dimension ldv: each chunk's tails, in the chunk's rows
    int64_t ldv;
    double *chunk_sc;  // per chunk (id = first row / h): tau_J, c_J for J = 0..n-1
    double *node_V;    // per tree node id: arity-1 stacked n x n tails, leading dim (arity-1) n
    double *node_sc;   // per tree node id: tau_J, c_J
    double *signs;     // n entries: -1 where the root's R(k,k) < 0 (rows the sign convention
                       // negates), else +1
};

struct F64Args {
    const double *A;
    int64_t m, lda;
    int n;
    int64_t unit;   // rows of a work unit: a tile (binary tree) or a slab (flat, hybrid)
    int64_t nunits; // ceil(m / unit)
    int nleaves;    // CTAs of the leaf phase; leaf c owns units [c*nunits/nleaves, ...)
    int arity;      // children per tree node (2 = the paper's binary operator)
    int h;          // rows folded per step of a leaf ("chunk"): h <= hs
    int hs;         // rows of S in shared memory: >= max(h, n), a multiple of 32 x warps
    int blk;        // rows per inner-loop block: divides hs / (32 x warps)
    int vec;        // elements per shared-memory access in that loop (divides blk and ldS)
    int ldS;        // leading dimension of S in shared memory (elements)
    double *slots;          // one n x n column-major slot per tree node (workspace)
    unsigned int *counters; // one arrival counter per tree node (workspace, zeroed per call)
    double *R;              // output, column-major n x n, ld ldr
    int64_t ldr;
    int *status;            // device status word (TSQR_STATUS_NONFINITE is or-ed in)
    QStore q;               // reflector storage (tsqr_qr's factorization only)
};

// Mixed-precision kernel arguments: the FP64 arguments (base.A unused) plus A of another
// type, and the FP64 view of the S region used by the tree operator.
struct MixedArgs {
    F64Args base;
    const void *A;  // FP32 or BF16, column-major, leading dimension base.lda
    int ldSd;       // leading dimension of the FP64 view of S (tree operator)
    int s_doubles;  // size of the S region in doubles
};

// One problem of a varlen batch, as the batched kernel sees it (device memory).
struct BatchProblem {
    const void *A;           // column-major m x n, leading dimension lda (FP64, FP32 or BF16)
    int64_t m, lda;
    double *R;               // column-major n x n, leading dimension n
    int64_t unit, nunits;    // rows per leaf, number of leaves
    int n, h, hs, blk, vec, ldS;  // as in F64Args
    int nleaves, arity;
    int64_t slot_off;        // first tree slot of this problem (doubles into the slots buffer)
    int64_t cnt_off;         // first tree counter of this problem
};

struct BatchArgs {
    const BatchProblem *probs;
    const int2 *items;       // (problem, leaf) work items, in the order CTAs take them
    int nitems;
    unsigned int *queue;     // work-queue head, zeroed per call
    double *slots;
    unsigned int *counters;  // zeroed per call
    int *status;
};

// Leading dimension of the tree operator's FP64 view of the S region: odd, and room for
// arity-1 stacked n x n triangles.
__host__ __device__ inline int tree_ldsd(int n, int arity) {
    const int v = (arity > 2 ? arity - 1 : 1) * n;
    return (v % 2 == 0) ? v + 1 : v;
}
// Size in doubles of the mixed kernels' S region: the FP32 chunk or the FP64 triangles.
__host__ __device__ inline int mixed_s_doubles_of(int n, int ldS, int arity) {
    const int leaf = (ldS * n + 1) / 2;
    const int tree = tree_ldsd(n, arity) * n;
    return leaf > tree ? leaf : tree;
}
// Largest arity (<= 8) whose stacked triangles fit in `s_doubles` doubles of the S region.
__host__ __device__ inline int arity_for(int n, int s_doubles) {
    int k = 2;
    while (k < 8 && tree_ldsd(n, k + 1) * n <= s_doubles) ++k;
    return k;
}

// Shared-memory carve-up (offsets in doubles), identical on host and device.  The S region
// holds s_doubles doubles.
struct SmemLayout {
    int S, Rp, f, fs, seg, tot, npart, scal, total;
};

__host__ __device__ inline SmemLayout smem_layout_s(int n, int s_doubles, int warps) {
    SmemLayout L;
    int o = 0;
    L.S = o;      o += s_doubles;
    L.Rp = o;     o += n * (n + 1) / 2 + 1;
    L.f = o;      o += n + 1;
    L.fs = o;     o += n / 2 + 1;  // FP32 copy of f (mixed leaf)
    L.seg = o;    o += warps * seg_stride(n);
    L.tot = o;    o += 2 * seg_stride(n);  // summed slots, then the per-column dot products
    L.npart = o;  o += warps * 32;
    L.scal = o;   o += 4;
    L.total = o;
    return L;
}

// The FP64 layout: S is an ldS x n FP64 chunk.
__host__ __device__ inline SmemLayout smem_layout(int n, int hs, int ldS, int warps) {
    (void)hs;
    return smem_layout_s(n, ldS * n, warps);
}

// Packed upper triangle, row-major: row j holds R(j, j..n-1) at rowoff(j).
__host__ __device__ inline int rowoff(int n, int j) { return j * n - (j * (j - 1)) / 2; }

}  // namespace tsqr
