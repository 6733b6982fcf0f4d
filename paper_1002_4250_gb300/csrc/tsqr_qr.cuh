// Kernel arguments and shared-memory layout of the Q-forming passes of tsqr_qr.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "tsqr_f64.cuh"

namespace tsqr {

// One level of the top-down tree pass: the parents are the nodes of level L (count, first
// node id), the children those of level L-1.
struct QTreeArgs {
    int n, arity;
    int level_off;            // first node id of level L (node (L, t) has id level_off + t)
    int child_cnt, child_off; // nodes of level L-1 and the first one's id
    int is_root;              // level L is the root: its block is diag(signs)
    const double *node_V;     // per node id: stacked tails, leading dimension (arity-1) n
    const double *node_sc;    // per node id: tau_J, c_J
    const double *signs;
    double *B;                // per node id: n x n block, leading dimension n (in and out)
    int qg;                   // columns per group: the blocks' columns are independent, and
                              // the kernel takes them qg at a time to bound shared memory
};

// The leaf pass: the leaf partition of the factorization (m, unit, nunits, nleaves, h) and
// its chunk buffer shape (hs rows, leading dimension ldS).
struct QLeafArgs {
    double *Q;                // out: columns q0 .. q0+qn-1 of Q
    int64_t m, ldq;
    const double *V;          // the chunks' tails (QStore::V, Q itself when qn = n)
    int64_t ldv;
    int q0, qn;               // the column group of this launch (columns are independent)
    int n;
    int64_t unit, nunits;
    int nleaves, h, hs, ldS;
    const double *chunk_sc;   // per chunk (id = first row / h): tau_J, c_J
    const double *B;          // per leaf: n x n block, leading dimension n
    const double *signs;      // the root's row signs (used when the only leaf is the root)
    int single;               // one leaf: its block is diag(signs)
    const double *wyS;        // the chunks' compact WY factors (the blocked leaf pass), or
                              // NULL: the pass forms them itself (one column group)
};

// Offsets in doubles: the tails X (ldS x n), the Q rows Z of the column group (ldS x qn), the
// carried block's columns (n x qn), the update factors g, the chunk's scalars, the
// partial-sum slots and their sums.
struct QLeafLayout {
    int X, Z, top, g, sc, seg, tot, total;
};

__host__ __device__ inline QLeafLayout q_leaf_layout(int n, int qn, int ldS, int warps_total) {
    QLeafLayout L;
    int o = 0;
    L.X = o;    o += ldS * n;
    L.Z = o;    o += ldS * qn;
    L.top = o;  o += n * qn;
    L.g = o;    o += qn + 1;
    L.sc = o;   o += 2 * n;
    L.seg = o;  o += warps_total * seg_stride(qn);
    L.tot = o;  o += 2 * seg_stride(qn);
    L.total = o;
    return L;
}

// Q^T applied to B (tsqr_lstsq): the factorization's leaf partition and chunk shape, its stored
// reflectors, and B (m x k, leading dimension ldb).  Each leaf folds its chunks of B, first to
// last, into a k-column block T (the rows of Q^T B that belong to its R); the leaves then
// climb the factorization's tree, where the last child to arrive applies the node's reflectors
// to its children's stacked blocks.  The root's block, with the sign convention's row signs,
// is the first n rows of Q^T B, written to C.
struct QtArgs {
    const double *V;          // the chunks' tails (QStore::V), leading dimension ldv
    int64_t ldv;
    const double *B;          // m x k, leading dimension ldb
    int64_t m, ldb;
    int n, k;
    int64_t unit, nunits;
    int nleaves, h, hs, ldS, arity;
    const double *chunk_sc;   // per chunk: tau_J, c_J
    const double *node_V;     // per node id: stacked tails, leading dimension (arity-1) n
    const double *node_sc;    // per node id: tau_J, c_J
    const double *signs;      // the root's row signs
    double *slots;            // per node id: n x k block, leading dimension n
    unsigned int *counters;   // per node id: arrivals (zeroed per call)
    double *C;                // out: n x k, leading dimension ldc
    int64_t ldc;
    // Column groups: blockIdx.y takes columns y k .. y k + k - 1 of the ktot columns of B (and
    // of Cout and C); each group has its own counters and slots, nodes apart.
    int ktot;
    int64_t nodes;
    // The whole of Q^T B (the trailing update of a panel factorization), when Cout is set: each
    // chunk's rows of Q^T B go to the same rows of Cout (B itself is allowed), and the rows a
    // tree node leaves behind (every child's block but the first) to rows grow0 .. of Cout, in
    // a fixed order.  Together with the n rows in C they are Q^T B up to a row permutation.
    double *Cout;
    int64_t ldco, grow0;
    // The chunks' compact WY factors (per chunk id, n x n, from tsqr_wy_kernel), for the
    // blocked leaf part; unused by the reflector-by-reflector one.
    const double *wyS;
};

// Compact WY form of each chunk's reflectors.  Reflector J of a chunk is v_J = [e_J; c_J x_J]
// (row J of the carried triangle, then the chunk's rows), so with V = [I; X diag(c)] the
// product H_0 H_1 ... H_{n-1} is I - V S V^T with S upper triangular (forward accumulation:
// S(J,J) = tau_J, S(0:J,J) = -tau_J S(0:J,0:J) V(:,0:J)^T v_J, and V(:,i)^T v_J = c_i c_J x_i . x_J
// for i < J).  One S per chunk id, n x n with leading dimension n.
struct WyArgs {
    const double *V;          // the chunks' tails, leading dimension ldv
    int64_t ldv, m;
    int n, h, ldX;            // chunk rows and the shared-memory leading dimension (>= h)
    int64_t nchunks;
    const double *chunk_sc;   // per chunk: tau_J, c_J
    double *S;                // out
};

// Blocked leaf part of the Q^T apply: the tails X diag(c) (ldS x n), B's chunk Z (ldS x kc),
// the carried block T (n x kc), S (n x n), W = V^T [T; Z] (n x kc), the partial sums of W's row
// slices (which then hold S^T W), the chunk's c, and the climb's counter word.
struct WyLayout {
    int X, Z, top, S, W, part, cs, flag, total;
};

// fused: the apply forms each chunk's S itself (one column group), its G in the part region.
__host__ __device__ inline WyLayout wy_layout(int n, int kc, int ldS, int nthreads,
                                              bool fused = false) {
    WyLayout L;
    int o = 0;
    L.X = o;    o += ldS * n;
    L.Z = o;    o += ldS * kc;
    L.top = o;  o += n * kc;
    L.S = o;    o += n * n;
    L.W = o;    o += n * kc;
    int part = (4 * nthreads > n * kc) ? 4 * nthreads : n * kc;
    if (fused && part < n * n) part = n * n;
    L.part = o; o += part;
    L.cs = o;   o += n;
    L.flag = o; o += 1;
    L.total = o;
    return L;
}

// Offsets in doubles: the tails X (ldS x n), B's chunk Z (ldS x k), the block T (n x k), the
// stacked children's blocks during the climb (reusing X and Z), the factors g, the chunk's
// scalars, the partial-sum slots and their sums, and one word for the climb's counter value.
struct QtLayout {
    int X, Z, top, g, sc, seg, tot, flag, total;
};

__host__ __device__ inline QtLayout qt_layout(int n, int k, int ldS, int warps_total) {
    QtLayout L;
    int o = 0;
    L.X = o;    o += ldS * n;
    L.Z = o;    o += ldS * k;
    L.top = o;  o += n * k;
    L.g = o;    o += k + 1;
    L.sc = o;   o += 2 * n;
    L.seg = o;  o += warps_total * seg_stride(k);
    L.tot = o;  o += 2 * seg_stride(k);
    L.flag = o; o += 1;
    L.total = o;
    return L;
}

// Blocked leaf pass: the tails X diag(c) (ldS x n), the carried block's columns T (n x qn),
// S (n x n), Y = S T (n x qn), and the chunk's c.
struct QLeafWyLayout {
    int X, top, S, Y, cs, G, total;
};

// fused: the pass forms each chunk's S itself (one column group), with G (n x n) beside it.
__host__ __device__ inline QLeafWyLayout q_leaf_wy_layout(int n, int qn, int ldS, bool fused) {
    QLeafWyLayout L;
    int o = 0;
    L.X = o;    o += ldS * n;
    L.top = o;  o += n * qn;
    L.S = o;    o += n * n;
    L.Y = o;    o += n * qn;
    L.cs = o;   o += n;
    L.G = o;    o += fused ? n * n : 0;
    L.total = o;
    return L;
}

}  // namespace tsqr
