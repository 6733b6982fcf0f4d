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
};

// The leaf pass: the leaf partition of the factorization (m, unit, nunits, nleaves, h) and
// its chunk buffer shape (hs rows, leading dimension ldS).
struct QLeafArgs {
    double *Q;                // in: the chunks' tails (QStore::V); out: Q
    int64_t m, ldq;
    int n;
    int64_t unit, nunits;
    int nleaves, h, hs, ldS;
    const double *chunk_sc;   // per chunk (id = first row / h): tau_J, c_J
    const double *B;          // per leaf: n x n block, leading dimension n
    const double *signs;      // the root's row signs (used when the only leaf is the root)
    int single;               // one leaf: its block is diag(signs)
};

// Offsets in doubles: the tails X and the Q rows Z (ldS x n each), the carried block (n x n),
// the update factors g, the chunk's scalars, the partial-sum slots and their sums.
struct QLeafLayout {
    int X, Z, top, g, sc, seg, tot, total;
};

__host__ __device__ inline QLeafLayout q_leaf_layout(int n, int ldS, int warps_total) {
    QLeafLayout L;
    int o = 0;
    L.X = o;    o += ldS * n;
    L.Z = o;    o += ldS * n;
    L.top = o;  o += n * n;
    L.g = o;    o += n + 1;
    L.sc = o;   o += 2 * n;
    L.seg = o;  o += warps_total * seg_stride(n);
    L.tot = o;  o += 2 * seg_stride(n);
    L.total = o;
    return L;
}

}  // namespace tsqr
