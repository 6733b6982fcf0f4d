// Thin QR (tsqr_qr): the R factorization of tsqr_r with its reflectors kept, then Q formed by
// applying them to the first n columns of the identity, top-down through the tree and then
// backwards through each leaf's chunks.  Section 3: computing Q means applying the stored
// Householder transformations to the identity, which needs every node's Householder vectors
// and the shape of the reduction tree.
//
// Q = H_tree [D; 0] spread over the leaves, D = diag(row signs of the sign convention), where a
// tree node with children c_0 .. c_{k-1} (stacked in index order, c_0 on top) maps its block
// B (n x n) to its children's blocks [B_0; ...; B_{k-1}] = H_node [B; 0]; a leaf maps its block
// to its rows of Q chunk by chunk, last chunk first: [B'; Q_c] = H_chunk [B; 0], B' going on
// to the previous chunk (the leaf folded its chunks in order, R_c = R([R_{c-1}; S_c])).
#include <cstdint>
#include <cuda_runtime.h>

#include "tsqr_fold.cuh"
#include "tsqr_internal.h"
#include "tsqr_qr.cuh"

namespace tsqr {

// ------------------------------------------------------------------------------------------
// Factorization with storage: tsqr_r's leaf + tree kernel keeping its reflectors in a.q.
// ------------------------------------------------------------------------------------------
template <int B>
__global__ void __launch_bounds__(416, 1) tsqr_qr_factor_kernel(const F64Args a) {
    leaf_tree_job<double, double, B, 1, B == 1, true>(a, a.A, a.ldS, a.ldS * a.n, blockIdx.x);
}

namespace {
const void *qr_factor_fn(int blk) {
    switch (blk) {
        case 4: return (const void *)tsqr_qr_factor_kernel<4>;
        case 3: return (const void *)tsqr_qr_factor_kernel<3>;
        case 2: return (const void *)tsqr_qr_factor_kernel<2>;
        default: return (const void *)tsqr_qr_factor_kernel<1>;
    }
}
}  // namespace

// ------------------------------------------------------------------------------------------
// Tree pass, one launch per level from the root down: CTA t applies node (L, t)'s reflectors
// to [B; 0] and writes its children's blocks.  Reflector J (reverse order) touches row J of the
// top block and rows 0..J of each stacked block; its columns are independent, so each column
// is handled by tpc lanes of one warp (no block barrier inside the loop).
// ------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(256) tsqr_q_tree_kernel(const QTreeArgs a) {
    extern __shared__ __align__(16) double smem[];
    const int n = a.n, k = a.arity, t = blockIdx.x;
    const int first = t * k;
    const int nchild = min(k, a.child_cnt - first);
    const size_t id = (size_t)a.level_off + t;
    const double *Bin = a.B + id * n * n;
    if (nchild == 1) {  // a promoted lone child: its block is the node's
        double *dst = a.B + ((size_t)a.child_off + first) * n * n;
        for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
            const int col = idx / n, row = idx - col * n;
            dst[idx] = a.is_root ? ((row == col) ? a.signs[row] : 0.0) : Bin[idx];
        }
        return;
    }
    const int c = nchild - 1, ldX = (k - 1) * n;
    const double *X = a.node_V + id * (size_t)ldX * n;
    const double *sc = a.node_sc + id * 2 * n;
    const int qg = a.qg;
    const int ldT = c * n;
    double *top = smem;           // n x qg, leading dimension n
    double *T = smem + n * qg;    // (nchild-1) n x qg, leading dimension (nchild-1) n
    int tpc = 1;  // lanes per column: a power of two <= 32 with tpc qg <= blockDim
    while (tpc < 32 && 2 * tpc * qg <= (int)blockDim.x) tpc *= 2;
    const int q0t = threadIdx.x / tpc, sub = threadIdx.x - q0t * tpc;
    for (int g0 = 0; g0 < n; g0 += qg) {
        const int gn = min(qg, n - g0);
        __syncthreads();  // the previous group's blocks are written out
        for (int idx = threadIdx.x; idx < n * gn; idx += blockDim.x) {
            const int col = idx / n, row = idx - col * n;
            top[idx] = a.is_root ? ((row == g0 + col) ? a.signs[row] : 0.0)
                                 : Bin[row + (size_t)(g0 + col) * n];
        }
        for (int idx = threadIdx.x; idx < ldT * gn; idx += blockDim.x) T[idx] = 0.0;
        __syncthreads();
        const bool active = q0t < gn;
        const int q = active ? q0t : gn - 1;  // idle lanes shadow the last column, writing nothing
        for (int J = n - 1; J >= 0; --J) {
            const double tau = sc[2 * J], cj = sc[2 * J + 1];
            if (tau == 0.0) continue;
            const int h1 = J + 1, E = c * h1;
            double d = 0.0;
            for (int e = sub; e < E; e += tpc) {
                const int tt = e / h1, i = e - tt * h1;
                d = fma(X[tt * n + i + (size_t)J * ldX], T[tt * n + i + q * ldT], d);
            }
            for (int o = tpc >> 1; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o, tpc);
            const double w = fma(cj, d, top[J + q * n]);
            __syncwarp();
            if (active && sub == 0) top[J + q * n] = fma(-tau, w, top[J + q * n]);
            const double gq = tau * cj * w;
            if (active) {
                for (int e = sub; e < E; e += tpc) {
                    const int tt = e / h1, i = e - tt * h1;
                    T[tt * n + i + q * ldT] = fma(-gq, X[tt * n + i + (size_t)J * ldX],
                                                  T[tt * n + i + q * ldT]);
                }
            }
            __syncwarp();
        }
        __syncthreads();
        for (int ch = 0; ch < nchild; ++ch) {
            double *dst = a.B + ((size_t)a.child_off + first + ch) * n * n;
            for (int idx = threadIdx.x; idx < n * gn; idx += blockDim.x) {
                const int col = idx / n, row = idx - col * n;
                dst[row + (size_t)(g0 + col) * n] =
                    (ch == 0) ? top[idx] : T[(ch - 1) * n + row + col * ldT];
            }
        }
    }
}

// ------------------------------------------------------------------------------------------
// Leaf pass.  One CTA per leaf, with the leaf fold's warps (W bulk + 1 reducer) and its
// lockstep item split.  Per chunk, last first: X = the chunk's tails (read from Q), Z = 0 and
// the carried block B ("top"); for J = n-1 .. 0, the bulk sweep applies reflector J+1's update
// Z(:,q) -= g_q x_{J+1} and forms x_J . Z(:,q) for every column q; the reducer sums the
// partials, w_q = B(J,q) + c_J d_q, B(J,q) -= tau_J w_q, g_q = tau_J c_J w_q.  After J = 0,
// Z(:,q) -= g_q x_0 and Z is the chunk's rows of Q.
// ------------------------------------------------------------------------------------------
// Software pipelined: the next block's operands are loaded before the current block is
// updated and stored (the two blocks never overlap: different rows, or the next column).
// ncols: the columns of Z (n for the Q leaf pass, k for the Q^T B pass).
template <int B>
__device__ __forceinline__ void q_sweep(const int lane, const int ncols, const int r, const int Hw,
                                        double *__restrict__ Z, const int ldS, const int r0,
                                        const double *__restrict__ xu,
                                        const double *__restrict__ xd,
                                        const double *__restrict__ g, double *__restrict__ seg) {
    const int run = ncols * r;
    const int nblk = run / B;
    const int p = lane * run;
    int kk = p / Hw;
    int i = p - kk * Hw;
    double *Zk = Z + (size_t)kk * ldS + r0;
    double acc = 0.0;
    double z[B], d[B];
#pragma unroll
    for (int q = 0; q < B; ++q) {
        z[q] = Zk[i + q];
        d[q] = xd[i + q];
    }
    if (xu) {
        double gk = g[kk];
        double u[B];
#pragma unroll
        for (int q = 0; q < B; ++q) u[q] = xu[i + q];
        for (int blk = 0; blk < nblk; ++blk) {
            int i2 = i + B, kk2 = kk;
            double *Zk2 = Zk;
            const bool cross = (i2 == Hw);
            if (cross) {
                i2 = 0;
                ++kk2;
                Zk2 += ldS;
            }
            double z2[B], d2[B], u2[B];
            if (blk + 1 < nblk) {
#pragma unroll
                for (int q = 0; q < B; ++q) {
                    z2[q] = Zk2[i2 + q];
                    d2[q] = xd[i2 + q];
                    u2[q] = xu[i2 + q];
                }
            }
            double x[B];
#pragma unroll
            for (int q = 0; q < B; ++q) x[q] = fma(-gk, u[q], z[q]);
#pragma unroll
            for (int q = 0; q < B; ++q) Zk[i + q] = x[q];
#pragma unroll
            for (int q = 0; q < B; ++q) acc = fma(d[q], x[q], acc);
            if (cross) {
                seg[lane + kk] = acc;
                acc = 0.0;
                gk = g[min(kk2, ncols - 1)];
            }
            i = i2;
            kk = kk2;
            Zk = Zk2;
#pragma unroll
            for (int q = 0; q < B; ++q) {
                z[q] = z2[q];
                d[q] = d2[q];
                u[q] = u2[q];
            }
        }
    } else {
        for (int blk = 0; blk < nblk; ++blk) {
            int i2 = i + B, kk2 = kk;
            double *Zk2 = Zk;
            const bool cross = (i2 == Hw);
            if (cross) {
                i2 = 0;
                ++kk2;
                Zk2 += ldS;
            }
            double z2[B], d2[B];
            if (blk + 1 < nblk) {
#pragma unroll
                for (int q = 0; q < B; ++q) {
                    z2[q] = Zk2[i2 + q];
                    d2[q] = xd[i2 + q];
                }
            }
#pragma unroll
            for (int q = 0; q < B; ++q) acc = fma(d[q], z[q], acc);
            if (cross) {
                seg[lane + kk] = acc;
                acc = 0.0;
            }
            i = i2;
            kk = kk2;
            Zk = Zk2;
#pragma unroll
            for (int q = 0; q < B; ++q) {
                z[q] = z2[q];
                d[q] = d2[q];
            }
        }
    }
    if (i != 0) seg[lane + kk] = acc;
}

// Block: W bulk warps (a multiple of 4 up to 12, hs a multiple of 32 W) and the reducer.
template <int B>
__global__ void __launch_bounds__(416, 1) tsqr_q_leaf_kernel(const QLeafArgs a) {
    extern __shared__ __align__(16) double smem[];
    const int n = a.n, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int Wb = (blockDim.x >> 5) - 1;
    const bool reducer = (warp == Wb);
    const int Hw = a.hs / Wb, r = Hw >> 5, r0 = warp * Hw;
    const int qn = a.qn, q0 = a.q0;
    const QLeafLayout L = q_leaf_layout(n, qn, a.ldS, Wb + 1);
    double *X = smem + L.X;
    double *Z = smem + L.Z;
    double *top = smem + L.top;
    double *g = smem + L.g;
    double *sc = smem + L.sc;
    const int ss = seg_stride(qn);
    double *seg_all = smem + L.seg;
    double *seg = seg_all + warp * ss;
    double *tot = smem + L.tot;
    const int nslot = 32 + qn;
    constexpr int kGroups = 4;
    const int leaf = blockIdx.x;

    for (int idx = threadIdx.x; idx < n * qn; idx += blockDim.x) {
        const int col = idx / n, row = idx - col * n;
        top[idx] = a.single ? ((row == q0 + col) ? a.signs[row] : 0.0)
                            : a.B[(size_t)leaf * n * n + row + (size_t)(q0 + col) * n];
    }
    const int64_t u0 = ((int64_t)leaf * a.nunits) / a.nleaves;
    const int64_t u1 = ((int64_t)(leaf + 1) * a.nunits) / a.nleaves;
    const int64_t rbeg = u0 * a.unit;
    const int64_t rend = (u1 * a.unit < a.m) ? u1 * a.unit : a.m;
    const int64_t nchunks = (rend - rbeg + a.h - 1) / a.h;
    for (int64_t c = nchunks - 1; c >= 0; --c) {
        const int64_t row0 = rbeg + c * a.h;
        const int rows = (int)((rend - row0 < a.h) ? rend - row0 : a.h);
        __syncthreads();  // the previous chunk's X and Z are no longer read
        for (int idx = threadIdx.x; idx < a.hs * n; idx += blockDim.x) {
            const int col = idx / a.hs, i = idx - col * a.hs;
            X[i + (size_t)col * a.ldS] = (i < rows) ? a.V[row0 + i + (int64_t)col * a.ldv] : 0.0;
        }
        for (int idx = threadIdx.x; idx < a.hs * qn; idx += blockDim.x) {
            const int col = idx / a.hs, i = idx - col * a.hs;
            Z[i + (size_t)col * a.ldS] = 0.0;
        }
        const double *csc = a.chunk_sc + (row0 / a.h) * 2 * n;
        for (int j = threadIdx.x; j < 2 * n; j += blockDim.x) sc[j] = csc[j];
        __syncthreads();
        for (int J = n - 1; J >= 0; --J) {
            if (!reducer) {
                for (int id = lane; id < nslot; id += 32) seg[id] = 0.0;
                __syncwarp();
                q_sweep<B>(lane, qn, r, Hw, Z, a.ldS, r0,
                           (J + 1 < n) ? X + (size_t)(J + 1) * a.ldS + r0 : nullptr,
                           X + (size_t)J * a.ldS + r0, g, seg);
            }
            __syncthreads();
            // slot sums over the bulk warps, spread over the whole CTA: slot id's partials in
            // kGroups runs of consecutive warps, each run summed by one lane of a kGroups-lane
            // team, the runs then combined by shuffles (a fixed order)
            for (int base = 0; base < nslot * kGroups; base += blockDim.x) {
                const int t = base + threadIdx.x;
                const int id = t / kGroups, gi = t - id * kGroups;
                double v = 0.0;
                if (id < nslot) {
                    const int w0 = (gi * Wb) / kGroups, w1 = ((gi + 1) * Wb) / kGroups;
                    for (int w = w0; w < w1; ++w) v += seg_all[w * ss + id];
                }
#pragma unroll
                for (int o = kGroups >> 1; o > 0; o >>= 1)
                    v += __shfl_xor_sync(0xffffffffu, v, o, kGroups);
                if (id < nslot && gi == 0) tot[id] = v;
            }
            __syncthreads();
            if (reducer) {
                const double tau = sc[2 * J], cj = sc[2 * J + 1];
                const int Nw = qn * Hw;
                for (int q = lane; q < qn; q += 32) {
                    // column q's partials: slots q + la .. q + lb (as in the leaf fold)
                    const int la = (32 * (q * Hw + 1) - 1) / Nw;
                    const int lb = (32 * (q + 1) * Hw - 1) / Nw;
                    double d0 = tot[q + la], d1 = 0.0;
                    for (int l = la + 1; l + 1 <= lb; l += 2) {
                        d0 += tot[q + l];
                        d1 += tot[q + l + 1];
                    }
                    if (((lb - la) & 1) == 1) d0 += tot[q + lb];
                    const double w = fma(cj, d0 + d1, top[J + q * n]);
                    top[J + q * n] = fma(-tau, w, top[J + q * n]);
                    g[q] = tau * cj * w;
                }
            }
            __syncthreads();
        }
        if (!reducer) {  // reflector 0's update
            for (int q = 0; q < qn; ++q) {
                const double gq = g[q];
                for (int t = 0; t < r; ++t) {
                    const int i = r0 + lane + 32 * t;
                    Z[i + (size_t)q * a.ldS] = fma(-gq, X[i], Z[i + (size_t)q * a.ldS]);
                }
            }
        }
        __syncthreads();
        for (int idx = threadIdx.x; idx < rows * qn; idx += blockDim.x) {
            const int col = idx / rows, i = idx - col * rows;
            a.Q[row0 + i + (int64_t)(q0 + col) * a.ldq] = Z[i + (size_t)col * a.ldS];
        }
    }
}

// The climb of the Q^T apply: the leaf's block T (top, n x kc) goes up the factorization's tree
// (same shape, node ids and stored reflectors); the last child to arrive at a node applies the
// node's reflectors to the children's stacked blocks (X's space holds all but the first), the
// others stay behind (to Og), and the root writes D T to Cg.
__device__ __forceinline__ void qt_climb(const QtArgs &a, const int leaf, const int kc, double *X,
                                         double *top, unsigned int *flag, double *Cg, double *Og,
                                         unsigned int *counters, double *slots) {
    const int n = a.n;
    const int k = a.arity;
    int cnt = a.nleaves, off = 0, t = leaf;
    int64_t left = 0;  // n-row blocks left behind by the levels below (cnt - next_cnt each)
    for (;;) {
        if (cnt == 1) {
            for (int idx = threadIdx.x; idx < n * kc; idx += blockDim.x) {
                const int col = idx / n, i = idx - col * n;
                Cg[i + (int64_t)col * a.ldc] = a.signs[i] * top[idx];
            }
            return;
        }
        const int next_off = off + cnt, next_cnt = (cnt + k - 1) / k;
        const int parent = t / k, first = parent * k;
        const int nchild = min(k, cnt - first);
        if (nchild == 1) {
            left += cnt - next_cnt;
            off = next_off;
            cnt = next_cnt;
            t = parent;
            continue;
        }
        double *mine = slots + (size_t)(off + t) * n * kc;
        for (int idx = threadIdx.x; idx < n * kc; idx += blockDim.x) mine[idx] = top[idx];
        __threadfence();
        __syncthreads();
        if (threadIdx.x == 0) flag[0] = atomicAdd(&counters[next_off + parent], 1u);
        __syncthreads();
        if (flag[0] + 1 < (unsigned)nchild) return;
        __threadfence();
        // the children's blocks in index order: the first on top, the others stacked in X
        const int cs = nchild - 1, ldY = cs * n;
        double *Y = X;
        for (int idx = threadIdx.x; idx < n * kc; idx += blockDim.x)
            top[idx] = __ldcg(slots + (size_t)(off + first) * n * kc + idx);
        for (int idx = threadIdx.x; idx < cs * n * kc; idx += blockDim.x) {
            const int col = idx / (cs * n), rr = idx - col * (cs * n);
            const int tt = rr / n, i = rr - tt * n;
            Y[rr + (size_t)col * ldY] =
                __ldcg(slots + (size_t)(off + first + 1 + tt) * n * kc + i + (size_t)col * n);
        }
        __syncthreads();
        const size_t id = (size_t)next_off + parent;
        const int ldX = (k - 1) * n;
        const double *Xn = a.node_V + id * (size_t)ldX * n;
        const double *nsc = a.node_sc + id * 2 * n;
        int tpc = 1;  // lanes per column: a power of two <= 32 with tpc kc <= blockDim
        while (tpc < 32 && 2 * tpc * kc <= (int)blockDim.x) tpc *= 2;
        const int q0 = threadIdx.x / tpc, sub = threadIdx.x - q0 * tpc;
        const bool active = q0 < kc;
        const int q = active ? q0 : kc - 1;
        for (int J = 0; J < n; ++J) {
            const double tau = nsc[2 * J], cj = nsc[2 * J + 1];
            if (tau == 0.0) continue;
            const int h1 = J + 1, E = cs * h1;
            double d = 0.0;
            for (int e = sub; e < E; e += tpc) {
                const int tt = e / h1, i = e - tt * h1;
                d = fma(Xn[tt * n + i + (size_t)J * ldX], Y[tt * n + i + (size_t)q * ldY], d);
            }
            for (int o = tpc >> 1; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o, tpc);
            const double w = fma(cj, d, top[J + q * n]);
            __syncwarp();
            if (active && sub == 0) top[J + q * n] = fma(-tau, w, top[J + q * n]);
            const double gq = tau * cj * w;
            if (active) {
                for (int e = sub; e < E; e += tpc) {
                    const int tt = e / h1, i = e - tt * h1;
                    Y[tt * n + i + (size_t)q * ldY] = fma(-gq, Xn[tt * n + i + (size_t)J * ldX],
                                                          Y[tt * n + i + (size_t)q * ldY]);
                }
            }
            __syncwarp();
        }
        __syncthreads();
        if (Og) {  // the blocks of children 1 .. cs stay behind: the node's n-row blocks
            const int64_t rb = a.grow0 + (left + (int64_t)parent * (k - 1)) * n;
            for (int idx = threadIdx.x; idx < cs * n * kc; idx += blockDim.x) {
                const int col = idx / (cs * n), rr = idx - col * (cs * n);
                Og[rb + rr + (int64_t)col * a.ldco] = Y[rr + (size_t)col * ldY];
            }
        }
        left += cnt - next_cnt;
        off = next_off;
        cnt = next_cnt;
        t = parent;
    }
}

// ------------------------------------------------------------------------------------------
// Q^T B (tsqr_lstsq, tsqr_caqr_r).  One CTA per leaf and column group, as the leaf pass: per
// chunk, first to last, X = the
// chunk's tails, Z = the chunk's rows of B and T the leaf's block (zero at the start, the rows
// of the zero triangle the first chunk was folded under); for J = 0 .. n-1 the bulk sweep
// applies reflector J-1's update Z(:,q) -= g_q x_{J-1} and forms x_J . Z(:,q) for every column
// q of Z; the reducer forms w_q = T(J,q) + c_J d_q, T(J,q) -= tau_J w_q, g_q = tau_J c_J w_q.
// Only T (the rows of Q^T B that belong to R) goes on; Z, after reflector n-1's update, is the
// chunk's rows of Q^T B, written to Cout where the whole product is wanted (a panel's trailing
// update) and otherwise dropped.  The leaf then climbs the factorization's tree with its T, and
// the last child to arrive at a node applies the node's reflectors, first to last, to
// [T_0; T_1; ...] (row J of T_0 and rows 0..J of every other block); T_1, T_2, ... then stay
// behind (to Cout) and T_0 goes up.  The root writes D T (D: the row signs) to C.
// ------------------------------------------------------------------------------------------
template <int B>
__global__ void __launch_bounds__(416, 1) tsqr_qt_kernel(const QtArgs a) {
    extern __shared__ __align__(16) double smem[];
    const int n = a.n, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int grp = blockIdx.y, kc = min(a.k, a.ktot - grp * a.k);
    const double *Bg = a.B + (int64_t)grp * a.k * a.ldb;
    double *Cg = a.C + (int64_t)grp * a.k * a.ldc;
    double *Og = a.Cout ? a.Cout + (int64_t)grp * a.k * a.ldco : nullptr;
    unsigned int *counters = a.counters + grp * a.nodes;
    double *slots = a.slots + grp * a.nodes * n * a.k;
    const int Wb = (blockDim.x >> 5) - 1;
    const bool reducer = (warp == Wb);
    const int Hw = a.hs / Wb, r = Hw >> 5, r0 = warp * Hw;
    const QtLayout L = qt_layout(n, kc, a.ldS, Wb + 1);
    double *X = smem + L.X;
    double *Z = smem + L.Z;
    double *top = smem + L.top;
    double *g = smem + L.g;
    double *sc = smem + L.sc;
    const int ss = seg_stride(kc);
    double *seg_all = smem + L.seg;
    double *seg = seg_all + warp * ss;
    double *tot = smem + L.tot;
    unsigned int *flag = reinterpret_cast<unsigned int *>(smem + L.flag);
    const int nslot = 32 + kc;
    constexpr int kGroups = 4;
    const int leaf = blockIdx.x;

    for (int idx = threadIdx.x; idx < n * kc; idx += blockDim.x) top[idx] = 0.0;
    const int64_t u0 = ((int64_t)leaf * a.nunits) / a.nleaves;
    const int64_t u1 = ((int64_t)(leaf + 1) * a.nunits) / a.nleaves;
    const int64_t rbeg = u0 * a.unit;
    const int64_t rend = (u1 * a.unit < a.m) ? u1 * a.unit : a.m;
    const int64_t nchunks = (rend - rbeg + a.h - 1) / a.h;
    for (int64_t c = 0; c < nchunks; ++c) {
        const int64_t row0 = rbeg + c * a.h;
        const int rows = (int)((rend - row0 < a.h) ? rend - row0 : a.h);
        __syncthreads();  // the previous chunk's X and Z are no longer read
        for (int idx = threadIdx.x; idx < a.hs * n; idx += blockDim.x) {
            const int col = idx / a.hs, i = idx - col * a.hs;
            X[i + (size_t)col * a.ldS] = (i < rows) ? a.V[row0 + i + (int64_t)col * a.ldv] : 0.0;
        }
        for (int idx = threadIdx.x; idx < a.hs * kc; idx += blockDim.x) {
            const int col = idx / a.hs, i = idx - col * a.hs;
            Z[i + (size_t)col * a.ldS] = (i < rows) ? Bg[row0 + i + (int64_t)col * a.ldb] : 0.0;
        }
        const double *csc = a.chunk_sc + (row0 / a.h) * 2 * n;
        for (int j = threadIdx.x; j < 2 * n; j += blockDim.x) sc[j] = csc[j];
        __syncthreads();
        for (int J = 0; J < n; ++J) {
            if (!reducer) {
                for (int id = lane; id < nslot; id += 32) seg[id] = 0.0;
                __syncwarp();
                q_sweep<B>(lane, kc, r, Hw, Z, a.ldS, r0,
                           (J > 0) ? X + (size_t)(J - 1) * a.ldS + r0 : nullptr,
                           X + (size_t)J * a.ldS + r0, g, seg);
            }
            __syncthreads();
            for (int base = 0; base < nslot * kGroups; base += blockDim.x) {
                const int t = base + threadIdx.x;
                const int id = t / kGroups, gi = t - id * kGroups;
                double v = 0.0;
                if (id < nslot) {
                    const int w0 = (gi * Wb) / kGroups, w1 = ((gi + 1) * Wb) / kGroups;
                    for (int w = w0; w < w1; ++w) v += seg_all[w * ss + id];
                }
#pragma unroll
                for (int o = kGroups >> 1; o > 0; o >>= 1)
                    v += __shfl_xor_sync(0xffffffffu, v, o, kGroups);
                if (id < nslot && gi == 0) tot[id] = v;
            }
            __syncthreads();
            if (reducer) {
                const double tau = sc[2 * J], cj = sc[2 * J + 1];
                const int Nw = kc * Hw;
                for (int q = lane; q < kc; q += 32) {
                    const int la = (32 * (q * Hw + 1) - 1) / Nw;
                    const int lb = (32 * (q + 1) * Hw - 1) / Nw;
                    double d0 = tot[q + la], d1 = 0.0;
                    for (int l = la + 1; l + 1 <= lb; l += 2) {
                        d0 += tot[q + l];
                        d1 += tot[q + l + 1];
                    }
                    if (((lb - la) & 1) == 1) d0 += tot[q + lb];
                    const double w = fma(cj, d0 + d1, top[J + q * n]);
                    top[J + q * n] = fma(-tau, w, top[J + q * n]);
                    g[q] = tau * cj * w;
                }
            }
            __syncthreads();
        }
        if (Og) {
            if (!reducer) {  // reflector n-1's update: Z is then the chunk's rows of Q^T B
                const double *xl = X + (size_t)(n - 1) * a.ldS;
                for (int q = 0; q < kc; ++q) {
                    const double gq = g[q];
                    for (int t = 0; t < r; ++t) {
                        const int i = r0 + lane + 32 * t;
                        Z[i + (size_t)q * a.ldS] = fma(-gq, xl[i], Z[i + (size_t)q * a.ldS]);
                    }
                }
            }
            __syncthreads();
            for (int idx = threadIdx.x; idx < rows * kc; idx += blockDim.x) {
                const int col = idx / rows, i = idx - col * rows;
                Og[row0 + i + (int64_t)col * a.ldco] = Z[i + (size_t)col * a.ldS];
            }
        }
    }

    qt_climb(a, leaf, kc, X, top, flag, Cg, Og, counters, slots);
}

// ------------------------------------------------------------------------------------------
// Compact WY factors.  One CTA per chunk (grid-strided): the scaled tails X diag(c) in shared
// memory, G(i,J) = (c_i x_i) . (c_J x_J) for i < J over the chunk's rows, then S column by
// column, S(0:J,J) = -tau_J S(0:J,0:J) G(0:J,J): row i of S needs only row i's earlier entries,
// so a lane owns a row.
// ------------------------------------------------------------------------------------------
// G(i,J) = x_i . x_J for i < J over the first `rows` rows of the scaled tails X (ldX x n): one
// pair per thread, column by column, two accumulators.
__device__ __forceinline__ void wy_gram(const double *X, const int ldX, const int rows,
                                        const int n, double *G) {
    const int npairs = n * (n - 1) / 2;
    for (int p = threadIdx.x; p < npairs; p += blockDim.x) {
        // pair p -> (i, J), i < J, column by column: J = the largest with J(J-1)/2 <= p
        int J = (int)((1.0 + sqrt(1.0 + 8.0 * p)) * 0.5);
        while (J * (J - 1) / 2 > p) --J;
        while ((J + 1) * J / 2 <= p) ++J;
        const int i = p - J * (J - 1) / 2;
        const double *xi = X + i * ldX, *xj = X + J * ldX;
        double d0 = 0.0, d1 = 0.0;
        int r = 0;
        for (; r + 1 < rows; r += 2) {
            d0 = fma(xi[r], xj[r], d0);
            d1 = fma(xi[r + 1], xj[r + 1], d1);
        }
        if (r < rows) d0 = fma(xi[r], xj[r], d0);
        G[i + J * n] = d0 + d1;
    }
}

// S from G and the chunk's tau (sc[2J]), column by column: column J's rows i < J each by a team
// of tpr lanes (the sum over k = i .. J-1 strided over the team, then a fixed butterfly).  G must
// be complete (a barrier before); S is complete after the call's last barrier.
__device__ __forceinline__ void wy_s_from_g(const double *G, const double *sc, const int n,
                                            double *S) {
    for (int idx = threadIdx.x; idx < n; idx += blockDim.x) {
        for (int i = 0; i < n; ++i) S[i + idx * n] = (i == idx) ? sc[2 * idx] : 0.0;
    }
    for (int J = 1; J < n; ++J) {
        __syncthreads();  // columns 0 .. J-1 are complete
        int tpr = 1;
        while (tpr < 32 && 2 * tpr * J <= (int)blockDim.x) tpr *= 2;
        const int team = threadIdx.x / tpr, sub = threadIdx.x - team * tpr;
        const int i = team < J ? team : J - 1;  // spare teams shadow the last row
        double v = 0.0;
        for (int k = i + sub; k < J; k += tpr) v = fma(S[i + k * n], G[k + J * n], v);
        for (int o = tpr >> 1; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o, tpr);
        if (team < J && sub == 0) S[i + J * n] = -sc[2 * J] * v;
    }
    __syncthreads();
}

__global__ void __launch_bounds__(256) tsqr_wy_kernel(const WyArgs a) {
    extern __shared__ __align__(16) double smem[];
    const int n = a.n, ldX = a.ldX;
    double *X = smem;               // ldX x n
    double *G = smem + ldX * n;     // n x n (strict upper triangle used)
    double *S = G + n * n;          // n x n
    for (int64_t c = blockIdx.x; c < a.nchunks; c += gridDim.x) {
        const int64_t row0 = c * a.h;
        const int rows = (int)((a.m - row0 < a.h) ? a.m - row0 : a.h);
        const double *sc = a.chunk_sc + c * 2 * n;
        __syncthreads();  // the previous chunk's S is written out
        for (int idx = threadIdx.x; idx < rows * n; idx += blockDim.x) {
            const int J = idx / rows, i = idx - J * rows;
            cp_async8(X + i + J * ldX, a.V + row0 + i + (int64_t)J * a.ldv, 8);
        }
        cp_async_commit();
        cp_async_wait_all();
        for (int idx = threadIdx.x; idx < rows * n; idx += blockDim.x) {  // X diag(c), own copies
            const int J = idx / rows, i = idx - J * rows;
            X[i + J * ldX] *= sc[2 * J + 1];
        }
        __syncthreads();
        wy_gram(X, ldX, rows, n, G);
        __syncthreads();
        wy_s_from_g(G, sc, n, S);
        double *out = a.S + c * (int64_t)n * n;
        for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) out[idx] = S[idx];
    }
}

// W = T + X^T Z over the chunk's first `rows` rows (X ldS x n, the scaled tails; Z ldS x kc;
// T, W n x kc).
// Thread tiles of 2 x 2 outputs; where they are fewer than the threads, the rows are split in
// slices whose partial sums are added in slice order.
__device__ __forceinline__ void wy_xtz(const double *X, const double *Z, const int ldS,
                                       const int rows, const int n, const int kc,
                                       const double *T, double *W, double *part) {
    const int NT = blockDim.x;
    const int ti = (n + 1) >> 1, tq = (kc + 1) >> 1, tiles = ti * tq;
    const int slices = tiles >= NT ? 1 : NT / tiles;
    const int rs = (rows + slices - 1) / slices;
    for (int u = threadIdx.x; u < tiles * slices; u += NT) {
        const int tile = u % tiles, sl = u / tiles;
        const int i0 = 2 * (tile % ti), q0 = 2 * (tile / ti);
        const int i1 = min(i0 + 1, n - 1), q1 = min(q0 + 1, kc - 1);
        const int ra = sl * rs, rb = min(rows, ra + rs);
        const double *x0 = X + (size_t)i0 * ldS, *x1 = X + (size_t)i1 * ldS;
        const double *z0 = Z + (size_t)q0 * ldS, *z1 = Z + (size_t)q1 * ldS;
        double a00 = 0.0, a01 = 0.0, a10 = 0.0, a11 = 0.0;
        for (int r = ra; r < rb; ++r) {
            const double xa = x0[r], xb = x1[r], za = z0[r], zb = z1[r];
            a00 = fma(xa, za, a00);
            a01 = fma(xa, zb, a01);
            a10 = fma(xb, za, a10);
            a11 = fma(xb, zb, a11);
        }
        if (slices == 1) {
            W[i0 + q0 * n] = T[i0 + q0 * n] + a00;
            if (q0 + 1 < kc) W[i0 + (q0 + 1) * n] = T[i0 + (q0 + 1) * n] + a01;
            if (i0 + 1 < n) W[i0 + 1 + q0 * n] = T[i0 + 1 + q0 * n] + a10;
            if (i0 + 1 < n && q0 + 1 < kc) W[i0 + 1 + (q0 + 1) * n] = T[i0 + 1 + (q0 + 1) * n] + a11;
        } else {
            double *pp = part + 4 * (size_t)(sl * tiles + tile);
            pp[0] = a00;
            pp[1] = a01;
            pp[2] = a10;
            pp[3] = a11;
        }
    }
    if (slices > 1) {
        __syncthreads();
        for (int o = threadIdx.x; o < n * kc; o += NT) {
            const int i = o % n, q = o / n;
            const int tile = (i >> 1) + (q >> 1) * ti, e = 2 * (i & 1) + (q & 1);
            double v = T[o];
            for (int sl = 0; sl < slices; ++sl) v += part[4 * (size_t)(sl * tiles + tile) + e];
            W[o] = v;
        }
    }
}

// Y = S^T W (trans) or S W, S upper triangular (n x n); T -= Y.
__device__ __forceinline__ void wy_sw(const double *S, const double *W, double *Y, double *T,
                                      const int n, const int kc, const bool trans) {
    for (int o = threadIdx.x; o < n * kc; o += blockDim.x) {
        const int i = o % n, q = o / n;
        const double *w = W + q * n;
        double v = 0.0;
        if (trans) {
            for (int j = 0; j <= i; ++j) v = fma(S[j + i * n], w[j], v);
        } else {
            for (int j = i; j < n; ++j) v = fma(S[i + j * n], w[j], v);
        }
        Y[o] = v;
        T[o] -= v;
    }
}

// Z(r, q) -= sum_j X(r, j) Y(j, q) for r < rows: thread tiles of 4 rows (tr apart, so that a
// warp's lanes read consecutive rows) by 2 columns.
__device__ __forceinline__ void wy_zupdate(double *Z, const double *X, const int ldS,
                                           const int rows, const int n, const int kc,
                                           const double *Y) {
    const int tr = (rows + 3) >> 2, tq = (kc + 1) >> 1;
    for (int u = threadIdx.x; u < tr * tq; u += blockDim.x) {
        const int rr = u % tr, q0 = 2 * (u / tr), q1 = min(q0 + 1, kc - 1);
        int rw[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) rw[k] = min(rr + k * tr, rows - 1);
        double z0[4], z1[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            z0[k] = Z[rw[k] + (size_t)q0 * ldS];
            z1[k] = Z[rw[k] + (size_t)q1 * ldS];
        }
        for (int j = 0; j < n; ++j) {
            const double y0 = Y[j + q0 * n], y1 = Y[j + q1 * n];
            const double *xj = X + (size_t)j * ldS;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const double x = xj[rw[k]];
                z0[k] = fma(-x, y0, z0[k]);
                z1[k] = fma(-x, y1, z1[k]);
            }
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            if (rr + k * tr < rows) {
                Z[rw[k] + (size_t)q0 * ldS] = z0[k];
                if (q0 + 1 < kc) Z[rw[k] + (size_t)q1 * ldS] = z1[k];
            }
        }
    }
}

// The Q^T apply with each chunk's reflectors as one blocked transformation: per chunk, first to
// last (the tails copied asynchronously with B's rows and S, then scaled), W = T + (X diag(c))^T Z,
// Y = S^T W, T -= Y and (where the whole product is wanted) Z -= X diag(c) Y, written to Cout.  Then the same climb.  Two passes over the chunk's rows
// in place of n fused sweeps, and no per-reflector barriers.
__global__ void __launch_bounds__(256, 1) tsqr_qt_wy_kernel(const QtArgs a) {
    extern __shared__ __align__(16) double smem[];
    const int n = a.n;
    const int grp = blockIdx.y, kc = min(a.k, a.ktot - grp * a.k);
    const double *Bg = a.B + (int64_t)grp * a.k * a.ldb;
    double *Cg = a.C + (int64_t)grp * a.k * a.ldc;
    double *Og = a.Cout ? a.Cout + (int64_t)grp * a.k * a.ldco : nullptr;
    unsigned int *counters = a.counters + grp * a.nodes;
    double *slots = a.slots + grp * a.nodes * n * a.k;
    const WyLayout L = wy_layout(n, kc, a.ldS, blockDim.x, a.wyS == nullptr);
    double *X = smem + L.X;
    double *Z = smem + L.Z;
    double *top = smem + L.top;
    double *S = smem + L.S;
    double *W = smem + L.W;
    double *part = smem + L.part;
    double *cs = smem + L.cs;
    unsigned int *flag = reinterpret_cast<unsigned int *>(smem + L.flag);
    const int leaf = blockIdx.x;

    for (int idx = threadIdx.x; idx < n * kc; idx += blockDim.x) top[idx] = 0.0;
    const int64_t u0 = ((int64_t)leaf * a.nunits) / a.nleaves;
    const int64_t u1 = ((int64_t)(leaf + 1) * a.nunits) / a.nleaves;
    const int64_t rbeg = u0 * a.unit;
    const int64_t rend = (u1 * a.unit < a.m) ? u1 * a.unit : a.m;
    const int64_t nchunks = (rend - rbeg + a.h - 1) / a.h;
    for (int64_t c = 0; c < nchunks; ++c) {
        const int64_t row0 = rbeg + c * a.h;
        const int rows = (int)((rend - row0 < a.h) ? rend - row0 : a.h);
        const int64_t cid = row0 / a.h;
        const double *csc = a.chunk_sc + cid * 2 * n;
        __syncthreads();  // the previous chunk's buffers are no longer read
        // asynchronous copies of the tails, B's rows and S; each thread then scales the tails
        // it copied (X diag(c), whose entries are at most 1 in magnitude, is the well-scaled
        // form: c alone overflows where a chunk's rank runs out and the tails become tiny)
        for (int idx = threadIdx.x; idx < rows * n; idx += blockDim.x) {
            const int col = idx / rows, i = idx - col * rows;
            cp_async8(X + i + (size_t)col * a.ldS, a.V + row0 + i + (int64_t)col * a.ldv, 8);
        }
        for (int idx = threadIdx.x; idx < rows * kc; idx += blockDim.x) {
            const int col = idx / rows, i = idx - col * rows;
            cp_async8(Z + i + (size_t)col * a.ldS, Bg + row0 + i + (int64_t)col * a.ldb, 8);
        }
        if (a.wyS) {
            const double *Sg = a.wyS + cid * (int64_t)n * n;
            for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x)
                cp_async8(S + idx, Sg + idx, 8);
        }
        cp_async_commit();
        for (int j = threadIdx.x; j < n; j += blockDim.x) cs[j] = csc[2 * j + 1];
        cp_async_wait_all();
        __syncthreads();
        for (int idx = threadIdx.x; idx < rows * n; idx += blockDim.x) {
            const int col = idx / rows, i = idx - col * rows;
            X[i + (size_t)col * a.ldS] *= cs[col];
        }
        __syncthreads();
        if (!a.wyS) {  // one column group: the chunk's S here (G in the part region, free now)
            wy_gram(X, a.ldS, rows, n, part);
            __syncthreads();
            wy_s_from_g(part, csc, n, S);
        }
        wy_xtz(X, Z, a.ldS, rows, n, kc, top, W, part);
        __syncthreads();
        wy_sw(S, W, part, top, n, kc, true);
        if (Og) {
            __syncthreads();
            wy_zupdate(Z, X, a.ldS, rows, n, kc, part);
            __syncthreads();
            for (int idx = threadIdx.x; idx < rows * kc; idx += blockDim.x) {
                const int col = idx / rows, i = idx - col * rows;
                Og[row0 + i + (int64_t)col * a.ldco] = Z[i + (size_t)col * a.ldS];
            }
        }
    }
    __syncthreads();
    qt_climb(a, leaf, kc, X, top, flag, Cg, Og, counters, slots);
}

// The leaf pass with each chunk's reflectors as one blocked transformation: the chunk's rows of
// [T; 0] under H_0 H_1 ... H_{n-1} = I - V S V^T are T - S T on top and -X diag(c) S T below.
// Per chunk, last to first: Y = S T, T -= Y, and the chunk's rows of Q, -X diag(c) Y, are
// written straight from registers.  Only half the flops of the sweep (no dot products with
// the chunk's rows, which are zero before the chunk's reflectors reach them).
__global__ void __launch_bounds__(256, 1) tsqr_q_leaf_wy_kernel(const QLeafArgs a) {
    extern __shared__ __align__(16) double smem[];
    const int n = a.n, qn = a.qn, q0 = a.q0;
    const QLeafWyLayout L = q_leaf_wy_layout(n, qn, a.ldS, a.wyS == nullptr);
    double *X = smem + L.X;
    double *top = smem + L.top;
    double *S = smem + L.S;
    double *Y = smem + L.Y;
    double *cs = smem + L.cs;
    const int leaf = blockIdx.x;
    for (int idx = threadIdx.x; idx < n * qn; idx += blockDim.x) {
        const int col = idx / n, row = idx - col * n;
        top[idx] = a.single ? ((row == q0 + col) ? a.signs[row] : 0.0)
                            : a.B[(size_t)leaf * n * n + row + (size_t)(q0 + col) * n];
    }
    const int64_t u0 = ((int64_t)leaf * a.nunits) / a.nleaves;
    const int64_t u1 = ((int64_t)(leaf + 1) * a.nunits) / a.nleaves;
    const int64_t rbeg = u0 * a.unit;
    const int64_t rend = (u1 * a.unit < a.m) ? u1 * a.unit : a.m;
    const int64_t nchunks = (rend - rbeg + a.h - 1) / a.h;
    for (int64_t c = nchunks - 1; c >= 0; --c) {
        const int64_t row0 = rbeg + c * a.h;
        const int rows = (int)((rend - row0 < a.h) ? rend - row0 : a.h);
        const int64_t cid = row0 / a.h;
        const double *csc = a.chunk_sc + cid * 2 * n;
        __syncthreads();  // the previous chunk's X, S and Y are no longer read
        for (int idx = threadIdx.x; idx < rows * n; idx += blockDim.x) {
            const int col = idx / rows, i = idx - col * rows;
            cp_async8(X + i + (size_t)col * a.ldS, a.V + row0 + i + (int64_t)col * a.ldv, 8);
        }
        if (a.wyS) {
            const double *Sg = a.wyS + cid * (int64_t)n * n;
            for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x)
                cp_async8(S + idx, Sg + idx, 8);
        }
        cp_async_commit();
        for (int j = threadIdx.x; j < n; j += blockDim.x) cs[j] = csc[2 * j + 1];
        cp_async_wait_all();
        __syncthreads();
        for (int idx = threadIdx.x; idx < rows * n; idx += blockDim.x) {  // X diag(c)
            const int col = idx / rows, i = idx - col * rows;
            X[i + (size_t)col * a.ldS] *= cs[col];
        }
        if (!a.wyS) {  // one column group: the chunk's S here, from the tails just loaded
            __syncthreads();
            wy_gram(X, a.ldS, rows, n, smem + L.G);
            __syncthreads();
            wy_s_from_g(smem + L.G, csc, n, S);
        }
        for (int o = threadIdx.x; o < n * qn; o += blockDim.x) {  // Y = S T (S upper)
            const int i = o % n, q = o / n;
            double v = 0.0;
            for (int j = i; j < n; ++j) v = fma(S[i + j * n], top[j + q * n], v);
            Y[o] = v;
        }
        __syncthreads();
        for (int o = threadIdx.x; o < n * qn; o += blockDim.x) top[o] -= Y[o];
        // Q rows: thread tiles of 4 rows (tr apart) by 2 columns, -sum_j X(r, j) Y(j, q)
        const int tr = (rows + 3) >> 2, tq = (qn + 1) >> 1;
        for (int u = threadIdx.x; u < tr * tq; u += blockDim.x) {
            const int rr = u % tr, qa = 2 * (u / tr), qb = min(qa + 1, qn - 1);
            int rw[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) rw[k] = min(rr + k * tr, rows - 1);
            double z0[4] = {0.0, 0.0, 0.0, 0.0}, z1[4] = {0.0, 0.0, 0.0, 0.0};
            for (int j = 0; j < n; ++j) {
                const double y0 = Y[j + qa * n], y1 = Y[j + qb * n];
                const double *xj = X + (size_t)j * a.ldS;
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const double x = xj[rw[k]];
                    z0[k] = fma(-x, y0, z0[k]);
                    z1[k] = fma(-x, y1, z1[k]);
                }
            }
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                if (rr + k * tr < rows) {
                    a.Q[row0 + rw[k] + (int64_t)(q0 + qa) * a.ldq] = z0[k];
                    if (qa + 1 < qn) a.Q[row0 + rw[k] + (int64_t)(q0 + qa + 1) * a.ldq] = z1[k];
                }
            }
        }
    }
}

// R X = C for R upper triangular (n x n), C (n x k, leading dimension ldc): one warp per column,
// rows last to first, each row's sum over the solved rows split across the lanes (a fixed
// butterfly).  A zero or non-finite result is noted in the status word.
__global__ void __launch_bounds__(1024) tsqr_trsm_kernel(const double *R, int64_t ldr,
                                                         const double *C, int64_t ldc, double *X,
                                                         int64_t ldx, int n, int k, int *status) {
    const int lane = threadIdx.x & 31;
    const int q = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (q >= k) return;
    double *x = X + (int64_t)q * ldx;
    bool bad = false;
    for (int i = n - 1; i >= 0; --i) {
        double s = 0.0;
        for (int j = i + 1 + lane; j < n; j += 32) s = fma(R[i + (int64_t)j * ldr], x[j], s);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        const double v = (C[i + (int64_t)q * ldc] - s) / R[i + (int64_t)i * ldr];
        if (lane == 0) x[i] = v;
        bad |= !isfinite(v);
        __syncwarp();
    }
    if (bad && lane == 0 && status) atomicOr(status, kStatusNonfiniteBit);
}

namespace {
const void *q_leaf_fn(int blk) {
    switch (blk) {
        case 4: return (const void *)tsqr_q_leaf_kernel<4>;
        case 3: return (const void *)tsqr_q_leaf_kernel<3>;
        case 2: return (const void *)tsqr_q_leaf_kernel<2>;
        default: return (const void *)tsqr_q_leaf_kernel<1>;
    }
}
}  // namespace

// ------------------------------------------------------------------------------------------
// host-side launchers
// ------------------------------------------------------------------------------------------
size_t q_leaf_smem_bytes(int n, int qn, int ldS, int warps) {
    return sizeof(double) * (size_t)q_leaf_layout(n, qn, ldS, warps + 1).total;
}

size_t q_tree_smem_bytes(int n, int arity, int qg) {
    return sizeof(double) * (size_t)arity * n * qg;
}

size_t qt_smem_bytes(int n, int k, int ldS, int warps) {
    return sizeof(double) * (size_t)qt_layout(n, k, ldS, warps + 1).total;
}

cudaError_t qt_prepare(size_t smem_bytes) {
    cudaError_t e = set_smem_attrs(tsqr_qt_kernel<4>, smem_bytes);
    if (e == cudaSuccess) e = set_smem_attrs(tsqr_qt_kernel<3>, smem_bytes);
    if (e == cudaSuccess) e = set_smem_attrs(tsqr_qt_kernel<2>, smem_bytes);
    if (e == cudaSuccess) e = set_smem_attrs(tsqr_qt_kernel<1>, smem_bytes);
    return e;
}

cudaError_t qt_launch(const QtArgs &a, int blk, int warps, size_t smem_bytes,
                      cudaStream_t stream) {
    const dim3 grid(a.nleaves, (a.ktot + a.k - 1) / a.k), block((warps + 1) * 32);
    switch (blk) {
        case 4: tsqr_qt_kernel<4><<<grid, block, smem_bytes, stream>>>(a); break;
        case 3: tsqr_qt_kernel<3><<<grid, block, smem_bytes, stream>>>(a); break;
        case 2: tsqr_qt_kernel<2><<<grid, block, smem_bytes, stream>>>(a); break;
        default: tsqr_qt_kernel<1><<<grid, block, smem_bytes, stream>>>(a); break;
    }
    return cudaGetLastError();
}

size_t q_leaf_wy_smem_bytes(int n, int qn, int ldS, bool fused) {
    return sizeof(double) * (size_t)q_leaf_wy_layout(n, qn, ldS, fused).total;
}

cudaError_t q_leaf_wy_launch(const QLeafArgs &a, size_t smem_bytes, cudaStream_t stream) {
    cudaError_t e = set_smem_attrs(tsqr_q_leaf_wy_kernel, smem_bytes);
    if (e != cudaSuccess) return e;
    tsqr_q_leaf_wy_kernel<<<a.nleaves, 256, smem_bytes, stream>>>(a);
    return cudaGetLastError();
}

size_t wy_smem_bytes(int n, int ldX) {
    return sizeof(double) * ((size_t)ldX * n + 2 * (size_t)n * n);
}

cudaError_t wy_launch(const WyArgs &a, size_t smem_bytes, int grid, cudaStream_t stream) {
    cudaError_t e = set_smem_attrs(tsqr_wy_kernel, smem_bytes);
    if (e != cudaSuccess) return e;
    tsqr_wy_kernel<<<grid, 256, smem_bytes, stream>>>(a);
    return cudaGetLastError();
}

constexpr int kWyThreads = 256;

size_t qt_wy_smem_bytes(int n, int kc, int ldS, bool fused) {
    return sizeof(double) * (size_t)wy_layout(n, kc, ldS, kWyThreads, fused).total;
}

cudaError_t qt_wy_launch(const QtArgs &a, size_t smem_bytes, cudaStream_t stream) {
    cudaError_t e = set_smem_attrs(tsqr_qt_wy_kernel, smem_bytes);
    if (e != cudaSuccess) return e;
    const dim3 grid(a.nleaves, (a.ktot + a.k - 1) / a.k);
    tsqr_qt_wy_kernel<<<grid, kWyThreads, smem_bytes, stream>>>(a);
    return cudaGetLastError();
}

cudaError_t trsm_launch(const double *R, int64_t ldr, const double *C, int64_t ldc, double *X,
                        int64_t ldx, int n, int k, int *status, cudaStream_t stream) {
    const int warps = 8;
    tsqr_trsm_kernel<<<(k + warps - 1) / warps, warps * 32, 0, stream>>>(R, ldr, C, ldc, X, ldx,
                                                                        n, k, status);
    return cudaGetLastError();
}

// leaf_smem / tree_smem = 0: the caller launches no Q pass (the attribute is left alone).
cudaError_t qr_prepare(size_t factor_smem, size_t leaf_smem, size_t tree_smem) {
    for (int b = 1; b <= 4; ++b) {
        cudaError_t e = set_smem_attrs(qr_factor_fn(b), factor_smem);
        if (e != cudaSuccess) return e;
        if (leaf_smem > 0) e = set_smem_attrs(q_leaf_fn(b), leaf_smem);
        if (e != cudaSuccess) return e;
    }
    return tree_smem > 0 ? set_smem_attrs(tsqr_q_tree_kernel, tree_smem) : cudaSuccess;
}

cudaError_t qr_factor_launch(const F64Args &a, int warps, size_t smem_bytes,
                             cudaStream_t stream) {
    const dim3 grid(a.nleaves), block((warps + 1) * 32);
    switch (a.blk) {
        case 4: tsqr_qr_factor_kernel<4><<<grid, block, smem_bytes, stream>>>(a); break;
        case 3: tsqr_qr_factor_kernel<3><<<grid, block, smem_bytes, stream>>>(a); break;
        case 2: tsqr_qr_factor_kernel<2><<<grid, block, smem_bytes, stream>>>(a); break;
        default: tsqr_qr_factor_kernel<1><<<grid, block, smem_bytes, stream>>>(a); break;
    }
    return cudaGetLastError();
}

cudaError_t q_tree_launch(const QTreeArgs &a, int grid, size_t smem_bytes, cudaStream_t stream) {
    tsqr_q_tree_kernel<<<grid, 256, smem_bytes, stream>>>(a);
    return cudaGetLastError();
}

cudaError_t q_leaf_launch(const QLeafArgs &a, int blk, int warps, size_t smem_bytes,
                          cudaStream_t stream) {
    const dim3 grid(a.nleaves), block((warps + 1) * 32);
    switch (blk) {
        case 4: tsqr_q_leaf_kernel<4><<<grid, block, smem_bytes, stream>>>(a); break;
        case 3: tsqr_q_leaf_kernel<3><<<grid, block, smem_bytes, stream>>>(a); break;
        case 2: tsqr_q_leaf_kernel<2><<<grid, block, smem_bytes, stream>>>(a); break;
        default: tsqr_q_leaf_kernel<1><<<grid, block, smem_bytes, stream>>>(a); break;
    }
    return cudaGetLastError();
}

}  // namespace tsqr
