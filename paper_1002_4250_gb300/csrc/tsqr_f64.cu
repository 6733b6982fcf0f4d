// FP64 kernels of libtsqr: the leaf/tree kernel of TSQR (Section 2 with the trees of
// Section 1 and Fig. 1) and a single-node kernel for the operator qr(R1, R2) of Table 3.
#include "tsqr_f64.cuh"
#include "tsqr_internal.h"

namespace tsqr {

// ------------------------------------------------------------------------------------------
// Asynchronous global -> shared copies (cp.async, 8 bytes each; src_bytes = 0 zero-fills).
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ void cp_async8(double *smem_dst, const double *gsrc, int src_bytes) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(d), "l"(gsrc),
                 "r"(src_bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// The next chunk of rows a leaf will fold (src == nullptr: none).
struct Prefetch {
    const double *src;  // row 0, column 0 of the chunk in A
    int64_t lda;
    int rows;           // rows of A in the chunk; the rest of the hs rows of S are zero-filled
};

// Start copying column `col` of the next chunk into column `col` of S.
__device__ __forceinline__ void prefetch_column(double *S, int ldS, int hs, const Prefetch pf,
                                                int col) {
    const double *src = pf.src + (int64_t)col * pf.lda;
    double *dst = S + (size_t)col * ldS;
    for (int i = threadIdx.x; i < hs; i += blockDim.x) {
        const bool ok = i < pf.rows;
        cp_async8(dst + i, ok ? src + i : pf.src, ok ? 8 : 0);
    }
    cp_async_commit();
}

// ------------------------------------------------------------------------------------------
// R <- R([R; S]) in shared memory, one Householder reflector per column J = 0..n-1.
//
// Rp: the top block R, packed upper triangle (row J at rowoff(n, J)).
// S : the bottom block, column-major with leading dimension ldS.
//   leaf (fold_leaf): S is a dense chunk of hs rows; warp w owns rows [w*Hw, (w+1)*Hw),
//     Hw = hs / W = 32 r.
//   tree operator (fold_tri, Table 3): S is the upper triangle R2, so the support of
//     reflector J in S is rows 0..J (the j+2-entry reflector of the paper's operator);
//     the warps split the trailing columns instead of the rows.
//
// Reflector J (the LAPACK dlarfg rule the paper's operator uses): alpha = R(J,J), x = the
// support of column J in S, sigma^2 = ||x||^2.  If sigma^2 == 0 it is the identity (the
// paper's tau == 0 skip).  Otherwise beta = -sign(alpha) sqrt(alpha^2 + sigma^2) with
// sign(0) = +1, tau = (beta - alpha) / beta and v = x / (alpha - beta).  S keeps x unscaled;
// for each trailing column k, with d_k = x . S(:,k):
//   w_k = R(J,k) + d_k / (alpha - beta),   R(J,k) -= tau w_k,   S(:,k) -= f_k x,
//   f_k = tau w_k / (alpha - beta) = -w_k / beta.
// 1/sqrt(alpha^2 + sigma^2) gives both |beta| and 1/beta; 1/(alpha - beta) is the one
// reciprocal (alpha - beta has the sign of alpha and magnitude >= |beta|: no cancellation).
//
// Each step J does:
//   A  (per warp)   column J gets reflector J-1 (f[J]); per-lane partial ||column J||^2;
//   B  (per warp)   every other trailing column k > J gets reflector J-1 and, in the same
//                   sweep, its partial dot product with column J.  The warp's (column, row)
//                   items are cut into 32 equal contiguous runs in column-major order, one
//                   per lane, processed in lockstep; a lane writes one partial per column its
//                   run touches into slot (lane + column) -- slot ids are distinct and
//                   ordered along the items;
//   barrier; warp J mod W sums the partials in a fixed order, forms reflector J, updates row
//   J of R and publishes f[k] for k > J; barrier.
// ------------------------------------------------------------------------------------------

// The reducer warp's part of step J.  npart holds W x 32 per-lane partial squared norms; dk[kk] the
// summed dot product of column J+1+kk with column J (written by the same warp).
__device__ __forceinline__ void reflect(const int lane, const int W, const int n, const int J,
                                        double *__restrict__ Rp, double *__restrict__ f,
                                        const double *__restrict__ npart,
                                        const double *__restrict__ dk) {
    const int U = n - J - 1;
    double v = npart[lane];
    for (int w = 1; w < W; ++w) v += npart[w * 32 + lane];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const double sig2 = __shfl_sync(0xffffffffu, v, 0);
    const int ro = rowoff(n, J);
    const double alpha = Rp[ro];
    // identity reflector only for an exactly zero tail; NaN/Inf propagate into R
    const bool ident = (sig2 == 0.0);
    double beta = alpha, tau = 0.0, c = 0.0, ib = 0.0;
    if (!ident) {
        const double t = fma(alpha, alpha, sig2);
        const double y = rsqrt(t);
        const double r = t * y;
        beta = (alpha >= 0.0) ? -r : r;
        ib = (alpha >= 0.0) ? -y : y;
        tau = fma(-alpha, ib, 1.0);
        c = __drcp_rn(alpha - beta);
    }
    for (int kk = lane; kk < U; kk += 32) {
        const int k = J + 1 + kk;
        const double d = dk[kk];
        const int idx = ro + 1 + kk;
        if (ident) {
            f[k] = 0.0;
        } else {
            const double rjk = Rp[idx];
            const double wk = fma(c, d, rjk);
            Rp[idx] = fma(-tau, wk, rjk);
            f[k] = -wk * ib;
        }
    }
    if (lane == 0) Rp[ro] = beta;
}

// Leaf fold.  Every lane owns r rows of its warp's block (Hw = 32 r) and a phase-B run of
// U r items starting at item lane * U r; runs and column boundaries are multiples of r, so
// blocks of B items (B divides r) never straddle a column: the inner loop has no per-item
// bookkeeping and all lanes stay in lockstep.  The next chunk of rows streams into columns
// no longer read (J-2 at step J) by cp.async.
template <int B>
__device__ __forceinline__ void fold_leaf(double *__restrict__ S, const int ldS, const int hs,
                                          double *__restrict__ Rp, double *__restrict__ f,
                                          double *__restrict__ seg_all, double *__restrict__ tot,
                                          double *__restrict__ npart, const int n,
                                          const Prefetch pf) {
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int W = blockDim.x >> 5;
    const int Hw = hs / W;
    const int r = Hw >> 5;
    const int r0 = warp * Hw;
    double *seg = seg_all + warp * kSegStride;

    for (int J = 0; J < n; ++J) {
        if (pf.src && J >= 2) prefetch_column(S, ldS, hs, pf, J - 2);
        const int U = n - J - 1;
        double *SJ = S + (size_t)J * ldS + r0;
        const double *Sj = S + (size_t)(J > 0 ? J - 1 : 0) * ldS + r0;

        // ---- A: column J gets reflector J-1; per-lane partial squared norm of column J
        double nacc = 0.0;
        if (J > 0) {
            const double fJ = f[J];
            for (int t = 0; t < r; ++t) {
                const int i = lane + 32 * t;
                const double s = fma(-fJ, Sj[i], SJ[i]);
                SJ[i] = s;
                nacc = fma(s, s, nacc);
            }
        } else {
            for (int t = 0; t < r; ++t) {
                const double s = SJ[lane + 32 * t];
                nacc = fma(s, s, nacc);
            }
        }
        npart[warp * 32 + lane] = nacc;
        for (int id = lane; id < 32 + U; id += 32) seg[id] = 0.0;
        __syncwarp();

        // ---- B: fused update by reflector J-1 and dots with column J
        if (U > 0) {
            const int run = U * r;
            const int p = lane * run;
            int kk = p / Hw;
            int i = p - kk * Hw;
            double *Sk = S + (size_t)(J + 1 + kk) * ldS + r0;
            double acc = 0.0;
            if (J > 0) {
                double fk = f[J + 1 + kk];
                for (int blk = 0; blk < run; blk += B) {
                    double x[B];
#pragma unroll
                    for (int q = 0; q < B; ++q) x[q] = fma(-fk, Sj[i + q], Sk[i + q]);
#pragma unroll
                    for (int q = 0; q < B; ++q) Sk[i + q] = x[q];
#pragma unroll
                    for (int q = 0; q < B; ++q) acc = fma(SJ[i + q], x[q], acc);
                    i += B;
                    if (i == Hw) {
                        seg[lane + kk] = acc;
                        acc = 0.0;
                        i = 0;
                        ++kk;
                        Sk += ldS;
                        fk = f[min(J + 1 + kk, n - 1)];
                    }
                }
            } else {
                for (int blk = 0; blk < run; blk += B) {
#pragma unroll
                    for (int q = 0; q < B; ++q) acc = fma(SJ[i + q], Sk[i + q], acc);
                    i += B;
                    if (i == Hw) {
                        seg[lane + kk] = acc;
                        acc = 0.0;
                        i = 0;
                        ++kk;
                        Sk += ldS;
                    }
                }
            }
            if (i != 0) seg[lane + kk] = acc;
        }
        __syncthreads();

        // ---- reducer (warp J mod W: the serial FP64 work visits every sub-partition in turn)
        if (warp == J % W) {
            for (int id = lane; id < 32 + U; id += 32) {
                double t = seg_all[id];
                for (int w = 1; w < W; ++w) t += seg_all[w * kSegStride + id];
                tot[id] = t;
            }
            __syncwarp();
            const int Nw = U * Hw;
            double *dk = tot + kSegStride;
            for (int kk = lane; kk < U; kk += 32) {
                const int la = (32 * (kk * Hw + 1) - 1) / Nw;
                const int lb = (32 * (kk + 1) * Hw - 1) / Nw;
                double d = tot[kk + la];
                for (int l = la + 1; l <= lb; ++l) d += tot[kk + l];
                dk[kk] = d;
            }
            __syncwarp();
            reflect(lane, W, n, J, Rp, f, npart, dk);
        }
        __syncthreads();
    }
    if (pf.src) {
        for (int col = n - 2; col < n; ++col)
            if (col >= 0) prefetch_column(S, ldS, hs, pf, col);
    }
}

// Tree-operator fold (Table 3): S = R2, reflector J's support in S is rows 0..J.  Warp 0
// updates column J; the warps split the trailing columns, each lane taking an equal
// contiguous run of the warp's (column, row) items in lockstep.
__device__ __forceinline__ void fold_tri(double *__restrict__ S, const int ldS,
                                         double *__restrict__ Rp, double *__restrict__ f,
                                         double *__restrict__ seg_all,
                                         double *__restrict__ npart, const int n) {
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int W = blockDim.x >> 5;
    double *seg = seg_all + warp * kSegStride;

    for (int J = 0; J < n; ++J) {
        const int U = n - J - 1;
        const int cw = J + 1;
        double *SJ = S + (size_t)J * ldS;
        const double *Sj = S + (size_t)(J > 0 ? J - 1 : 0) * ldS;
        const int kc0 = (warp * U) / W, kc1 = ((warp + 1) * U) / W;

        double nacc = 0.0;
        if (warp == 0) {
            const double fJ = (J > 0) ? f[J] : 0.0;
            for (int i = lane; i < cw; i += 32) {
                double s = SJ[i];
                if (J > 0) {
                    s = fma(-fJ, Sj[i], s);
                    SJ[i] = s;
                }
                nacc = fma(s, s, nacc);
            }
        }
        npart[warp * 32 + lane] = nacc;
        for (int id = lane; id < 32 + U; id += 32) seg[id] = 0.0;
        __syncthreads();

        const int N = (kc1 - kc0) * cw;
        if (N > 0) {
            int p = (int)(((long long)lane * N) >> 5);
            const int pend = (int)(((long long)(lane + 1) * N) >> 5);
            if (p < pend) {
                int kk = p / cw;
                int i = p - kk * cw;
                int k = J + 1 + kc0 + kk;
                double *Sk = S + (size_t)k * ldS;
                double fk = (J > 0) ? f[k] : 0.0;
                double acc = 0.0;
                for (;;) {
                    double s = Sk[i];
                    if (J > 0) {
                        s = fma(-fk, Sj[i], s);
                        Sk[i] = s;
                    }
                    acc = fma(SJ[i], s, acc);
                    if (++p == pend) break;
                    if (++i == cw) {
                        seg[lane + kk] = acc;
                        acc = 0.0;
                        i = 0;
                        ++kk;
                        ++k;
                        Sk += ldS;
                        fk = (J > 0) ? f[k] : 0.0;
                    }
                }
                seg[lane + kk] = acc;
            }
        }
        __syncthreads();

        if (warp == J % W) {
            double *dk = seg_all + W * kSegStride + kSegStride;
            for (int kk = lane; kk < U; kk += 32) {
                double d = 0.0;
                bool first = true;
                for (int w = 0; w < W; ++w) {
                    const int a0 = (w * U) / W, a1 = ((w + 1) * U) / W;
                    if (kk < a0 || kk >= a1) continue;
                    const int rel = kk - a0;
                    const int Nw = (a1 - a0) * cw;
                    const int la = (32 * (rel * cw + 1) - 1) / Nw;
                    const int lb = (32 * (rel + 1) * cw - 1) / Nw;
                    for (int l = la; l <= lb; ++l) {
                        const double x = seg_all[w * kSegStride + rel + l];
                        d = first ? x : d + x;
                        first = false;
                    }
                }
                dk[kk] = d;
            }
            __syncwarp();
            reflect(lane, W, n, J, Rp, f, npart, dk);
        }
        __syncthreads();
    }
}

// Packed upper triangle (smem) -> column-major n x n (global), zeros below the diagonal.
__device__ __forceinline__ void store_packed(const double *__restrict__ Rp, int n,
                                             double *__restrict__ dst, int64_t ld) {
    for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
        const int col = idx / n, row = idx - col * n;
        dst[row + (int64_t)col * ld] = (row <= col) ? Rp[rowoff(n, row) + col - row] : 0.0;
    }
}

// Column-major global (L2, bypassing L1) -> packed upper triangle in smem.
__device__ __forceinline__ void load_packed_cg(const double *src, int64_t ld, int n,
                                               double *__restrict__ Rp) {
    for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
        const int col = idx / n, row = idx - col * n;
        if (row <= col) Rp[rowoff(n, row) + col - row] = __ldcg(src + row + (int64_t)col * ld);
    }
}

// Column-major global -> S (upper triangle kept, strict lower part stored as zero).
__device__ __forceinline__ void load_tri_cg(const double *src, int64_t ld, int n,
                                            double *__restrict__ S, int ldS) {
    for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
        const int col = idx / n, row = idx - col * n;
        S[row + col * ldS] = (row <= col) ? __ldcg(src + row + (int64_t)col * ld) : 0.0;
    }
}

// Root: rows flipped so that diag(R) >= 0 (Section 2), strict lower part zero, NaN/Inf noted.
__device__ __forceinline__ void store_normalized(const double *__restrict__ Rp, int n,
                                                 double *__restrict__ R, int64_t ldr,
                                                 int *status) {
    bool bad = false;
    for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
        const int col = idx / n, row = idx - col * n;
        double v = 0.0;
        if (row <= col) {
            v = Rp[rowoff(n, row) + col - row];
            if (Rp[rowoff(n, row)] < 0.0) v = -v;
            bad |= !isfinite(v);
        }
        R[row + (int64_t)col * ldr] = v;
    }
    if (bad && status) atomicOr(status, kStatusNonfiniteBit);
}

// ------------------------------------------------------------------------------------------
// Leaf + tree kernel.  CTA c owns the work units [c*nunits/nleaves, (c+1)*nunits/nleaves) of A
// (one tile for the binary tree, a run of slabs for the flat and hybrid trees) and folds their
// rows, h at a time, into its R (a flat tree over its chunks, Section 1, with the next chunk
// streamed in by cp.async during the current fold), then climbs the binary tree (Fig. 1): it
// publishes R in its node's slot and bumps the parent's counter; the second child to arrive
// combines [R_left; R_right] (left = lower index, always on top) and climbs on; the first
// returns.  No CTA ever waits for another, and the operand order depends only on the indices.
// ------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(256, 1) tsqr_f64_kernel(const F64Args a) {
    extern __shared__ __align__(16) double smem[];
    const int n = a.n;
    const SmemLayout L = smem_layout(n, a.hs, a.ldS, blockDim.x >> 5);
    double *S = smem + L.S;
    double *Rp = smem + L.Rp;
    double *f = smem + L.f;
    double *seg = smem + L.seg;
    double *tot = smem + L.tot;
    double *npart = smem + L.npart;
    unsigned int *flag = reinterpret_cast<unsigned int *>(smem + L.scal);

    const int leaf = blockIdx.x;
    for (int i = threadIdx.x; i < n * (n + 1) / 2; i += blockDim.x) Rp[i] = 0.0;

    // rows of this leaf, folded in chunks of h rows
    const int64_t u0 = ((int64_t)leaf * a.nunits) / a.nleaves;
    const int64_t u1 = ((int64_t)(leaf + 1) * a.nunits) / a.nleaves;
    const int64_t rbeg = u0 * a.unit;
    const int64_t rend = (u1 * a.unit < a.m) ? u1 * a.unit : a.m;
    const int64_t nchunks = (rend - rbeg + a.h - 1) / a.h;
    if (nchunks > 0) {
        Prefetch first;
        first.src = a.A + rbeg;
        first.lda = a.lda;
        first.rows = (int)((rend - rbeg < a.h) ? rend - rbeg : a.h);
        for (int col = 0; col < n; ++col) prefetch_column(S, a.ldS, a.hs, first, col);
        cp_async_wait_all();
        __syncthreads();
    }
    for (int64_t c = 0; c < nchunks; ++c) {
        Prefetch next;
        next.src = nullptr;
        next.lda = a.lda;
        next.rows = 0;
        if (c + 1 < nchunks) {
            const int64_t r1 = rbeg + (c + 1) * a.h;
            next.src = a.A + r1;
            next.rows = (int)((rend - r1 < a.h) ? rend - r1 : a.h);
        }
        switch (a.blk) {
            case 4: fold_leaf<4>(S, a.ldS, a.hs, Rp, f, seg, tot, npart, n, next); break;
            case 3: fold_leaf<3>(S, a.ldS, a.hs, Rp, f, seg, tot, npart, n, next); break;
            case 2: fold_leaf<2>(S, a.ldS, a.hs, Rp, f, seg, tot, npart, n, next); break;
            default: fold_leaf<1>(S, a.ldS, a.hs, Rp, f, seg, tot, npart, n, next); break;
        }
        if (next.src) {
            cp_async_wait_all();
            __syncthreads();
        }
    }

    int level = 0, t = leaf;
    for (;;) {
        const int cnt = a.tree.count[level];
        if (cnt == 1) {
            store_normalized(Rp, n, a.R, a.ldr, a.status);
            return;
        }
        const int sib = t ^ 1;
        if (sib >= cnt) {  // odd last node: promoted unchanged
            ++level;
            t >>= 1;
            continue;
        }
        double *mine = a.slots + (size_t)(a.tree.offset[level] + t) * n * n;
        store_packed(Rp, n, mine, n);
        __threadfence();
        __syncthreads();
        if (threadIdx.x == 0)
            flag[0] = atomicAdd(&a.counters[a.tree.offset[level + 1] + (t >> 1)], 1u);
        __syncthreads();
        if (flag[0] == 0) return;  // the sibling combines
        __threadfence();
        const double *other = a.slots + (size_t)(a.tree.offset[level] + sib) * n * n;
        if (t & 1) {
            // this CTA holds the right (lower) operand: it becomes S, the left one comes to Rp
            for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
                const int col = idx / n, row = idx - col * n;
                S[row + col * a.ldS] = (row <= col) ? Rp[rowoff(n, row) + col - row] : 0.0;
            }
            __syncthreads();
            load_packed_cg(other, n, n, Rp);
        } else {
            load_tri_cg(other, n, n, S, a.ldS);
        }
        __syncthreads();
        fold_tri(S, a.ldS, Rp, f, seg, npart, n);
        ++level;
        t >>= 1;
    }
}

// One tree node: R = qr(R1, R2) (Table 3), optionally sign-normalized.
__global__ void __launch_bounds__(256, 1) tsqr_f64_combine_kernel(int n, const double *R1, int64_t ld1,
                                                               const double *R2, int64_t ld2,
                                                               double *R, int64_t ldr,
                                                               int normalize, int ldS, int hs,
                                                               int *status) {
    extern __shared__ __align__(16) double smem[];
    const SmemLayout L = smem_layout(n, hs, ldS, blockDim.x >> 5);
    double *S = smem + L.S;
    double *Rp = smem + L.Rp;
    load_packed_cg(R1, ld1, n, Rp);
    load_tri_cg(R2, ld2, n, S, ldS);
    __syncthreads();
    fold_tri(S, ldS, Rp, smem + L.f, smem + L.seg, smem + L.npart, n);
    if (normalize)
        store_normalized(Rp, n, R, ldr, status);
    else
        store_packed(Rp, n, R, ldr);
}

// ------------------------------------------------------------------------------------------
// host-side launchers
// ------------------------------------------------------------------------------------------
size_t f64_smem_bytes(int n, int hs, int ldS, int warps) {
    return sizeof(double) * (size_t)smem_layout(n, hs, ldS, warps).total;
}

cudaError_t f64_prepare(size_t smem_bytes) {
    cudaError_t e = cudaFuncSetAttribute(tsqr_f64_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem_bytes);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(tsqr_f64_combine_kernel,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes);
}

int f64_blocks_per_sm(int warps, size_t smem_bytes) {
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, tsqr_f64_kernel, warps * 32,
                                                      smem_bytes) != cudaSuccess)
        return 0;
    return nb;
}

cudaError_t f64_launch(const F64Args &a, int warps, size_t smem_bytes, cudaStream_t stream) {
    tsqr_f64_kernel<<<a.nleaves, warps * 32, smem_bytes, stream>>>(a);
    return cudaGetLastError();
}

cudaError_t f64_combine_launch(int n, const double *R1, int64_t ld1, const double *R2,
                               int64_t ld2, double *R, int64_t ldr, int normalize, int warps,
                               int ldS, int hs, size_t smem_bytes, int *status,
                               cudaStream_t stream) {
    tsqr_f64_combine_kernel<<<1, warps * 32, smem_bytes, stream>>>(n, R1, ld1, R2, ld2, R, ldr,
                                                                  normalize, ldS, hs, status);
    return cudaGetLastError();
}

}  // namespace tsqr
