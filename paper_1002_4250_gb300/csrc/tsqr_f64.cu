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
//   kTri == false (leaf): S is a dense chunk of hs rows; warp w owns rows [w*hs/W, (w+1)*hs/W).
//   kTri == true  (tree operator, Table 3): S is the upper triangle R2, so the support of
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
//                   per lane; a lane writes one partial per column its run touches into slot
//                   (lane + column) -- slot ids are distinct and ordered along the items;
//   barrier; warp 0 sums the partials in a fixed order, forms reflector J, updates row J of
//   R and publishes f[k] for k > J; barrier.
// In leaf mode, columns that are no longer read (J-2 at step J) receive the next chunk of
// rows by cp.async while the fold goes on.
// ------------------------------------------------------------------------------------------
template <bool kTri>
__device__ __forceinline__ void fold(double *__restrict__ S, const int ldS, const int hs,
                                     double *__restrict__ Rp, double *__restrict__ f,
                                     double *__restrict__ seg_all, double *__restrict__ tot,
                                     double *__restrict__ npart, const int n,
                                     const Prefetch pf) {
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int W = blockDim.x >> 5;
    const int Hw = hs / W;
    double *seg = seg_all + warp * kSegStride;

    for (int J = 0; J < n; ++J) {
        if (!kTri && pf.src && J >= 2) prefetch_column(S, ldS, hs, pf, J - 2);
        const int U = n - J - 1;
        double *SJ = S + (size_t)J * ldS;
        const double *Sj = S + (size_t)(J > 0 ? J - 1 : 0) * ldS;
        int r0, cw, kc0, kc1;
        if (kTri) {
            r0 = 0;
            cw = J + 1;
            kc0 = (warp * U) / W;
            kc1 = ((warp + 1) * U) / W;
        } else {
            r0 = warp * Hw;
            cw = Hw;
            kc0 = 0;
            kc1 = U;
        }

        // ---- A: column J gets reflector J-1; per-lane partial squared norm of column J
        double nacc = 0.0;
        if (!kTri || warp == 0) {
            if (J > 0) {
                const double fJ = f[J];
                for (int i = lane; i < cw; i += 32) {
                    const double s = fma(-fJ, Sj[r0 + i], SJ[r0 + i]);
                    SJ[r0 + i] = s;
                    nacc = fma(s, s, nacc);
                }
            } else {
                for (int i = lane; i < cw; i += 32) {
                    const double s = SJ[r0 + i];
                    nacc = fma(s, s, nacc);
                }
            }
        }
        npart[warp * 32 + lane] = nacc;
        for (int id = lane; id < 32 + U; id += 32) seg[id] = 0.0;
        if (kTri)
            __syncthreads();
        else
            __syncwarp();

        // ---- B: fused update by reflector J-1 and dots with column J, one column segment
        //      of the lane's run at a time
        const int N = (kc1 - kc0) * cw;
        if (N > 0) {
            int p = (int)(((long long)lane * N) >> 5);
            const int pend = (int)(((long long)(lane + 1) * N) >> 5);
            int kk = p / cw;
            int i = p - kk * cw;
            while (p < pend) {
                const int len = min(cw - i, pend - p);
                const int k = J + 1 + kc0 + kk;
                // distinct columns of S: the three never overlap
                double *__restrict__ Sk = S + (size_t)k * ldS + r0 + i;
                const double *__restrict__ a = Sj + r0 + i;
                const double *__restrict__ b = SJ + r0 + i;
                double acc = 0.0;
                if (J > 0) {
                    const double fk = f[k];
#pragma unroll 4
                    for (int t = 0; t < len; ++t) {
                        const double s = fma(-fk, a[t], Sk[t]);
                        Sk[t] = s;
                        acc = fma(b[t], s, acc);
                    }
                } else {
#pragma unroll 4
                    for (int t = 0; t < len; ++t) acc = fma(b[t], Sk[t], acc);
                }
                seg[lane + kk] = acc;
                p += len;
                i = 0;
                ++kk;
            }
        }
        __syncthreads();

        // ---- reducer: reflector J, row J of R, factors f[k] for k > J
        if (warp == 0) {
            double v = npart[lane];
            for (int w = 1; w < W; ++w) v += npart[w * 32 + lane];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
            const double sig2 = __shfl_sync(0xffffffffu, v, 0);
            if (!kTri && W > 1) {
                for (int id = lane; id < 32 + U; id += 32) {
                    double t = seg_all[id];
                    for (int w = 1; w < W; ++w) t += seg_all[w * kSegStride + id];
                    tot[id] = t;
                }
                __syncwarp();
            }
            const double *totp = (!kTri && W > 1) ? tot : seg_all;
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
                double d;
                if (!kTri) {
                    const int Nw = U * Hw;
                    const int la = (32 * (kk * Hw + 1) - 1) / Nw;
                    const int lb = (32 * (kk + 1) * Hw - 1) / Nw;
                    d = totp[kk + la];
                    for (int l = la + 1; l <= lb; ++l) d += totp[kk + l];
                } else {
                    d = 0.0;
                    bool first = true;
                    for (int w = 0; w < W; ++w) {
                        const int a0 = (w * U) / W, a1 = ((w + 1) * U) / W;
                        if (kk < a0 || kk >= a1) continue;
                        const int rel = kk - a0;
                        const int Nw = (a1 - a0) * (J + 1);
                        const int la = (32 * (rel * (J + 1) + 1) - 1) / Nw;
                        const int lb = (32 * (rel + 1) * (J + 1) - 1) / Nw;
                        for (int l = la; l <= lb; ++l) {
                            const double x = seg_all[w * kSegStride + rel + l];
                            d = first ? x : d + x;
                            first = false;
                        }
                    }
                }
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
        __syncthreads();
    }
    if (!kTri && pf.src) {
        for (int col = n - 2; col < n; ++col)
            if (col >= 0) prefetch_column(S, ldS, hs, pf, col);
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
__global__ void __launch_bounds__(256) tsqr_f64_kernel(const F64Args a) {
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
        fold<false>(S, a.ldS, a.hs, Rp, f, seg, tot, npart, n, next);
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
        fold<true>(S, a.ldS, a.hs, Rp, f, seg, tot, npart, n, Prefetch{nullptr, 0, 0});
        ++level;
        t >>= 1;
    }
}

// One tree node: R = qr(R1, R2) (Table 3), optionally sign-normalized.
__global__ void __launch_bounds__(256) tsqr_f64_combine_kernel(int n, const double *R1, int64_t ld1,
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
    fold<true>(S, ldS, hs, Rp, smem + L.f, smem + L.seg, smem + L.tot, smem + L.npart, n,
               Prefetch{nullptr, 0, 0});
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
