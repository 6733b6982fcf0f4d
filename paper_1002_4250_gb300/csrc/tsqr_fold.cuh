// Device code shared by libtsqr's kernels: the shared-memory fold R <- R([R; S]) that serves
// both as the leaf (S = a chunk of rows of A, Section 2 step 1 fused with a flat tree,
// Section 1) and as the tree operator qr(R1, R2) (S = R2, an upper triangle; Section 2,
// Table 3), and the body of the leaf + binary-tree kernel (Fig. 1) with the "last child to
// arrive combines" rule.
//
// Cost model this is written for (measured on GB300): one warp-wide FP64 instruction occupies a
// sub-partition's FP64 unit for ~64 cycles whether 1 or 32 lanes are active, FP64 latency is
// ~65 cycles, sqrt ~620 and divide ~375 cycles; shared-memory traffic, integer work, shuffles
// and barriers are nearly free by comparison.  Hence the bulk pass spreads its (row, column)
// items evenly over all 32 lanes in lockstep, fuses the update by reflector j with the dot
// products for reflector j+1, sums partials along fixed index orders (bit-reproducible), and
// does the per-column scalar work once per CTA on one warp.
#pragma once

#include <cuda_bf16.h>
#include <type_traits>

#include "tsqr_f64.cuh"
#include "tsqr_internal.h"

namespace tsqr {

// ------------------------------------------------------------------------------------------
// Asynchronous global -> shared copies (cp.async of 8 or 4 bytes; src_bytes = 0 zero-fills).
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ void cp_async8(void *smem_dst, const void *gsrc, int src_bytes) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(d), "l"(gsrc),
                 "r"(src_bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_async4(void *smem_dst, const void *gsrc, int src_bytes) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(d), "l"(gsrc),
                 "r"(src_bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// A chunk of rows of A (src == nullptr: none).
template <typename Tin>
struct Chunk {
    const Tin *src;  // row 0, column 0 of the chunk in A
    int64_t lda;
    int rows;        // rows of A in the chunk; the rest of the hs rows of S are zero-filled
};

// Element types: T is the leaf's storage and arithmetic type in shared memory, Tin the type
// of A in global memory.  Same type: copied by cp.async.  BF16 -> FP32: widened (exactly)
// through registers.
template <typename T, typename Tin>
struct Copy {
    static constexpr bool kAsync = sizeof(T) == sizeof(Tin);
};

__device__ __forceinline__ float widen(__nv_bfloat16 x) { return __bfloat162float(x); }
__device__ __forceinline__ double fmat(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float fmat(float a, float b, float c) { return fmaf(a, b, c); }

// Copy column `col` of the chunk into column `col` of S (asynchronously when the types agree).
template <typename T, typename Tin>
__device__ __forceinline__ void load_column(T *S, int ldS, int hs, const Chunk<Tin> c, int col) {
    const Tin *src = c.src + (int64_t)col * c.lda;
    T *dst = S + (size_t)col * ldS;
    if constexpr (Copy<T, Tin>::kAsync) {
        for (int i = threadIdx.x; i < hs; i += blockDim.x) {
            const bool ok = i < c.rows;
            if constexpr (sizeof(T) == 8)
                cp_async8(dst + i, ok ? (const void *)(src + i) : (const void *)c.src, ok ? 8 : 0);
            else
                cp_async4(dst + i, ok ? (const void *)(src + i) : (const void *)c.src, ok ? 4 : 0);
        }
        cp_async_commit();
    } else {
        for (int i = threadIdx.x; i < hs; i += blockDim.x)
            dst[i] = (i < c.rows) ? (T)widen(src[i]) : (T)0;
    }
}

// ------------------------------------------------------------------------------------------
// R <- R([R; S]) in shared memory, one Householder reflector per column J = 0..n-1.
//
// Rp: the top block R, packed upper triangle (row J at rowoff(n, J)).
// S : the bottom block, column-major with leading dimension ldS.
//   leaf (fold_leaf): S is a dense chunk of hs rows; warp w owns rows [w*Hw, (w+1)*Hw),
//     Hw = hs / W = 32 r.
//   tree operator (fold_stack, Table 3): S holds c stacked upper triangles (c = 1 is the
//     paper's R2), so the support of reflector J in S is rows 0..J of each triangle (the
//     j+2-entry reflector of the paper's operator for c = 1); the warps split the trailing
//     columns instead of the rows.
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
//   then one warp sums the partials in a fixed order, forms reflector J, updates row J of R
//   and publishes f[k] for k > J (in the leaf a dedicated reducer warp, whose scalar work
//   overlaps phase B; in the tree operator warp J mod W).
// ------------------------------------------------------------------------------------------

// Conversions between a double x with 1 <= |x| < 4 and float, on the IEEE-754 bit fields with
// integer instructions: double <-> float conversions issue to the FP64 unit, whose every
// instruction the reducer pays for.  Toward zero to float (the top 23 fraction bits; the seeds
// below need ~2^-20 only); exact back to double.
__device__ __forceinline__ float seed_f32(const double x) {
    const long long b = __double_as_longlong(x);
    const unsigned sign = (unsigned)((unsigned long long)b >> 63) << 31;
    const int e = (int)((b >> 52) & 0x7ff) - 1023 + 127;
    const unsigned frac = (unsigned)((b >> 29) & 0x7fffff);
    return __uint_as_float(sign | ((unsigned)e << 23) | frac);
}
// y a normal float
__device__ __forceinline__ double widen_f32(const float y) {
    const unsigned u = __float_as_uint(y);
    const long long sign = (long long)(u >> 31) << 63;
    const long long e = (long long)((u >> 23) & 0xff) - 127 + 1023;
    return __longlong_as_double(sign | (e << 52) | ((long long)(u & 0x7fffff) << 29));
}

// 1/sqrt(t) for finite t > 0 from the FP32 hardware estimate y by one third-order step of the
// series (1 - h)^(-1/2) = 1 + h/2 + 3h^2/8 + ..., h = 1 - t y^2: y (1 + h/2 + 3h^2/8), whose
// error is about 5|h|^3/16, below FP64 rounding for the estimate's ~2^-22 (four dependent FP64
// operations, against six for two Newton steps: each costs about 65 cycles on the reflector's
// serial chain).  t is first scaled by an even power of two into [1, 4) (exact, on the exponent
// bits) so that the FP32 estimate cannot overflow or underflow.  Zero, subnormal, infinite and
// NaN arguments take the library's rsqrt.
__device__ __forceinline__ double recip_sqrt(double t) {
    const long long b = __double_as_longlong(t);
    const int e = (int)((b >> 52) & 0x7ff);
    if (e == 0 || e == 0x7ff) return rsqrt(t);
    const int k = (e - 1023) >> 1;  // t = tm 4^k, tm in [1, 4)
    const double tm = __longlong_as_double(b - ((long long)(2 * k) << 52));
    const double y = widen_f32(rsqrtf(seed_f32(tm)));
    const double h = fma(-tm * y, y, 1.0);
    const double yh = y * h, p = fma(h, 0.375, 0.5);  // independent: one level
    const double y1 = fma(yh, p, y);
    return __longlong_as_double(__double_as_longlong(y1) - ((long long)k << 52));  // y1 2^-k
}

// 1/x for finite nonzero x from the FP32 estimate y of 1/xm, x = xm 2^k, |xm| in [1, 2) (exact
// rescaling), by one third-order step y (1 + h + h^2) = y + (y h)(1 + h), h = 1 - xm y (error
// |h|^3; three dependent FP64 operations, against four for two Newton steps).  Zero,
// subnormal, infinite and NaN arguments, and |x| >= 2^1022 (whose reciprocal is subnormal),
// divide.
__device__ __forceinline__ double recip(double x) {
    const long long b = __double_as_longlong(x);
    const int e = (int)((b >> 52) & 0x7ff);
    if (e == 0 || e >= 0x7fd) return 1.0 / x;
    const int k = e - 1023;
    const double xm = __longlong_as_double(b - ((long long)k << 52));
    const double y = widen_f32(__fdividef(1.0f, seed_f32(xm)));
    const double h = fma(-xm, y, 1.0);
    const double yh = y * h, q = 1.0 + h;  // independent: one level
    const double y1 = fma(yh, q, y);
    return __longlong_as_double(__double_as_longlong(y1) - ((long long)k << 52));
}

// Reflector J's scalars from alpha = R(J,J) and sigma^2 (see the comment above).
struct Reflector {
    double beta, tau, c, ib;
    bool ident;
};

__device__ __forceinline__ Reflector make_reflector(const double alpha, const double sig2) {
    Reflector h;
    // identity reflector only for an exactly zero tail; NaN/Inf propagate into R
    h.ident = (sig2 == 0.0);
    h.beta = alpha;
    h.tau = 0.0;
    h.c = 0.0;
    h.ib = 0.0;
    if (!h.ident) {
        const double t = fma(alpha, alpha, sig2);
        const double y = recip_sqrt(t);
        const double r = t * y;
        const bool pos = alpha >= 0.0;
        h.beta = pos ? -r : r;
        h.ib = pos ? -y : y;
        h.tau = fma(-alpha, h.ib, 1.0);
        h.c = recip(alpha - h.beta);
    }
    return h;
}

// sigma^2 from W x 32 per-lane partials, summed in a fixed order (same value in every lane).
__device__ __forceinline__ double sum_norm_partials(const int lane, const int W,
                                                    const double *__restrict__ npart) {
    double v = npart[lane];
    for (int w = 1; w < W; ++w) v += npart[w * 32 + lane];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return __shfl_sync(0xffffffffu, v, 0);
}

// Row J of R and the factors f[k], k > J, from the reflector and the dot products dk[kk] of
// column J+1+kk with column J.  With T = float the bulk's FP32 copy fT of f is written too
// (one conversion per factor here instead of one per column crossing in every bulk lane).
template <typename T = double>
__device__ __forceinline__ void apply_reflector(const int lane, const int n, const int J,
                                                const Reflector &h, double *__restrict__ Rp,
                                                double *__restrict__ f,
                                                const double *__restrict__ dk,
                                                T *fT = nullptr) {
    const int U = n - J - 1;
    const int ro = rowoff(n, J);
    for (int kk = lane; kk < U; kk += 32) {
        const int k = J + 1 + kk;
        const int idx = ro + 1 + kk;
        double fk = 0.0;
        if (!h.ident) {
            const double rjk = Rp[idx];
            const double wk = fma(h.c, dk[kk], rjk);
            Rp[idx] = fma(-h.tau, wk, rjk);
            fk = -wk * h.ib;
        }
        f[k] = fk;
        if constexpr (!std::is_same<T, double>::value) fT[k] = (T)fk;
    }
    if (lane == 0) Rp[ro] = h.beta;
}

// V consecutive elements of T in one shared-memory access (V*sizeof(T) <= 16 bytes; the
// address must be V*sizeof(T)-aligned).
template <int V, typename T>
__device__ __forceinline__ void ld_vec(const T *p, T *out) {
    if constexpr (V == 1) {
        out[0] = p[0];
    } else if constexpr (sizeof(T) == 8) {
        static_assert(V == 2, "FP64 vectors are double2");
        const double2 v = *reinterpret_cast<const double2 *>(p);
        out[0] = v.x;
        out[1] = v.y;
    } else if constexpr (V == 2) {
        const float2 v = *reinterpret_cast<const float2 *>(p);
        out[0] = v.x;
        out[1] = v.y;
    } else {
        static_assert(V == 4, "FP32 vectors are float2 or float4");
        const float4 v = *reinterpret_cast<const float4 *>(p);
        out[0] = v.x;
        out[1] = v.y;
        out[2] = v.z;
        out[3] = v.w;
    }
}

template <int V, typename T>
__device__ __forceinline__ void st_vec(T *p, const T *in) {
    if constexpr (V == 1) {
        p[0] = in[0];
    } else if constexpr (sizeof(T) == 8) {
        *reinterpret_cast<double2 *>(p) = make_double2(in[0], in[1]);
    } else if constexpr (V == 2) {
        *reinterpret_cast<float2 *>(p) = make_float2(in[0], in[1]);
    } else {
        *reinterpret_cast<float4 *>(p) = make_float4(in[0], in[1], in[2], in[3]);
    }
}

template <int B, int V, typename T>
__device__ __forceinline__ void ld_block(const T *p, T *out) {
#pragma unroll
    for (int q = 0; q < B; q += V) ld_vec<V>(p + q, out + q);
}

// Phase B of step J for one bulk lane, plain form (the FP64 path, whose limit is the FP64
// pipe): blocks of B rows, loaded, updated, stored and dotted in program order.
template <typename T, int B>
__device__ __forceinline__ void phase_b_plain(const int lane, const int J, const int U,
                                              const int r, const int Hw, const int n,
                                              T *__restrict__ S, const int ldS, const int r0,
                                              const T *__restrict__ Sj,
                                              const T *__restrict__ SJ,
                                              const T *fT,
                                              T *__restrict__ seg) {
    const int run = U * r;
    const int p = lane * run;
    int kk = p / Hw;
    int i = p - kk * Hw;
    T *Sk = S + (size_t)(J + 1 + kk) * ldS + r0;
    T acc = (T)0;
    if (J > 0) {
        T fk = fT[J + 1 + kk];
        for (int blk = 0; blk < run; blk += B) {
            T x[B];
#pragma unroll
            for (int q = 0; q < B; ++q) x[q] = fmat(-fk, Sj[i + q], Sk[i + q]);
#pragma unroll
            for (int q = 0; q < B; ++q) Sk[i + q] = x[q];
#pragma unroll
            for (int q = 0; q < B; ++q) acc = fmat(SJ[i + q], x[q], acc);
            i += B;
            if (i == Hw) {
                seg[lane + kk] = acc;
                acc = (T)0;
                i = 0;
                ++kk;
                Sk += ldS;
                fk = fT[min(J + 1 + kk, n - 1)];
            }
        }
    } else {
        for (int blk = 0; blk < run; blk += B) {
#pragma unroll
            for (int q = 0; q < B; ++q) acc = fmat(SJ[i + q], Sk[i + q], acc);
            i += B;
            if (i == Hw) {
                seg[lane + kk] = acc;
                acc = (T)0;
                i = 0;
                ++kk;
                Sk += ldS;
            }
        }
    }
    if (i != 0) seg[lane + kk] = acc;
}

// Phase B of step J for one bulk lane, pipelined form (the mixed path, whose FP32 bulk is
// latency-bound): its run of U r items (column-major over the U trailing
// columns x its warp's Hw rows), in blocks of B rows that never straddle a column.  Software
// pipelined: the next block's three operands are loaded before the current block is updated
// and stored (the two blocks never overlap: different rows, or the next column).
template <typename T, int B, int V>
__device__ __forceinline__ void phase_b(const int lane, const int J, const int U, const int r,
                                        const int Hw, const int n, T *__restrict__ S,
                                        const int ldS, const int r0, const T *__restrict__ Sj,
                                        const T *__restrict__ SJ, const T *fT,
                                        T *__restrict__ seg) {
    const int run = U * r;
    const int nblk = run / B;
    const int p = lane * run;
    int kk = p / Hw;
    int i = p - kk * Hw;
    T *Sk = S + (size_t)(J + 1 + kk) * ldS + r0;
    T acc = (T)0;
    T s[B], b[B];
    ld_block<B, V>(Sk + i, s);
    ld_block<B, V>(SJ + i, b);
    if (J > 0) {
        T fk = fT[J + 1 + kk];
        T a[B];
        ld_block<B, V>(Sj + i, a);
        for (int blk = 0; blk < nblk; ++blk) {
            int i2 = i + B, kk2 = kk;
            T *Sk2 = Sk;
            const bool cross = (i2 == Hw);
            if (cross) {
                i2 = 0;
                ++kk2;
                Sk2 += ldS;
            }
            T a2[B], s2[B], b2[B];
            if (blk + 1 < nblk) {
                ld_block<B, V>(Sk2 + i2, s2);
                ld_block<B, V>(Sj + i2, a2);
                ld_block<B, V>(SJ + i2, b2);
            }
            T x[B];
#pragma unroll
            for (int q = 0; q < B; ++q) x[q] = fmat(-fk, a[q], s[q]);
#pragma unroll
            for (int q = 0; q < B; q += V) st_vec<V>(Sk + i + q, x + q);
#pragma unroll
            for (int q = 0; q < B; ++q) acc = fmat(b[q], x[q], acc);
            if (cross) {
                seg[lane + kk] = acc;
                acc = (T)0;
                fk = fT[min(J + 1 + kk2, n - 1)];
            }
            i = i2;
            kk = kk2;
            Sk = Sk2;
#pragma unroll
            for (int q = 0; q < B; ++q) {
                a[q] = a2[q];
                s[q] = s2[q];
                b[q] = b2[q];
            }
        }
    } else {
        for (int blk = 0; blk < nblk; ++blk) {
            int i2 = i + B, kk2 = kk;
            T *Sk2 = Sk;
            const bool cross = (i2 == Hw);
            if (cross) {
                i2 = 0;
                ++kk2;
                Sk2 += ldS;
            }
            T s2[B], b2[B];
            if (blk + 1 < nblk) {
                ld_block<B, V>(Sk2 + i2, s2);
                ld_block<B, V>(SJ + i2, b2);
            }
#pragma unroll
            for (int q = 0; q < B; ++q) acc = fmat(b[q], s[q], acc);
            if (cross) {
                seg[lane + kk] = acc;
                acc = (T)0;
            }
            i = i2;
            kk = kk2;
            Sk = Sk2;
#pragma unroll
            for (int q = 0; q < B; ++q) {
                s[q] = s2[q];
                b[q] = b2[q];
            }
        }
    }
    if (i != 0) seg[lane + kk] = acc;
}

// Where one chunk's reflectors go when the fold keeps them (tsqr_qr): the tails of column J
// into V(0:rows-1, J) (leading dimension ldv), (tau_J, c_J) into sc[2J], sc[2J+1].
struct QChunk {
    double *V;
    int64_t ldv;
    int rows;
    double *sc;
};

// A bulk lane's rows (r0 + lane + 32 t, t < r) of column `col` of the chunk to qc.V, rows
// past the chunk's last row of A skipped.
template <typename T>
__device__ __forceinline__ void store_tail_rows(const T *S, const int ldS, const int r0,
                                                const int r, const int lane, const int col,
                                                const QChunk &qc) {
    const T *src = S + (size_t)col * ldS;
    double *dst = qc.V + (int64_t)col * qc.ldv;
    for (int t = 0; t < r; ++t) {
        const int i = r0 + lane + 32 * t;
        if (i < qc.rows) dst[i] = (double)src[i];
    }
}

// Leaf fold.  Warps 0..Wb-1 ("bulk" warps) own the chunk's rows; warp Wb is the reducer.
// Every bulk lane owns r rows of its warp's block (Hw = 32 r) and a phase-B run of U r items
// starting at item lane * U r; runs and column boundaries are multiples of r, so blocks of B
// items (B divides r) never straddle a column: the inner loop has no per-item bookkeeping and
// all lanes stay in lockstep.  The reducer forms reflector J's scalars (its long FP64 chain)
// while the bulk warps run phase B, then sums the dot products and updates R and f:
//   A (bulk) | barrier | B (bulk) || scalars (reducer) | barrier | dots, R, f (reducer) | barrier.
// The next chunk of rows streams into columns no longer read (J-2 at step J) by cp.async when
// A's type is T; a BF16 A is widened after the fold instead.  T = double is the FP64 path;
// T = float the mixed path, where the bulk arithmetic and its dot-product partials are FP32
// and the reflector norms, scalars, R and f are FP64.  On the mixed path the bulk lanes do no
// FP64 work beyond one conversion of their norm partial per column: they read an FP32 copy
// fT of f and write FP32 partials, which the reducer sums across warps in FP32 and converts
// once per slot (an FP64-unit instruction costs the same whatever the active lanes, and lanes
// cross column boundaries at different blocks).  With T = double, fT is f itself.
// With kStore (FP64 only) the fold also keeps its reflectors (qc): column J's tail is final
// once phase A of step J has run, and is written out during step J+1, before the prefetch of
// step J+2 reuses the column.
template <typename T, typename Tin, int B, int V, bool kPipe, bool kStore = false>
__device__ __forceinline__ void fold_leaf(T *__restrict__ S, const int ldS, const int hs,
                                          double *__restrict__ Rp, double *__restrict__ f,
                                          T *fT, double *__restrict__ seg_dbl,
                                          double *__restrict__ tot, double *__restrict__ npart,
                                          const int n, const Chunk<Tin> pf,
                                          const QChunk qc = QChunk{}) {
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int Wb = (blockDim.x >> 5) - 1;
    const bool reducer = (warp == Wb);
    const int Hw = hs / Wb;
    const int r = Hw >> 5;
    const int r0 = warp * Hw;
    const int ss = seg_stride(n);
    T *seg_all = reinterpret_cast<T *>(seg_dbl);
    T *seg = seg_all + warp * ss;

    for (int J = 0; J < n; ++J) {
        if (Copy<T, Tin>::kAsync && pf.src && J >= 2) load_column(S, ldS, hs, pf, J - 2);
        if constexpr (kStore) {
            if (!reducer && J >= 1) store_tail_rows(S, ldS, r0, r, lane, J - 1, qc);
        }
        const int U = n - J - 1;
        T *SJ = S + (size_t)J * ldS + r0;
        const T *Sj = S + (size_t)(J > 0 ? J - 1 : 0) * ldS + r0;

        // ---- A: column J gets reflector J-1; per-lane partial squared norm of column J
        if (!reducer) {
            T nacc = (T)0, nacc2 = (T)0;  // two chains: half the latency for tall lanes
            if (J > 0) {
                const T fJ = fT[J];
                int t = 0;
                for (; t + 1 < r; t += 2) {
                    const int i = lane + 32 * t;
                    const T s = fmat(-fJ, Sj[i], SJ[i]);
                    const T s2 = fmat(-fJ, Sj[i + 32], SJ[i + 32]);
                    SJ[i] = s;
                    SJ[i + 32] = s2;
                    nacc = fmat(s, s, nacc);
                    nacc2 = fmat(s2, s2, nacc2);
                }
                if (t < r) {
                    const int i = lane + 32 * t;
                    const T s = fmat(-fJ, Sj[i], SJ[i]);
                    SJ[i] = s;
                    nacc = fmat(s, s, nacc);
                }
            } else {
                int t = 0;
                for (; t + 1 < r; t += 2) {
                    const T s = SJ[lane + 32 * t];
                    const T s2 = SJ[lane + 32 * t + 32];
                    nacc = fmat(s, s, nacc);
                    nacc2 = fmat(s2, s2, nacc2);
                }
                if (t < r) {
                    const T s = SJ[lane + 32 * t];
                    nacc = fmat(s, s, nacc);
                }
            }
            npart[warp * 32 + lane] = (double)(nacc + nacc2);
            for (int id = lane; id < 32 + U; id += 32) seg[id] = (T)0;
        }
        __syncthreads();

        Reflector h;
        if (reducer) {
            // ---- reflector J's scalars, overlapping phase B
            h = make_reflector(Rp[rowoff(n, J)], sum_norm_partials(lane, Wb, npart));
            if constexpr (kStore) {
                if (lane == 0) {
                    qc.sc[2 * J] = h.ident ? 0.0 : h.tau;
                    qc.sc[2 * J + 1] = h.ident ? 0.0 : h.c;
                }
            }
        } else if (U > 0) {
            // ---- B: fused update by reflector J-1 and dots with column J
            if constexpr (kPipe)
                phase_b<T, B, V>(lane, J, U, r, Hw, n, S, ldS, r0, Sj, SJ, fT, seg);
            else
                phase_b_plain<T, B>(lane, J, U, r, Hw, n, S, ldS, r0, Sj, SJ, fT, seg);
        }
        __syncthreads();

        // ---- reducer: dot products in a fixed order, row J of R, factors f[k] for k > J
        if (reducer) {
            for (int id = lane; id < 32 + U; id += 32) {
                T t = seg_all[id];
                for (int w = 1; w < Wb; ++w) t += seg_all[w * ss + id];
                tot[id] = (double)t;
            }
            __syncwarp();
            const int Nw = U * Hw;
            double *dk = tot + ss;
            for (int kk = lane; kk < U; kk += 32) {
                const int la = (32 * (kk * Hw + 1) - 1) / Nw;
                const int lb = (32 * (kk + 1) * Hw - 1) / Nw;
                double d0 = tot[kk + la], d1 = 0.0;  // two chains: half the latency
                for (int l = la + 1; l + 1 <= lb; l += 2) {
                    d0 += tot[kk + l];
                    d1 += tot[kk + l + 1];
                }
                if (((lb - la) & 1) == 1) d0 += tot[kk + lb];
                dk[kk] = d0 + d1;
            }
            __syncwarp();
            apply_reflector<T>(lane, n, J, h, Rp, f, dk, fT);
        }
        __syncthreads();
    }
    if constexpr (kStore) {
        if (!reducer) store_tail_rows(S, ldS, r0, r, lane, n - 1, qc);
        __syncthreads();  // the prefetch below reuses column n-1
    }
    if (Copy<T, Tin>::kAsync && pf.src) {
        for (int col = n - 2; col < n; ++col)
            if (col >= 0) load_column(S, ldS, hs, pf, col);
    }
}

// Tree-operator fold: R <- R([R; T_1; ...; T_c]) for c upper triangles stacked in S (FP64,
// column-major, leading dimension ldSd; triangle t in rows t n .. t n + n-1).  For c = 1 this
// is the operator qr(R1, R2) of Table 3; c > 1 reduces c+1 tree nodes in one sweep (the stacked
// triangles' QR, which associativity allows, Section 2).  At step J the reflector's support in
// S is rows 0..J of every triangle (the paper's j+2-entry reflector for c = 1).
// Warp 0 updates column J, forms its squared norm and then reflector J's scalars while the
// other warps (which split the trailing columns) run the fused update + dot sweep; warp 0 then
// sums their partials in a fixed order and updates R and f.  Needs at least two warps.
// With nsc non-null the reflectors' (tau_J, c_J) go to nsc[2J], nsc[2J+1] (their tails stay
// in S: rows 0..J of each triangle's column J).
// worker_sums: every worker warp sums its own columns' dot-product partials right after its
// sweep, while warp 0 forms the reflector (shorter chain: for a combine that runs alone);
// otherwise warp 0 sums them all after the barrier (a quarter of the FP64 instructions, whose
// pipe time counts when many combines run at once).  Both give the same bytes.
__device__ __forceinline__ void fold_stack(double *__restrict__ S, const int ldSd, const int c,
                                           double *__restrict__ Rp, double *__restrict__ f,
                                           double *__restrict__ seg_all,
                                           double *__restrict__ dk, const int n,
                                           double *nsc = nullptr,
                                           const bool worker_sums = true) {
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int Wp = (blockDim.x >> 5) - 1;  // worker warps 1..Wp
    const int ss = seg_stride(n);
    double *seg = seg_all + (warp > 0 ? warp - 1 : 0) * ss;

    for (int J = 0; J < n; ++J) {
        const int U = n - J - 1;
        const int h1 = J + 1;    // active rows per triangle
        const int cw = c * h1;   // active rows per column
        double *SJ = S + (size_t)J * ldSd;
        const double *Sj = S + (size_t)(J > 0 ? J - 1 : 0) * ldSd;

        double sig2 = 0.0;
        if (warp == 0) {
            // ---- A: column J gets reflector J-1; its squared norm
            const double fJ = (J > 0) ? f[J] : 0.0;
            double nacc = 0.0;
            for (int q = lane; q < cw; q += 32) {
                const int t = q / h1;
                const int row = q + t * (n - h1);  // t n + (q - t h1)
                double x = SJ[row];
                if (J > 0) {
                    x = fma(-fJ, Sj[row], x);
                    SJ[row] = x;
                }
                nacc = fma(x, x, nacc);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) nacc += __shfl_down_sync(0xffffffffu, nacc, o);
            sig2 = __shfl_sync(0xffffffffu, nacc, 0);
        } else {
            for (int id = lane; id < 32 + U; id += 32) seg[id] = 0.0;
        }
        __syncthreads();

        Reflector hr;
        if (warp == 0) {
            hr = make_reflector(Rp[rowoff(n, J)], sig2);
            if (nsc && lane == 0) {
                nsc[2 * J] = hr.ident ? 0.0 : hr.tau;
                nsc[2 * J + 1] = hr.ident ? 0.0 : hr.c;
            }
        } else {
            // ---- B: worker warp w owns trailing columns [kc0, kc1); its (column, row) items
            //      are cut into 32 equal contiguous runs in lockstep
            const int w = warp - 1;
            const int kc0 = (w * U) / Wp, kc1 = ((w + 1) * U) / Wp;
            const int N = (kc1 - kc0) * cw;
            if (N > 0) {
                int p = (int)(((long long)lane * N) >> 5);
                const int pend = (int)(((long long)(lane + 1) * N) >> 5);
                if (p < pend) {
                    int kk = p / cw;
                    int q = p - kk * cw;
                    int t = q / h1;
                    int i = q - t * h1;
                    int row = t * n + i;
                    int k = J + 1 + kc0 + kk;
                    double *Sk = S + (size_t)k * ldSd;
                    double fk = (J > 0) ? f[k] : 0.0;
                    double acc = 0.0;
                    for (;;) {
                        double x = Sk[row];
                        if (J > 0) {
                            x = fma(-fk, Sj[row], x);
                            Sk[row] = x;
                        }
                        acc = fma(SJ[row], x, acc);
                        if (++p == pend) break;
                        ++row;
                        if (++i == h1) {
                            i = 0;
                            row += n - h1;
                            if (++t == c) {
                                seg[lane + kk] = acc;
                                acc = 0.0;
                                t = 0;
                                row = 0;
                                ++kk;
                                ++k;
                                Sk += ldSd;
                                fk = (J > 0) ? f[k] : 0.0;
                            }
                        }
                    }
                    seg[lane + kk] = acc;
                }
            }
            // ---- the warp's columns' dot products, while warp 0 forms the reflector: column
            //      kc0 + rel sums the partials of the warp's lanes la..lb (whose runs touch it)
            //      in a fixed order
            __syncwarp();
            for (int rel = lane; worker_sums && rel < kc1 - kc0; rel += 32) {
                const int la = (32 * (rel * cw + 1) - 1) / N;
                const int lb = (32 * (rel + 1) * cw - 1) / N;
                const double *sg = seg + rel;
                double d0 = sg[la], d1 = 0.0;
                for (int l = la + 1; l + 1 <= lb; l += 2) {
                    d0 += sg[l];
                    d1 += sg[l + 1];
                }
                if (((lb - la) & 1) == 1) d0 += sg[lb];
                dk[kc0 + rel] = d0 + d1;
            }
        }
        __syncthreads();

        if (warp == 0) {
            if (!worker_sums) {
                // ---- warp 0 sums column kk's partials: those of its owner warp's lanes la..lb
                //      (the same sums in the same order as the worker warps')
                for (int kk = lane; kk < U; kk += 32) {
                    const int w = ((kk + 1) * Wp - 1) / U;
                    const int kc0 = (w * U) / Wp, kc1 = ((w + 1) * U) / Wp;
                    const int rel = kk - kc0;
                    const int Nw = (kc1 - kc0) * cw;
                    const int la = (32 * (rel * cw + 1) - 1) / Nw;
                    const int lb = (32 * (rel + 1) * cw - 1) / Nw;
                    const double *sg = seg_all + w * ss + rel;
                    double d0 = sg[la], d1 = 0.0;
                    for (int l = la + 1; l + 1 <= lb; l += 2) {
                        d0 += sg[l];
                        d1 += sg[l + 1];
                    }
                    if (((lb - la) & 1) == 1) d0 += sg[lb];
                    dk[kk] = d0 + d1;
                }
                __syncwarp();
            }
            apply_reflector(lane, n, J, hr, Rp, f, dk);
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
// streamed in during the current fold), then climbs the k-ary tree (k = 2: Fig. 1): it
// publishes R in its node's slot and bumps the parent's counter; the last child to arrive
// stacks the children in index order (the lowest on top), folds them and climbs on; the
// others return.  No CTA ever waits for another, and the operand order depends only on the
// indices.
// ------------------------------------------------------------------------------------------
// The k-ary tree above leaf `leaf` (k = a.arity; level l has ceil(nleaves / k^l) nodes,
// stored level after level): publish R in the node's slot and bump the parent's counter; the
// last child to arrive stacks the children in index order (the lowest on top), folds them and
// climbs on; the others return.  The root writes the sign-normalized R.  Rp holds the leaf's
// R; Sd (leading dimension ldSd) must hold arity-1 stacked n x n triangles.
// Tree levels of at most this many nodes combine with fold_stack's worker sums: few combines
// run at once there, each bound by its serial chain (the binary tree over 4,194,304 x 32,
// 16,384 leaves, ran 2.7% slower with worker sums at every level; the 10,000 x 16 one, 40
// leaves, 12% faster).
constexpr int kWorkerSumNodes = 152;

template <bool kStore>
// worker_sum_nodes: levels with at most this many nodes combine with fold_stack's worker sums
// (0 for the batch kernels, whose problems' combines run many at once).
__device__ __forceinline__ void climb_tree(const F64Args &a, double *Sd, const int ldSd,
                                           double *Rp, double *f, double *seg, double *tot,
                                           unsigned int *flag, const int leaf,
                                           const int worker_sum_nodes = kWorkerSumNodes) {
    const int n = a.n;
    // k-ary tree: node t of level l+1 has children k t .. k t + k-1 of level l
    const int k = a.arity;
    int cnt = a.nleaves, off = 0, t = leaf;  // nodes and first node id of the current level
    for (;;) {
        if (cnt == 1) {
            if constexpr (kStore) {
                for (int k2 = threadIdx.x; k2 < n; k2 += blockDim.x)
                    a.q.signs[k2] = (Rp[rowoff(n, k2)] < 0.0) ? -1.0 : 1.0;
            }
            store_normalized(Rp, n, a.R, a.ldr, a.status);
            return;
        }
        const int next_off = off + cnt, next_cnt = (cnt + k - 1) / k;
        const int parent = t / k, first = parent * k;
        const int nchild = min(k, cnt - first);
        if (nchild == 1) {  // a lone last child: promoted unchanged
            off = next_off;
            cnt = next_cnt;
            t = parent;
            continue;
        }
        store_packed(Rp, n, a.slots + (size_t)(off + t) * n * n, n);
        __threadfence();
        __syncthreads();
        if (threadIdx.x == 0) flag[0] = atomicAdd(&a.counters[next_off + parent], 1u);
        __syncthreads();
        if (flag[0] + 1 < (unsigned)nchild) return;  // a later sibling combines
        __threadfence();
        // the last child to arrive stacks the children in index order: the first on top
        load_packed_cg(a.slots + (size_t)(off + first) * n * n, n, n, Rp);
        for (int ch = 1; ch < nchild; ++ch)
            load_tri_cg(a.slots + (size_t)(off + first + ch) * n * n, n, n,
                        Sd + (size_t)(ch - 1) * n, ldSd);
        __syncthreads();
        if constexpr (kStore) {
            const size_t id = (size_t)next_off + parent;
            const int ldv = (k - 1) * n;
            fold_stack(Sd, ldSd, nchild - 1, Rp, f, seg, tot + seg_stride(n), n,
                       a.q.node_sc + id * 2 * n, next_cnt <= worker_sum_nodes);
            // the node's tails: rows 0..(nchild-1) n - 1 of S (zero below each diagonal)
            double *dst = a.q.node_V + id * (size_t)ldv * n;
            const int rows = (nchild - 1) * n;
            for (int idx = threadIdx.x; idx < rows * n; idx += blockDim.x) {
                const int col = idx / rows, row = idx - col * rows;
                dst[row + (size_t)col * ldv] = Sd[row + (size_t)col * ldSd];
            }
        } else {
            fold_stack(Sd, ldSd, nchild - 1, Rp, f, seg, tot + seg_stride(n), n, nullptr,
                       next_cnt <= worker_sum_nodes);
        }
        off = next_off;
        cnt = next_cnt;
        t = parent;
    }
}

// One leaf of one problem: fold the leaf's rows into R, then climb the problem's k-ary tree
// (k = a.arity; level l has ceil(nleaves / k^l) nodes, stored level after level).  T: leaf storage and
// arithmetic type; Tin: type of A.  S is the leaf's chunk (T, leading dimension a.ldS); the
// tree operator works in the same memory viewed as FP64 with leading dimension ldSd.  Returns
// when the CTA is not the last of a node's children to arrive, or after writing the root.
// The tree operator's FP64 view of S (leading dimension ldSd) must hold arity-1 stacked n x n
// triangles.
// With kStore (FP64 only) every chunk's and every tree node's reflectors, and the root's row
// signs, are kept in a.q for forming Q (tsqr_qr); chunk boundaries are then multiples of a.h.
template <typename T, typename Tin, int B, int V, bool kPipe, bool kStore = false>
__device__ __forceinline__ void leaf_tree_job(const F64Args &a, const Tin *A, const int ldSd,
                                              const int s_doubles, const int leaf,
                                              const int worker_sum_nodes = kWorkerSumNodes) {
    extern __shared__ __align__(16) double smem[];
    const int n = a.n;
    const SmemLayout L = smem_layout_s(n, s_doubles, blockDim.x >> 5);
    T *S = reinterpret_cast<T *>(smem + L.S);
    double *Sd = smem + L.S;
    double *Rp = smem + L.Rp;
    double *f = smem + L.f;
    T *fT;
    if constexpr (std::is_same<T, double>::value)
        fT = f;
    else
        fT = reinterpret_cast<T *>(smem + L.fs);
    double *seg = smem + L.seg;
    double *tot = smem + L.tot;
    double *npart = smem + L.npart;
    unsigned int *flag = reinterpret_cast<unsigned int *>(smem + L.scal);

    for (int i = threadIdx.x; i < n * (n + 1) / 2; i += blockDim.x) Rp[i] = 0.0;

    // rows of this leaf, folded in chunks of h rows
    const int64_t u0 = ((int64_t)leaf * a.nunits) / a.nleaves;
    const int64_t u1 = ((int64_t)(leaf + 1) * a.nunits) / a.nleaves;
    const int64_t rbeg = u0 * a.unit;
    const int64_t rend = (u1 * a.unit < a.m) ? u1 * a.unit : a.m;
    const int64_t nchunks = (rend - rbeg + a.h - 1) / a.h;
    if (nchunks > 0) {
        Chunk<Tin> first;
        first.src = A + rbeg;
        first.lda = a.lda;
        first.rows = (int)((rend - rbeg < a.h) ? rend - rbeg : a.h);
        for (int col = 0; col < n; ++col) load_column(S, a.ldS, a.hs, first, col);
        cp_async_wait_all();
        __syncthreads();
    }
    for (int64_t c = 0; c < nchunks; ++c) {
        Chunk<Tin> next;
        next.src = nullptr;
        next.lda = a.lda;
        next.rows = 0;
        if (c + 1 < nchunks) {
            const int64_t r1 = rbeg + (c + 1) * a.h;
            next.src = A + r1;
            next.rows = (int)((rend - r1 < a.h) ? rend - r1 : a.h);
        }
        QChunk qc{};
        if constexpr (kStore) {
            const int64_t row0 = rbeg + c * a.h;
            qc.V = a.q.V + row0;
            qc.ldv = a.q.ldv;
            qc.rows = (int)((rend - row0 < a.h) ? rend - row0 : a.h);
            qc.sc = a.q.chunk_sc + (row0 / a.h) * 2 * n;
        }
        fold_leaf<T, Tin, B, V, kPipe, kStore>(S, a.ldS, a.hs, Rp, f, fT, seg, tot, npart, n,
                                               next, qc);
        if (next.src) {
            if constexpr (!Copy<T, Tin>::kAsync) {
                __syncthreads();
                for (int col = 0; col < n; ++col) load_column(S, a.ldS, a.hs, next, col);
            }
            cp_async_wait_all();
            __syncthreads();
        }
    }

    climb_tree<kStore>(a, Sd, ldSd, Rp, f, seg, tot, flag, leaf, worker_sum_nodes);
}


}  // namespace tsqr
