// Blocked mixed-precision leaf of libtsqr (FP32 or BF16 A): the flat fold R <- R([R; chunk])
// of Section 2's step 1 done by panels of 16 columns, each panel's reflectors applied to the
// columns right of it as one compact WY block on the tensor cores.
//
// Per chunk of h rows (in shared memory as FP32) and per panel P of 16 columns:
//   1. Panel factorization, column by column (the LAPACK dlarfg rule of the paper's operator,
//      Table 3): each thread holds its rows of the panel in registers; for reflector J the
//      threads update column J and the panel's later columns by reflector J-1 and form the
//      16 dot products of column J with every panel column (its squared norm, the dot
//      products with the earlier tails that the block's T factor needs, and those with the
//      later columns).
//      The per-lane partials (up to eight rows) and their sums over a warp's lanes are FP32;
//      the sums over the warps and every reflector scalar (beta, tau, 1/(alpha - beta)) are in
//      double-FP32 arithmetic (hi + lo pairs, about 44-48 bits) on the FP32 pipe.  Per
//      reflector: every panel warp sums its lanes' partials, one barrier, then every panel warp
//      forms the FP32 factors of the later columns while a scalar warp forms the reflector's
//      double-FP32 scalars and row J of R.
//   2. Compact WY form of the panel: with the tails x_J kept UNSCALED in the chunk and
//      v_J = [e_J; c_J x_J], the product H_0 ... H_15 equals I - V S V^T (LAPACK's dlarft
//      forward recurrence, S^-1 = diag(1 / tau) + strict_upper(G) in Joffrain et al.'s form),
//      G(i, J) = c_i c_J x_i . x_J.  S is formed after the panel's reflectors by 16-lane teams.
//   3. Trailing update of the columns T right of the panel (rows P of R, all rows of the
//      chunk): Z = X^T C(:, T) (tensor cores), W = R(P, T) + diag(c) Z, Y = S^T W,
//      R(P, T) -= Y, C(:, T) -= X (diag(c) Y) (tensor cores).
// The tensor-core products are split-TF32 (compensated) products with FP32 accumulation: every
// FP32 operand is exactly three TF32 parts (11 + 11 + 2 significant bits, split by truncation),
// diag(c) Y is split into three too, and the six partial products down to 2^-22 of the leading
// one are summed (the smallest first), so each product is as accurate as an FP32 dot product.
// R is held in double-FP32 during the leaf and converted (exactly) to FP64 for the FP64 tree
// (climb_tree / fold_stack, the paper's operator).
//
// Why this precision split: everything that multiplies the running triangle R (the reflector
// scalars, S, the R rows) is accurate to far below FP32 rounding, so R's accumulated content
// is transformed orthogonally to that accuracy chunk after chunk; the FP32 roundings land in
// the chunk's rows.  The dot products carry FP32 rounding (the per-lane partials and the lane
// sums), an error relative to the chunk's entries like the FP32 update's own.  The tails being
// exactly three TF32 parts makes the V the tensor cores use and the V that S is built from the
// same matrix: the tails are used exactly as stored.
#include <cuda.h>  // CUtensorMap and its encoding enums (the driver call is found at run time)
#include <cuda_bf16.h>
#include <cstring>
#include <mutex>
#include <type_traits>

#include "tsqr_fold.cuh"
#include "tsqr_tc.cuh"

namespace tsqr {

namespace wy {

constexpr int kThreads = 256;
constexpr int kWarps = 8;
constexpr int kPw = 16;       // panel width
constexpr int kMaxPartials = 24;  // partial Z tiles (row group x n-tile) in shared memory

// The Z product's tile sets for nt8 8-column tiles: the fewest (1, 2 or 4) whose
// (8 / sets) row groups x nt8 partial tiles fit kMaxPartials (nt8 <= 3 with 8 row groups, <= 6
// with 4, <= 12 with 2: n <= 112).
__host__ __device__ constexpr int z_tile_sets(int nt8) { return nt8 >= 7 ? 4 : nt8 >= 4 ? 2 : 1; }

// ------------------------------------------------------------------------------------------
// Double-FP32 ("df") arithmetic: a value is hi + lo with |lo| <= ulp(hi) / 2.  Error-free
// transformations (Knuth's TwoSum, Dekker's fast TwoSum, TwoProduct by FMA) in round-to-nearest
// intrinsics, which the compiler never contracts or reorders.
// ------------------------------------------------------------------------------------------
struct df {
    float hi, lo;
};
__device__ __forceinline__ df mk(float h, float l = 0.f) {
    df r;
    r.hi = h;
    r.lo = l;
    return r;
}
__device__ __forceinline__ df two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return mk(s, e);
}
__device__ __forceinline__ df fast_two_sum(float a, float b) {  // requires |a| >= |b| or a == 0
    const float s = __fadd_rn(a, b);
    return mk(s, __fsub_rn(b, __fsub_rn(s, a)));
}
__device__ __forceinline__ df dadd(df a, df b) {
    const df s = two_sum(a.hi, b.hi);
    return fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ df dneg(df a) { return mk(-a.hi, -a.lo); }
__device__ __forceinline__ df dsub(df a, df b) { return dadd(a, dneg(b)); }
__device__ __forceinline__ df two_prod(float a, float b) {
    const float p = __fmul_rn(a, b);
    return mk(p, __fmaf_rn(a, b, -p));
}
__device__ __forceinline__ df dmul(df a, df b) {
    const df p = two_prod(a.hi, b.hi);
    return fast_two_sum(p.hi, __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, p.lo)));
}
// The hardware's approximate reciprocal and square root (about 2^-22 relative); one Newton
// step in double-FP32 below makes either accurate to about 2^-44.
__device__ __forceinline__ float rcp_approx(float x) {
    float y;
    asm("rcp.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float sqrt_approx(float x) {
    float y;
    asm("sqrt.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
// 1/a: one Newton step y + y (1 - a y) from the approximate reciprocal y
__device__ __forceinline__ df drecip(df a) {
    const float y = rcp_approx(a.hi);
    const df e = dsub(mk(1.f), dmul(a, mk(y)));
    return fast_two_sum(y, __fmul_rn(y, e.hi));
}
// sqrt(a), a > 0: one Newton step y + (a - y^2) / (2 y) from the approximate square root
__device__ __forceinline__ df dsqrt(df a) {
    const float y = sqrt_approx(a.hi);
    const df e = dsub(a, two_prod(y, y));
    return fast_two_sum(y, __fmul_rn(e.hi, rcp_approx(__fmul_rn(2.f, y))));
}
__device__ __forceinline__ df shfl_df(df v, int src, int width = 32) {
    return mk(__shfl_sync(0xffffffffu, v.hi, src, width), __shfl_sync(0xffffffffu, v.lo, src, width));
}
__device__ __forceinline__ df shfl_xor_df(df v, int m) {
    return mk(__shfl_xor_sync(0xffffffffu, v.hi, m), __shfl_xor_sync(0xffffffffu, v.lo, m));
}

// Reflector J's scalars (the dlarfg rule: beta = -sign(alpha) sqrt(alpha^2 + sigma^2),
// sign(0) = +1; an exactly zero tail gives the identity) in double-FP32.
struct Refl {
    df beta, tau, c, ib;
    bool ident;
};
__device__ __forceinline__ Refl make_refl(const df alpha, const df sig2) {
    Refl r;
    r.ident = (sig2.hi == 0.f);
    r.beta = alpha;
    r.tau = mk(0.f);
    r.c = mk(0.f);
    r.ib = mk(0.f);
    if (!r.ident) {
        const df rt = dsqrt(dadd(dmul(alpha, alpha), sig2));
        const bool pos = alpha.hi >= 0.f;
        r.beta = pos ? dneg(rt) : rt;
        r.ib = drecip(r.beta);
        r.tau = dmul(dsub(r.beta, alpha), r.ib);
        r.c = drecip(dsub(alpha, r.beta));
    }
    return r;
}

// ------------------------------------------------------------------------------------------
// TF32 parts: tf32_trunc keeps the top 11 significant bits (the low 13 fraction bits cleared,
// one logic instruction; rounding with cvt.rna.tf32 instead cost 9% of the leaf's time at
// n = 64).
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ float tf32_trunc(float x) {
    return __uint_as_float(__float_as_uint(x) & 0xffffe000u);
}
// Two FP32 values (24 bits) each = h + m + l exactly: h its top 11 significant bits, m the next
// 11, l the last 2 (both differences exact: each drops bits below the part it removes), the
// differences taken two at a time as paired FMAs x + (-1) h (the same results as subtractions)
__device__ __forceinline__ void split3x2(float x0, float x1, float &h0, float &h1, float &m0,
                                         float &m1, float &l0, float &l1) {
    h0 = tf32_trunc(x0);
    h1 = tf32_trunc(x1);
    const float2 mone = make_float2(-1.f, -1.f);
    const float2 r = __ffma2_rn(make_float2(h0, h1), mone, make_float2(x0, x1));
    m0 = tf32_trunc(r.x);
    m1 = tf32_trunc(r.y);
    const float2 l = __ffma2_rn(make_float2(m0, m1), mone, r);
    l0 = l.x;
    l1 = l.y;
}
// a double-FP32 value to three TF32 parts (33 bits), by truncation as split3x2: h and m exact
// parts of the leading bits, l the rest truncated to 11 bits (below 2^-33 of the value)
__device__ __forceinline__ void split3_df(df x, float &h, float &m, float &l) {
    h = tf32_trunc(x.hi);
    const df r = two_sum(__fsub_rn(x.hi, h), x.lo);
    m = tf32_trunc(r.hi);
    l = tf32_trunc(__fadd_rn(__fsub_rn(r.hi, m), r.lo));
}

// ------------------------------------------------------------------------------------------
// The chunk in shared memory: FP32, in boxes of 32 rows x 16 columns (2 KB), box (i / 32,
// col / 16) at ((i / 32) NP + col / 16) 2048 bytes; in a box, column col % 16 is one 128-byte
// line, its 16-byte units XOR-swizzled by col % 8 (the layout of a 128-byte-swizzled TMA box):
// a warp reading 32 consecutive rows of a column, or 4 consecutive rows of 8 columns, touches
// 32 different banks.  Returns the float index.
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ int cidx(int i, int col, int NP) {
    return ((((i >> 5) * NP + (col >> 4)) << 9) + ((col & 15) << 5) +
            ((((i & 31) >> 2) ^ (col & 7)) << 2) + (i & 3));
}

// Shared-memory carve-up (bytes), identical on host and device.
struct Layout {
    int C;      // the chunk (h x 16 NP floats); the tree's FP64 stacked triangles afterwards
    int R;      // R, packed upper triangle row by row, one df (8 bytes) per entry; FP64 later
    int red;    // cross-warp partial sums: 2 buffers x 8 warps x 16 df
    int tau;    // 16 df
    int cc;     // 16 df
    int G;      // 16 x 16 df: x_i . x_J (i < J), scaled by c_i c_J before S is formed
    int S;      // 16 x 16 df (column-major)
    int bar;    // the update's mbarrier (8 bytes), the tensor-memory address (4 bytes), and
                // from byte 16 one mbarrier per panel for the chunk's TMA loads
    int W;      // 16 x ntmax df: W, then Y
    int B;      // diag(c) Y in three TF32 parts, K-major operands of 16 x ntmax16 each
    int P;      // kMaxPartials x 16 x 8 floats: partial Z tiles
    int f, seg, tot, flag;  // the tree's buffers (overlay W.. once the chunks are done)
    int total;
};

__host__ __device__ inline int round_up_i(int x, int a) { return (x + a - 1) / a * a; }

__host__ __device__ inline Layout layout(int n, int h) {
    Layout L;
    const int NP = (n + kPw - 1) / kPw;
    const int ntmax = round_up_i(n, 8) - kPw > 0 ? round_up_i(n, 8) - kPw : 8;
    const int ntmax16 = round_up_i(n, 16) - kPw > 0 ? round_up_i(n, 16) - kPw : 16;
    int o = 0;
    L.C = o;   o += h * NP * 64;
    L.R = o;   o += round_up_i(n * (n + 1) / 2 * 8, 16);
    L.red = o; o += 2 * kWarps * 16 * 8;
    L.tau = o; o += 16 * 8;
    L.cc = o;  o += 16 * 8;
    L.G = o;   o += 16 * 16 * 8;
    L.S = o;   o += 16 * 16 * 8;
    L.bar = o; o += 16 + 8 * 8;
    const int chunk_end_base = o;
    L.W = o;   o += 16 * ntmax * 8;
    L.B = o;   o += 3 * ntmax16 * 64;
    L.P = o;   o += kMaxPartials * 16 * 8 * 4;
    const int chunk_end = o;
    // the tree (after the last chunk) reuses the region from W on
    int t = chunk_end_base;
    L.f = t;    t += (n + 1) * 8;
    L.seg = t;  t += kWarps * seg_stride(n) * 8;
    L.tot = t;  t += 2 * seg_stride(n) * 8;
    L.flag = t; t += 16;
    L.total = chunk_end > t ? chunk_end : t;
    return L;
}

// ------------------------------------------------------------------------------------------
// Warp-wide FP32 sums of 16 partials per lane: a transposing butterfly (each level halves the
// values a lane keeps and exchanges the other half with its partner), five levels, 16
// exchanges and 16 additions.  Lane l ends with the sum of value idx(l) = 8 b4 + 4 b3 + 2 b2 +
// b1 (bi = bit i of l); lanes l and l ^ 1 hold the same value.  Fixed order: bit-reproducible.
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ float warp_sum16_f(const float (&v)[16], const int lane) {
    const bool b4 = lane & 16, b3 = lane & 8, b2 = lane & 4, b1 = lane & 2;
    float a[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const float send = b4 ? v[i] : v[i + 8];
        const float keep = b4 ? v[i + 8] : v[i];
        a[i] = __fadd_rn(keep, __shfl_xor_sync(0xffffffffu, send, 16));
    }
    float b[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float send = b3 ? a[i] : a[i + 4];
        const float keep = b3 ? a[i + 4] : a[i];
        b[i] = __fadd_rn(keep, __shfl_xor_sync(0xffffffffu, send, 8));
    }
    float c[2];
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const float send = b2 ? b[i] : b[i + 2];
        const float keep = b2 ? b[i + 2] : b[i];
        c[i] = __fadd_rn(keep, __shfl_xor_sync(0xffffffffu, send, 4));
    }
    const float send = b1 ? c[0] : c[1];
    const float keep = b1 ? c[1] : c[0];
    const float d = __fadd_rn(keep, __shfl_xor_sync(0xffffffffu, send, 2));
    return __fadd_rn(d, __shfl_xor_sync(0xffffffffu, d, 1));  // commutative: l, l ^ 1 agree
}
__device__ __forceinline__ int sum16_index(int lane) {
    return ((lane >> 4) & 1) * 8 + ((lane >> 3) & 1) * 4 + ((lane >> 2) & 1) * 2 + ((lane >> 1) & 1);
}

// The panel's T factor S (S^-1 = diag(1 / tau) + strict_upper(G), the compact form of LAPACK's
// dlarft): 16 teams of 16 lanes, team Jc forms column Jc by back substitution,
// S(Jc, Jc) = tau_Jc, S(i, Jc) = -tau_i sum_{l = i+1..Jc} G(i, l) S(l, Jc), with
// G(i, l) = (c_i (x_i . x_l)) c_l scaled first (|c x| <= 1: no intermediate overflows).  Needs
// 256 threads; S is column-major (S[Jc * 16 + i]); columns and rows from pw on are zero.
__device__ __forceinline__ void s_factor(const int tid, const int pw, df *G, df *S,
                                         const df *tau, const df *c) {
    {
        const int i = tid >> 4, J = tid & 15;
        if (i < J && J < pw) G[i * 16 + J] = dmul(dmul(c[i], G[i * 16 + J]), c[J]);
    }
    __syncthreads();
    const int Jc = tid >> 4, i = tid & 15;
    df acc = mk(0.f), s_mine = mk(0.f);
    for (int l = 15; l >= 0; --l) {
        if (l <= Jc && i == l) s_mine = (l == Jc) ? tau[l] : dneg(dmul(tau[l], acc));
        const df sl = shfl_df(s_mine, l, 16);
        if (l <= Jc && i < l) acc = dadd(acc, dmul(G[i * 16 + l], sl));
    }
    if (Jc >= pw || i > Jc) s_mine = mk(0.f);
    S[Jc * 16 + i] = s_mine;
}

// ------------------------------------------------------------------------------------------
// Chunk load: rows [0, rows) of A's columns [0, n) at src (leading dimension lda) into the
// chunk layout, zeros elsewhere (rows >= rows, columns >= n up to 16 NP): exact, since zero
// rows leave R unchanged.  FP32 by cp.async (16 bytes where vec4, else 4), BF16 widened.
// ------------------------------------------------------------------------------------------
template <typename Tin>
__device__ __forceinline__ void load_chunk(float *C, const Tin *src, int64_t lda, int rows, int n,
                                           int h, int NP, bool vec4) {
    const int cols = 16 * NP;
    if constexpr (sizeof(Tin) == 4) {
        if (vec4) {
            const int groups = h / 4;
            for (int idx = threadIdx.x; idx < groups * cols; idx += blockDim.x) {
                const int col = idx / groups, i = 4 * (idx - col * groups);
                float *dst = C + cidx(i, col, NP);
                if (col < n) {
                    const int nb = rows - i >= 4 ? 16 : (rows > i ? 4 * (rows - i) : 0);
                    const void *g = nb ? (const void *)(src + (int64_t)col * lda + i) : (const void *)src;
                    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
                    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(g),
                                 "r"(nb)
                                 : "memory");
                } else {
                    *reinterpret_cast<float4 *>(dst) = make_float4(0.f, 0.f, 0.f, 0.f);
                }
            }
        } else {
            for (int idx = threadIdx.x; idx < h * cols; idx += blockDim.x) {
                const int col = idx / h, i = idx - col * h;
                float *dst = C + cidx(i, col, NP);
                if (col < n) {
                    const bool ok = i < rows;
                    cp_async4(dst, ok ? (const void *)(src + (int64_t)col * lda + i) : (const void *)src,
                              ok ? 4 : 0);
                } else {
                    *dst = 0.f;
                }
            }
        }
        cp_async_commit();
        cp_async_wait_all();
    } else {
        // eight independent loads in flight per thread (h x cols is a multiple of 8 x 256)
        for (int idx0 = threadIdx.x; idx0 < h * cols; idx0 += 8 * blockDim.x) {
            float v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int idx = idx0 + u * blockDim.x, col = idx / h, i = idx - col * h;
                v[u] = (col < n && i < rows) ? __bfloat162float(src[(int64_t)col * lda + i]) : 0.f;
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int idx = idx0 + u * blockDim.x, col = idx / h, i = idx - col * h;
                C[cidx(i, col, NP)] = v[u];
            }
        }
    }
}

struct WyArgs2 {
    F64Args base;    // m, lda, n, unit, nunits, nleaves, arity, h, tree buffers, R, status
    const void *A;   // FP32 or BF16
    int ldSd;        // leading dimension of the tree's FP64 view of the chunk region
    int vec4;        // FP32 A with 16-byte aligned columns (cp.async of 4 rows)
    int tma;         // chunks arrive by TMA box loads (FP32, aligned, leaves of whole chunks)
};

// TMA state of a chunk loop: the tensor map, the next chunk's first row (-1: none), one
// mbarrier per panel, the parity of the current chunk's phase, and (kept by thread 0, which
// issues every load) the panels with a load in flight and the parity each such load completes.
struct Tma {
    const CUtensorMap *map;
    int64_t rnext;
    uint64_t *bar;
    uint32_t phase;
    uint32_t pend, ppar;
};

// TMA loads of panel k (columns 16 k .. 16 k + 15) of the chunk at row r0: h / 32 boxes of 32
// rows x 16 columns, one per 2 KB box region of the chunk layout; zeros past A's last row and
// column.  FP32 boxes land as the layout itself (the tensor map's 128-byte swizzle is the
// layout's XOR); BF16 boxes (1 KB, unswizzled, column after column) land in the upper half of
// the region and are widened in place by widen_panel.  One warp: lane 0 arms the barrier with
// the panel's bytes, then lane l issues boxes l, l + 32, ...; the barrier's phase completes once
// all bytes have landed.
template <typename Tin>
__device__ __forceinline__ void tma_panel(float *C, Tma &t, int64_t r0, int k, int h, int NP,
                                          uint32_t parity) {
    constexpr uint32_t box_bytes = 32u * 16u * sizeof(Tin);
    constexpr int half = sizeof(Tin) == 2 ? 256 : 0;
    const int lane = threadIdx.x & 31;
    if (lane == 0) tc::mbar_expect_tx(t.bar + k, (uint32_t)(h / 32) * box_bytes);
    __syncwarp();
    for (int rb = lane; rb < h / 32; rb += 32)
        tc::tma_load_2d(C + (size_t)(rb * NP + k) * 512 + half, t.map, (int)(r0 + 32 * rb), 16 * k,
                        t.bar + k);
    t.pend |= 1u << k;
    t.ppar = (t.ppar & ~(1u << k)) | (parity << k);
}

// Panel k's BF16 boxes, staged by tma_panel<__nv_bfloat16>, widened to the FP32 layout in place.
// Warp w takes boxes w, w + 8, ... of the chunk's h / 32: every lane reads its row of the 16
// columns before the warp writes any of them back over the staging half.
template <int HB>
__device__ __forceinline__ void widen_panel(float *C, int k, int NP) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int rb = warp; rb < 4 * HB; rb += kWarps) {
        const __nv_bfloat16 *st =
            reinterpret_cast<const __nv_bfloat16 *>(C + (size_t)(rb * NP + k) * 512 + 256);
        float v[kPw];
#pragma unroll
        for (int c = 0; c < kPw; ++c) v[c] = __bfloat162float(st[c * 32 + lane]);
        __syncwarp();
#pragma unroll
        for (int c = 0; c < kPw; ++c) C[cidx(32 * rb + lane, 16 * k + c, NP)] = v[c];
    }
}

// Bounded wait for panels k0 .. k1-1 of the current chunk (and their widening for BF16); the
// CTA agrees on the outcome.  False: a wait gave up (recorded in the status word).
template <typename Tin, int HB>
__device__ __forceinline__ bool wait_panels(float *C, Tma &t, int k0, int k1, int NP,
                                            int *status) {
    bool got = true;
    for (int k = k0; k < k1; ++k) got = got && tc::mbar_wait(t.bar + k, t.phase, 1LL << 22);
    if (__syncthreads_and(got ? 1 : 0) == 0) {
        if (status && threadIdx.x == 0) atomicOr(status, kStatusTimeoutBit);
        return false;
    }
    for (int k = k0; k < k1; ++k) t.pend &= ~(1u << k);
    if constexpr (sizeof(Tin) == 2)
        for (int k = k0; k < k1; ++k) widen_panel<HB>(C, k, NP);
    return true;
}

// ------------------------------------------------------------------------------------------
// One panel: factorization (reflectors J = 0 .. pw-1 of columns J0 + J), S, and the update of
// the columns right of it.  Chunks of h = 128 HB rows.
// ------------------------------------------------------------------------------------------
// Tensor memory of a CTA: for M-block b (rows 128 b .. 128 b + 127) the update's accumulator D_b
// at columns [DW b, DW b + DW) (DW = the widest trailing block, 16 to 48 columns) and the tails'
// three TF32 parts (A operand, 16 columns each) at [DW MB + 48 b, DW MB + 48 b + 48);
// MB = h / 128 M-blocks, (DW + 48) MB <= 512 columns in all.
struct Tmem {
    uint32_t base;   // allocated address (lane 0)
    uint64_t *bar;   // mbarrier the update's mma commit arrives on
    uint32_t phase;  // parity of the next commit's phase
    bool ok;         // false once a bounded wait gave up
    bool pending;    // a commit (of phase `phase`) not yet waited for: its wait gave up
};
__host__ __device__ constexpr int tmem_dw(int n) {
    return ((n + 15) / 16) * 16 - 16 > 16 ? ((n + 15) / 16) * 16 - 16 : 16;
}
__host__ __device__ constexpr int tmem_need(int n, int h) { return (tmem_dw(n) + 48) * (h / 128); }
__host__ __device__ constexpr uint32_t tmem_cols(int n, int h) {
    return tmem_need(n, h) <= 256 ? 256u : 512u;
}

// Warps that factorize a panel of h = 128 HB rows: four, one per sub-partition (HB rows per
// lane, up to 8, which the registers hold), and warp kPanelWarps, the scalar warp.
constexpr int kPanelWarps = 4;

// A column's barrier (named barrier 1): the panel warps and the scalar warp, once the warps'
// sums are in.
__device__ __forceinline__ void panel_sync() {
    asm volatile("bar.sync 1, %0;\n" ::"n"((kPanelWarps + 1) * 32) : "memory");
}

// Reflector J's double-FP32 scalars from the sums tot (lane l: value l & 15; tot of lane J is
// the squared norm of the tail) and alpha = R(Jg, Jg): row Jg of R (R(Jg, Jg) = beta and
// R(Jg, k) -= tau w_k, w_k = R(Jg, k) + c (x_J . x_k)), tau and c for the T factor, the dots
// with the earlier tails into G.
__device__ __forceinline__ void scalar_update(unsigned char *sm, const Layout &L, const int n,
                                              const int J0, const int J, const int pw,
                                              const int lane, const df tot) {
    df *Rd = reinterpret_cast<df *>(sm + L.R);
    df *tau_s = reinterpret_cast<df *>(sm + L.tau);
    df *c_s = reinterpret_cast<df *>(sm + L.cc);
    df *G = reinterpret_cast<df *>(sm + L.G);
    const int vi = lane & 15;
    const int Jg = J0 + J;
    const df alpha = Rd[rowoff(n, Jg)];
    const Refl rf = make_refl(alpha, shfl_df(tot, J));
    if (lane < 16) {
        if (vi > J && vi < pw && !rf.ident) {
            df *rjk = Rd + rowoff(n, Jg) + vi - J;
            const df wk = dadd(*rjk, dmul(rf.c, tot));
            *rjk = dsub(*rjk, dmul(rf.tau, wk));
        }
        if (vi < J) G[vi * 16 + J] = tot;  // x_vi . x_J (scaled in s_factor)
        if (vi == J) {
            tau_s[J] = rf.tau;
            c_s[J] = rf.c;
            Rd[rowoff(n, Jg)] = rf.beta;
        }
    }
}

// With TMA loads (t != nullptr): panel 0 has arrived when this is called; panel 0 waits for
// the other panels before its Z product reads them; and with a next chunk (t->rnext >= 0),
// panel k's columns of the next chunk are loaded as soon as this chunk no longer reads them:
// after the Z product (or, for the last panel, after its reflectors).
template <typename Tin, int HB>
__device__ __forceinline__ void panel_step(unsigned char *sm, const Layout &L, const int n,
                                           const int NP, const int k, Tmem &tm, int *status,
                                           Tma *t) {
    constexpr int h = 128 * HB;
    float *C = reinterpret_cast<float *>(sm + L.C);
    df *Rd = reinterpret_cast<df *>(sm + L.R);
    df *red = reinterpret_cast<df *>(sm + L.red);
    df *tau_s = reinterpret_cast<df *>(sm + L.tau);
    df *c_s = reinterpret_cast<df *>(sm + L.cc);
    df *G = reinterpret_cast<df *>(sm + L.G);
    df *S = reinterpret_cast<df *>(sm + L.S);
    df *W = reinterpret_cast<df *>(sm + L.W);
    float *B = reinterpret_cast<float *>(sm + L.B);
    float *P = reinterpret_cast<float *>(sm + L.P);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int J0 = kPw * k;
    const int pw = min(kPw, n - J0);

    // ---- 1. panel factorization in registers, by PW = 4 warps (one per sub-partition, whose
    //         lanes hold PR = h / 128 rows each, up to 8: half the warp-level reductions per
    //         row of eight warps)
    constexpr int PW = kPanelWarps;
    constexpr int PR = h / (32 * PW);
    const bool panel_warp = warp < PW;
    // the panel's rows in registers as pairs of columns (2 j, 2 j + 1): the update and the dot
    // products take paired FP32 FMAs (two IEEE FMAs an instruction, the same results)
    float2 x2[PR][kPw / 2];
#define TSQR_XE(q, kk) (((kk) & 1) ? x2[q][(kk) >> 1].y : x2[q][(kk) >> 1].x)
    if (panel_warp) {
#pragma unroll
        for (int q = 0; q < PR; ++q) {
            const int i = 32 * PW * q + 32 * warp + lane;
#pragma unroll
            for (int j = 0; j < kPw / 2; ++j)
                x2[q][j] = make_float2(C[cidx(i, J0 + 2 * j, NP)], C[cidx(i, J0 + 2 * j + 1, NP)]);
        }
        // The loop over the panel's columns is not unrolled (one copy of its body per half keeps
        // the instruction cache warm); the register columns are addressed with static indices.
        // Columns 0-7 are final once J >= 8: the second half updates columns 8-15 only, and
        // each half picks column J among its eight.
        // nfv: the negated factors -f_k, paired; xp: the previous column J-1's rows, both halves
        float2 nfv[kPw / 2], xp[PR];
#pragma unroll
        for (int j = 0; j < kPw / 2; ++j) nfv[j] = make_float2(0.f, 0.f);
#pragma unroll
        for (int q = 0; q < PR; ++q) xp[q] = make_float2(0.f, 0.f);
        auto column = [&](const int J, auto lo) {
            constexpr int LO = decltype(lo)::value;
            // columns LO.. get reflector J-1; the factors of the columns before J (and of the
            // padding columns) are zero, so every one of them takes the same exact FMA
#pragma unroll
            for (int j = LO / 2; j < kPw / 2; ++j)
#pragma unroll
                for (int q = 0; q < PR; ++q) x2[q][j] = __ffma2_rn(nfv[j], xp[q], x2[q][j]);
            float2 xj[PR];
#pragma unroll
            for (int q = 0; q < PR; ++q) {
                float tv = TSQR_XE(q, LO);
#pragma unroll
                for (int kk = LO + 1; kk < LO + 8; ++kk) tv = (kk == J) ? TSQR_XE(q, kk) : tv;
                xj[q] = make_float2(tv, tv);
            }
            float v[kPw];
#pragma unroll
            for (int j = 0; j < kPw / 2; ++j) {
                float2 sacc = __fmul2_rn(xj[0], x2[0][j]);
#pragma unroll
                for (int q = 1; q < PR; ++q) sacc = __ffma2_rn(xj[q], x2[q][j], sacc);
                v[2 * j] = sacc.x;
                v[2 * j + 1] = sacc.y;
            }
            // row Jg of R (FP32 parts) for the factors below, read before the barrier: the
            // scalar warp updates the row after it
            const int Jg = J0 + J;
            const int vi = lane & 15;
            const float a_f = Rd[rowoff(n, Jg)].hi;
            const float r_f = (vi > J && vi < pw) ? Rd[rowoff(n, Jg) + vi - J].hi : 0.f;
            const float ws = warp_sum16_f(v, lane);
            df *rb = red + (J & 1) * kWarps * 16;
            if ((lane & 1) == 0) rb[warp * 16 + sum16_index(lane)] = mk(ws);  // lo = 0: exact adds
            panel_sync();
            // every panel warp forms the factors f_k of the panel update (lane k forms f_k), in
            // FP32 (the update itself is FP32) from the warps' FP32 sums; the scalar warp forms
            // the reflector's double-FP32 scalars and row Jg of R meanwhile
            const float tf = __fadd_rn(__fadd_rn(rb[vi].hi, rb[16 + vi].hi),
                                       __fadd_rn(rb[32 + vi].hi, rb[48 + vi].hi));
            const float sig = __fadd_rn(__fadd_rn(rb[J].hi, rb[16 + J].hi),
                                        __fadd_rn(rb[32 + J].hi, rb[48 + J].hi));
            float fk = 0.f;
            if (sig != 0.f && vi > J && vi < pw) {
                // the hardware's approximate square root and reciprocals (about 2^-22): a few
                // FP32 ulps in f_k, the size of the update's own rounding
                const float rt = sqrt_approx(__fmaf_rn(a_f, a_f, sig));
                const float beta = a_f >= 0.f ? -rt : rt;
                const float w = __fmaf_rn(rcp_approx(__fsub_rn(a_f, beta)), tf, r_f);
                fk = -__fmul_rn(w, rcp_approx(beta));
            }
            const float nfk = -fk;
#pragma unroll
            for (int j = 0; j < kPw / 2; ++j)
                nfv[j] = make_float2(__shfl_sync(0xffffffffu, nfk, 2 * j),
                                     __shfl_sync(0xffffffffu, nfk, 2 * j + 1));
#pragma unroll
            for (int q = 0; q < PR; ++q) xp[q] = xj[q];
        };
#pragma unroll 1
        for (int J = 0; J < min(pw, 8); ++J) column(J, std::integral_constant<int, 0>{});
#pragma unroll 1
        for (int J = 8; J < pw; ++J) column(J, std::integral_constant<int, 8>{});
    }
    if (warp == PW) {
        // the scalar warp: after each column's barrier, reflector J's double-FP32 scalars and
        // row Jg of R from the cross-warp sums, while the panel warps form the factors and go
        // on with the next column (a buffer of sums is rewritten only after every panel warp
        // and this warp have passed the next column's barrier, so after their reads of it)
#pragma unroll 1
        for (int J = 0; J < pw; ++J) {
            panel_sync();
            const df *rb = red + (J & 1) * kWarps * 16;
            const int vi = lane & 15;
            const df tot = dadd(dadd(rb[vi], rb[16 + vi]), dadd(rb[32 + vi], rb[48 + vi]));
            scalar_update(sm, L, n, J0, J, pw, lane, tot);
        }
    }
    if (J0 + kPw < n) {  // S is needed only where columns right of the panel remain
        __syncthreads();
        s_factor(threadIdx.x, pw, G, S, tau_s, c_s);
    }
    const int n8 = round_up_i(n, 8);
    const int T0 = J0 + kPw;           // first trailing column
    const int ntp = n8 - T0;           // trailing columns, padded to 8
    if (ntp > 0 && panel_warp) {
        // the tails (unscaled) back to the chunk, for the Z product
#pragma unroll
        for (int q = 0; q < PR; ++q) {
            const int i = 32 * PW * q + 32 * warp + lane;
#pragma unroll
            for (int kk = 0; kk < kPw; ++kk) C[cidx(i, J0 + kk, NP)] = TSQR_XE(q, kk);
        }
        // the tails' three TF32 parts, this thread's rows, into tensor memory (the A operand of
        // the update): row 32 PW q + 32 w + l is lane 32 (w % 4) + l of M-block (PW q + w) / 4
        constexpr int MB = h / 128;
        const uint32_t lane_base = (uint32_t)(32 * (warp & 3)) << 16;
#pragma unroll
        for (int q = 0; q < PR; ++q) {
            const int b = (PW * q + warp) >> 2;
            float hi[8], mid[8], lo[8];
#pragma unroll
            for (int half = 0; half < 2; ++half) {
#pragma unroll
                for (int e = 0; e < 8; e += 2)
                    split3x2(TSQR_XE(q, 8 * half + e), TSQR_XE(q, 8 * half + e + 1), hi[e],
                             hi[e + 1], mid[e], mid[e + 1], lo[e], lo[e + 1]);
                const uint32_t col = (uint32_t)(tmem_dw(n) * MB + 48 * b + 8 * half);
                tc::tmem_st8(tm.base + lane_base + col, hi);
                tc::tmem_st8(tm.base + lane_base + col + 16u, mid);
                tc::tmem_st8(tm.base + lane_base + col + 32u, lo);
            }
        }
        tc::tmem_st_wait();
    }
#undef TSQR_XE
    if (ntp <= 0) {
        // the last panel: nothing reads its columns again in this chunk
        if (t && t->rnext >= 0) {
            tc::fence_proxy_async();
            __syncthreads();
            if (warp == 0) tma_panel<Tin>(C, *t, t->rnext, k, h, NP, t->phase ^ 1u);
        }
        __syncthreads();
        return;
    }
    // the Z product reads the trailing panels: with TMA loads, wait for them (and widen BF16)
    if (t && k == 0 && !wait_panels<Tin, HB>(C, *t, 1, NP, NP, status)) {
        tm.ok = false;
        return;
    }
    __syncthreads();

    // ---- 2a. Z = X^T C(:, T) on the tensor cores.  The 8 warps are KG row groups x TS sets of
    //          n-tiles (8 columns each): a warp splits its X fragments once per 8 rows and uses
    //          them for up to three tiles of its set at a time (a set of more tiles, past 64
    //          columns, takes several rounds over its rows).  Per tile three accumulators
    //          (below); partial tiles per row group go to P (KG NT8 <= kMaxPartials).
    const int NT8 = ntp / 8;
    const int TS = z_tile_sets(NT8);
    const int TPS = (NT8 + TS - 1) / TS;  // tiles per set (<= 3 for n <= 64)
    const int KG = kWarps / TS;           // row groups
    const int g4 = lane >> 2, t4 = lane & 3;
    const int grp = warp / TS, set = warp % TS;
    const int jt1 = min(NT8, set * TPS + TPS);
    for (int jt0 = set * TPS; jt0 < jt1; jt0 += 3) {
        const int r0 = grp * (h / KG), r1 = r0 + h / KG;  // multiples of 16
        // three accumulators per tile, smallest products first: ea (X_mid C_mid, X_lo C_hi,
        // X_hi C_lo), eb (X_mid C_hi, X_hi C_mid), hh (X_hi C_hi): shorter dependent mma chains
        float e[3][4] = {}, eb[3][4] = {}, hh[3][4] = {};
        // chunk addresses (cidx) split into a column part and a row part: every column read
        // here is g4 mod 8 (J0 and the tiles' first columns are multiples of 8), so a row's
        // swizzle is ((i % 32) / 4) ^ g4 for all of them
        const int ox0 = ((J0 >> 4) << 9) + (g4 << 5) + t4;  // column J0 + g4
        const int ox1 = ox0 + (8 << 5);                     // column J0 + g4 + 8
        int oc[3];
#pragma unroll
        for (int t = 0; t < 3; ++t) {
            const int c0 = T0 + 8 * (jt0 + t);
            oc[t] = ((c0 >> 4) << 9) + (((c0 & 15) + g4) << 5) + t4;  // column c0 + g4
        }
        for (int k0 = r0; k0 < r1; k0 += 16) {
            const int rb = ((k0 >> 5) * NP) << 9;
            const int s0 = (k0 & 31) >> 2;  // 0 or 4
#pragma unroll
            for (int half = 0; half < 2; ++half) {  // rows k0 + 8 half + t4 (sa), + 4 (sb)
                const int sa = rb + (((s0 + 2 * half) ^ g4) << 2);
                const int sb = rb + (((s0 + 2 * half + 1) ^ g4) << 2);
                const float xa[4] = {C[sa + ox0], C[sa + ox1], C[sb + ox0], C[sb + ox1]};
                float ah[4], am[4], al[4];
#pragma unroll
                for (int q = 0; q < 4; q += 2)
                    split3x2(xa[q], xa[q + 1], ah[q], ah[q + 1], am[q], am[q + 1], al[q],
                             al[q + 1]);
#pragma unroll
                for (int t = 0; t < 3; ++t) {
                    if (jt0 + t < jt1) {
                        const float cb[2] = {C[sa + oc[t]], C[sb + oc[t]]};
                        float bh[2], bm[2], bl[2];
#pragma unroll
                        split3x2(cb[0], cb[1], bh[0], bh[1], bm[0], bm[1], bl[0], bl[1]);
                        tc::mma_m16n8k8(e[t], am, bm);
                        tc::mma_m16n8k8(eb[t], am, bh);
                        tc::mma_m16n8k8(hh[t], ah, bh);
                        tc::mma_m16n8k8(e[t], al, bh);
                        tc::mma_m16n8k8(eb[t], ah, bm);
                        tc::mma_m16n8k8(e[t], ah, bl);
                    }
                }
            }
        }
#pragma unroll
        for (int t = 0; t < 3; ++t) {
            const int jt = jt0 + t;
            if (jt < jt1) {
                float *pt = P + (grp * NT8 + jt) * 128;  // tile, 16 x 8 row-major
                pt[g4 * 8 + 2 * t4] = __fadd_rn(__fadd_rn(e[t][0], eb[t][0]), hh[t][0]);
                pt[g4 * 8 + 2 * t4 + 1] = __fadd_rn(__fadd_rn(e[t][1], eb[t][1]), hh[t][1]);
                pt[(g4 + 8) * 8 + 2 * t4] = __fadd_rn(__fadd_rn(e[t][2], eb[t][2]), hh[t][2]);
                pt[(g4 + 8) * 8 + 2 * t4 + 1] = __fadd_rn(__fadd_rn(e[t][3], eb[t][3]), hh[t][3]);
            }
        }
    }
    if (t && t->rnext >= 0) tc::fence_proxy_async();  // the panel's columns are read for the last time
    __syncthreads();
    if (t && t->rnext >= 0 && warp == 0) tma_panel<Tin>(C, *t, t->rnext, k, h, NP, t->phase ^ 1u);

    // ---- 2b. W = R(P, T) + diag(c) Z
    for (int e = threadIdx.x; e < kPw * ntp; e += blockDim.x) {
        const int J = e / ntp, cc = e - J * ntp;
        const int col = T0 + cc;
        df wv = mk(0.f);
        if (J < pw && col < n) {
            const int jt = cc >> 3, c8 = cc & 7;
            df z = mk(P[jt * 128 + J * 8 + c8]);
            for (int grp = 1; grp < KG; ++grp) z = dadd(z, mk(P[(grp * NT8 + jt) * 128 + J * 8 + c8]));
            wv = dadd(Rd[rowoff(n, J0 + J) + col - (J0 + J)], dmul(c_s[J], z));
        }
        W[J * ntp + cc] = wv;
    }
    __syncthreads();

    // ---- 2c. Y = S^T W; R(P, T) -= Y; diag(c) Y in three TF32 parts, each a K-major
    //          operand of 16 (K) x ntp16 (N): core matrix (c / 8, J / 4) at (c / 8) 512 +
    //          (J / 4) 128 bytes, row c % 8 at 16 bytes, element J % 4 at 4
    const int ntp16 = round_up_i(ntp, 16);
    const int part_bytes = ntp16 * 64;
    for (int e = threadIdx.x; e < kPw * ntp16; e += blockDim.x) {
        const int J = e / ntp16, cc = e - J * ntp16;
        const int col = T0 + cc;
        float bh = 0.f, bm = 0.f, bl = 0.f;
        if (J < pw && col < n) {
            df y0 = mk(0.f), y1 = mk(0.f);  // two chains: half the latency
            int i = 0;
            for (; i + 1 <= J; i += 2) {
                y0 = dadd(y0, dmul(S[J * 16 + i], W[i * ntp + cc]));
                y1 = dadd(y1, dmul(S[J * 16 + i + 1], W[(i + 1) * ntp + cc]));
            }
            if (i <= J) y0 = dadd(y0, dmul(S[J * 16 + i], W[i * ntp + cc]));
            const df y = dadd(y0, y1);
            df *r = Rd + rowoff(n, J0 + J) + col - (J0 + J);
            *r = dsub(*r, y);
            split3_df(dmul(c_s[J], y), bh, bm, bl);
        }
        const int off = (cc >> 3) * 512 + (J >> 2) * 128 + (cc & 7) * 16 + (J & 3) * 4;
        *reinterpret_cast<float *>(reinterpret_cast<unsigned char *>(B) + off) = bh;
        *reinterpret_cast<float *>(reinterpret_cast<unsigned char *>(B) + part_bytes + off) = bm;
        *reinterpret_cast<float *>(reinterpret_cast<unsigned char *>(B) + 2 * part_bytes + off) = bl;
    }
    tc::fence_proxy_async();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();

    // ---- 2d. C(:, T) -= X (diag(c) Y) on the 5th-generation tensor cores: per M-block b,
    //          D_b = X_lo B_mid + X_hi B_lo + X_lo B_hi + X_hi B_mid + X_hi B_hi (smallest
    //          first, FP32 accumulation in tensor memory; X's parts in tensor memory, B's in
    //          shared memory), issued by one thread; then every thread subtracts its rows of D
    {
        constexpr int MB = h / 128;
        if (threadIdx.x == 0) {
            const uint32_t idesc = tc::instr_desc(tc::kFmtTF32, 128, ntp16, false, false);
            const uint32_t bsm = tc::smem_u32(B);
            // (A part, B part), 0 = hi, 1 = mid, 2 = lo; the products below 2^-33 are dropped
            const int terms[6][2] = {{1, 1}, {2, 0}, {0, 2}, {1, 0}, {0, 1}, {0, 0}};
            for (int b = 0; b < MB; ++b) {
                const uint32_t dcol = tm.base + (uint32_t)(tmem_dw(n) * b);
                const uint32_t acol = tm.base + (uint32_t)(tmem_dw(n) * MB + 48 * b);
                bool acc = false;
                for (int t = 0; t < 6; ++t)
                    for (int s2 = 0; s2 < 2; ++s2) {
                        const uint64_t bd = tc::smem_desc(
                            bsm + (uint32_t)(terms[t][1] * part_bytes + 256 * s2), 128, 512,
                            tc::kSwNone);
                        tc::mma_tf32_ts(dcol, acol + (uint32_t)(16 * terms[t][0] + 8 * s2), bd,
                                        idesc, acc);
                        acc = true;
                    }
            }
            tc::mma_commit(tm.bar);
        }
        // every thread polls (bounded); the CTA agrees on the outcome, so that all its threads
        // take the same path
        const bool done = __syncthreads_and(tc::mbar_wait(tm.bar, tm.phase, 1LL << 22) ? 1 : 0) != 0;
        if (done) {
            tm.phase ^= 1u;
        } else {
            // the commit stays pending (phase tm.phase): the caller waits for it once more,
            // bounded, before it releases the tensor memory
            tm.ok = false;
            tm.pending = true;
            if (status && threadIdx.x == 0) atomicOr(status, kStatusTimeoutBit);
        }
        tc::fence_after_sync();
        if (done) {
            const uint32_t lane_base = (uint32_t)(32 * (warp & 3)) << 16;
            // M-block b (rows 128 b ..) by warps 0-3 for even b, 4-7 for odd b
            for (int b = warp >> 2; b < MB; b += 2) {
                const int i = 128 * b + 32 * (warp & 3) + lane;
                for (int c0 = 0; c0 < ntp16; c0 += 8) {
                    float v[8];
                    tc::tmem_ld8(tm.base + lane_base + (uint32_t)(tmem_dw(n) * b + c0), v);
                    tc::tmem_ld_wait();
#pragma unroll
                    for (int e = 0; e < 8; e += 2) {  // C - D as paired FMAs C + (-1) D: exact
                        float *pc0 = C + cidx(i, T0 + c0 + e, NP);
                        float *pc1 = C + cidx(i, T0 + c0 + e + 1, NP);
                        const float2 d = __ffma2_rn(make_float2(v[e], v[e + 1]),
                                                    make_float2(-1.f, -1.f),
                                                    make_float2(*pc0, *pc1));
                        *pc0 = d.x;
                        *pc1 = d.y;
                    }
                }
            }
        }
        tc::fence_before_sync();
    }
    __syncthreads();
}

// One leaf: rows [rbeg, rend) of A folded into R chunk by chunk (TMA box loads where t is
// given, else thread copies), then R converted exactly to FP64 in place at L.R for the tree.
// Returns false when a wait gave up (recorded in the status word and agreed by the CTA); the
// caller then waits out what is in flight.
template <typename Tin, int HB>
__device__ __forceinline__ bool wy_leaf(unsigned char *sm, const Layout &L, const int n,
                                        const Tin *A, const int64_t lda, const int64_t rbeg,
                                        const int64_t rend, const bool vec4, Tmem &tm, Tma *t,
                                        int *status) {
    constexpr int h = 128 * HB;
    const int NP = (n + kPw - 1) / kPw;
    df *Rd = reinterpret_cast<df *>(sm + L.R);
    for (int e = threadIdx.x; e < n * (n + 1) / 2; e += blockDim.x) Rd[e] = mk(0.f);
    float *Cf = reinterpret_cast<float *>(sm + L.C);
    if (t && rbeg < rend && threadIdx.x < 32)
        for (int k = 0; k < NP; ++k) tma_panel<Tin>(Cf, *t, rbeg, k, h, NP, 0u);
    for (int64_t r0 = rbeg; r0 < rend && tm.ok; r0 += h) {
        const int rows = (int)((rend - r0 < h) ? rend - r0 : h);
        if (!t) {
            __syncthreads();  // the previous chunk's (or leaf's) last reads of C are done
            load_chunk<Tin>(Cf, A + r0, lda, rows, n, h, NP, vec4);
            __syncthreads();
        } else {
            t->rnext = (r0 + h < rend) ? r0 + h : -1;
            // panel 0 of this chunk (panel_step waits for the others before they are read)
            if (!wait_panels<Tin, HB>(Cf, *t, 0, 1, NP, status)) {
                tm.ok = false;
                break;
            }
            __syncthreads();
        }
        for (int k = 0; k < NP && tm.ok; ++k) panel_step<Tin, HB>(sm, L, n, NP, k, tm, status, t);
        if (t && tm.ok) t->phase ^= 1u;
    }
    tc::fence_before_sync();
    __syncthreads();
    if (!tm.ok) return false;
    // R to FP64 (exact: hi + lo), in place, for the FP64 tree
    double *Rp = reinterpret_cast<double *>(sm + L.R);
    for (int e = threadIdx.x; e < n * (n + 1) / 2; e += blockDim.x) {
        const df v = Rd[e];
        Rp[e] = (double)v.hi + (double)v.lo;
    }
    __syncthreads();
    return true;
}

// The tree above a leaf's R (FP64 at L.R): the FP64 climb of the one-reduction kernels, with
// the chunk region as the stacked triangles' buffer.
__device__ __forceinline__ void wy_climb(unsigned char *sm, const Layout &L, const F64Args &b,
                                         const int ldSd, const int leaf,
                                         const int worker_sum_nodes = kWorkerSumNodes) {
    climb_tree<false>(b, reinterpret_cast<double *>(sm + L.C), ldSd,
                      reinterpret_cast<double *>(sm + L.R), reinterpret_cast<double *>(sm + L.f),
                      reinterpret_cast<double *>(sm + L.seg),
                      reinterpret_cast<double *>(sm + L.tot),
                      reinterpret_cast<unsigned int *>(sm + L.flag), leaf, worker_sum_nodes);
}

// One matrix: CTA = leaf, then the tree.
template <typename Tin, int HB>
__global__ void __launch_bounds__(kThreads, HB == 2 ? 2 : 1)
    tsqr_mixed_wy_kernel(const WyArgs2 a, const __grid_constant__ CUtensorMap tmap) {
    extern __shared__ __align__(16) unsigned char sm_raw[];
    // the chunk region starts on a 1024-byte boundary (the 128-byte swizzle's period)
    unsigned char *sm = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(sm_raw) + 1023) & ~(uintptr_t)1023);
    constexpr int h = 128 * HB;
    const F64Args &b = a.base;
    const int n = b.n;
    const int NP = (n + kPw - 1) / kPw;
    const Layout L = layout(n, h);

    const int leaf = blockIdx.x;
    const int64_t u0 = ((int64_t)leaf * b.nunits) / b.nleaves;
    const int64_t u1 = ((int64_t)(leaf + 1) * b.nunits) / b.nleaves;
    const int64_t rbeg = u0 * b.unit;
    const int64_t rend = (u1 * b.unit < b.m) ? u1 * b.unit : b.m;
    // the update's mbarrier and tensor memory (released before the tree), the TMA's mbarriers
    uint64_t *bar = reinterpret_cast<uint64_t *>(sm + L.bar);
    uint32_t *tbase = reinterpret_cast<uint32_t *>(sm + L.bar + 8);
    uint64_t *tbar = reinterpret_cast<uint64_t *>(sm + L.bar + 16);
    const bool use_tma = a.tma != 0;
    if (threadIdx.x == 0) {
        tc::mbar_init(bar, 1);
        for (int k = 0; k < NP; ++k) tc::mbar_init(tbar + k, 1);
        tc::fence_mbar_init();
    }
    if (threadIdx.x < 32) {
        tc::tmem_alloc(tbase, tmem_cols(n, h));
        tc::tmem_relinquish();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    Tmem tm;
    tm.base = *tbase;
    tm.bar = bar;
    tm.phase = 0;
    tm.ok = true;
    tm.pending = false;
    Tma t{&tmap, -1, tbar, 0u, 0u, 0u};
    const bool ok = wy_leaf<Tin, HB>(sm, L, n, static_cast<const Tin *>(a.A), b.lda, rbeg, rend,
                                       a.vec4 != 0, tm, use_tma ? &t : nullptr, b.status);
    if (!ok) {
        // a tensor-core or TMA wait gave up: wait once more, bounded, for the mma and the loads
        // in flight, release the tensor memory and leave R unwritten
        if (threadIdx.x == 0) {
            if (tm.pending) tc::mbar_wait(bar, tm.phase, 1LL << 22);
            for (int k = 0; k < NP; ++k)
                if ((t.pend >> k) & 1u) tc::mbar_wait(tbar + k, (t.ppar >> k) & 1u, 1LL << 22);
        }
        __syncthreads();
        if (threadIdx.x < 32) tc::tmem_dealloc(tm.base, tmem_cols(n, h));
        return;
    }
    if (threadIdx.x < 32) tc::tmem_dealloc(tm.base, tmem_cols(n, h));
    __syncthreads();
    wy_climb(sm, L, b, a.ldSd, leaf);
}

// A varlen batch of mixed-precision problems (n <= 112), one persistent launch: every CTA takes
// (problem, leaf) items from the queue (largest first), folds the leaf's rows with thread
// copies and climbs that problem's tree; the chunk height h is the batch's.  The tensor
// memory (tcols columns, enough for the widest problem) and the update's mbarrier are held for
// the whole launch.  No CTA ever waits for another.
template <typename Tin, int HB>
__global__ void __launch_bounds__(kThreads, 1) tsqr_batched_wy_kernel(const BatchArgs bt,
                                                                      const int tcols) {
    extern __shared__ __align__(16) unsigned char sm_raw[];
    __shared__ uint64_t s_bar;
    __shared__ uint32_t s_tbase;
    __shared__ int s_item;
    unsigned char *sm = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(sm_raw) + 1023) & ~(uintptr_t)1023);
    constexpr int h = 128 * HB;
    if (threadIdx.x == 0) {
        tc::mbar_init(&s_bar, 1);
        tc::fence_mbar_init();
    }
    if (threadIdx.x < 32) {
        tc::tmem_alloc(&s_tbase, (uint32_t)tcols);
        tc::tmem_relinquish();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    Tmem tm;
    tm.base = s_tbase;
    tm.bar = &s_bar;
    tm.phase = 0;
    tm.ok = true;
    tm.pending = false;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_item = (int)atomicAdd(bt.queue, 1u);
        __syncthreads();
        const int it = s_item;
        if (it >= bt.nitems) break;
        const int2 w = bt.items[it];
        const BatchProblem P = bt.probs[w.x];
        const int n = P.n;
        const Layout L = layout(n, h);
        const int64_t rbeg = (int64_t)w.y * P.unit;
        const int64_t rend = (rbeg + P.unit < P.m) ? rbeg + P.unit : P.m;
        const Tin *A = static_cast<const Tin *>(P.A);
        const bool vec4 = sizeof(Tin) == 4 && (reinterpret_cast<uintptr_t>(A) % 16 == 0) &&
                          (P.lda % 4 == 0);
        if (!wy_leaf<Tin, HB>(sm, L, n, A, P.lda, rbeg, rend, vec4, tm, nullptr, bt.status))
            break;
        F64Args a{};
        a.A = nullptr;
        a.m = P.m;
        a.lda = P.lda;
        a.n = n;
        a.unit = P.unit;
        a.nunits = P.nunits;
        a.nleaves = P.nleaves;
        a.arity = P.arity;
        a.h = h;
        a.hs = h;
        a.blk = 1;
        a.vec = 1;
        a.ldS = P.ldS;
        a.slots = bt.slots + P.slot_off;
        a.counters = bt.counters + P.cnt_off;
        a.R = P.R;
        a.ldr = n;
        a.status = bt.status;
        wy_climb(sm, L, a, tree_ldsd(n, P.arity), w.y, 0);
    }
    if (tm.pending && threadIdx.x == 0) tc::mbar_wait(&s_bar, tm.phase, 1LL << 22);
    tc::fence_before_sync();
    __syncthreads();
    if (threadIdx.x < 32) tc::tmem_dealloc(s_tbase, (uint32_t)tcols);
}

}  // namespace wy

// ------------------------------------------------------------------------------------------
// Host side
// ------------------------------------------------------------------------------------------
namespace {
template <typename Tin>
const void *wy_fn(int hb) {
    switch (hb) {
        case 8: return (const void *)wy::tsqr_mixed_wy_kernel<Tin, 8>;
        case 6: return (const void *)wy::tsqr_mixed_wy_kernel<Tin, 6>;
        case 5: return (const void *)wy::tsqr_mixed_wy_kernel<Tin, 5>;
        case 4: return (const void *)wy::tsqr_mixed_wy_kernel<Tin, 4>;
        case 3: return (const void *)wy::tsqr_mixed_wy_kernel<Tin, 3>;
        default: return (const void *)wy::tsqr_mixed_wy_kernel<Tin, 2>;
    }
}
template <typename Tin>
void wy_launch_t(const wy::WyArgs2 &a, const CUtensorMap &tmap, int hb, size_t smem,
                 cudaStream_t stream) {
    const dim3 grid(a.base.nleaves), block(wy::kThreads);
    switch (hb) {
        case 8: wy::tsqr_mixed_wy_kernel<Tin, 8><<<grid, block, smem, stream>>>(a, tmap); break;
        case 6: wy::tsqr_mixed_wy_kernel<Tin, 6><<<grid, block, smem, stream>>>(a, tmap); break;
        case 5: wy::tsqr_mixed_wy_kernel<Tin, 5><<<grid, block, smem, stream>>>(a, tmap); break;
        case 4: wy::tsqr_mixed_wy_kernel<Tin, 4><<<grid, block, smem, stream>>>(a, tmap); break;
        case 3: wy::tsqr_mixed_wy_kernel<Tin, 3><<<grid, block, smem, stream>>>(a, tmap); break;
        default: wy::tsqr_mixed_wy_kernel<Tin, 2><<<grid, block, smem, stream>>>(a, tmap); break;
    }
}

// cuTensorMapEncodeTiled from the driver, looked up once through the runtime (the library
// does not link the driver library itself).
using EncodeTiledFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                   const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                   const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                   CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn encode_tiled() {
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
        cudaGetLastError();
    });
    return fn;
}

// A (FP32 or BF16) as a 2-D tensor (rows innermost, lda apart) read in boxes of 32 rows x 16
// columns with zero fill outside: FP32 with the 128-byte swizzle (the chunk layout), BF16
// unswizzled (staged, then widened).  False where the TMA cannot read A: a base that is not
// 16-byte aligned, lda x element size not a multiple of 16 bytes, or no encoder.
bool make_tensor_map(const void *A, bool bf16, int64_t m, int n, int64_t lda, CUtensorMap *tmap) {
    EncodeTiledFn enc = encode_tiled();
    const int64_t es = bf16 ? 2 : 4;
    // box rows are int coordinates up to a chunk past the last row
    if (!enc || reinterpret_cast<uintptr_t>(A) % 16 != 0 || (lda * es) % 16 != 0 || m < 1 ||
        m > 0x7fffffffLL - 4096)
        return false;
    const cuuint64_t dims[2] = {(cuuint64_t)m, (cuuint64_t)n};
    const cuuint64_t strides[1] = {(cuuint64_t)(lda * es)};
    const cuuint32_t box[2] = {32, 16};
    const cuuint32_t estr[2] = {1, 1};
    return enc(tmap, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2,
               const_cast<void *>(A), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
               bf16 ? CU_TENSOR_MAP_SWIZZLE_NONE : CU_TENSOR_MAP_SWIZZLE_128B,
               CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}
}  // namespace

// The layout plus 1024 bytes to align its base to the swizzle period.
size_t mixed_wy_smem_bytes(int n, int h) { return (size_t)wy::layout(n, h).total + 1024; }

// Whether an h-row chunk (h = 256, 384, 512, 640, 768 or 1024) fits the tensor memory for width n.
bool mixed_wy_tmem_fits(int n, int h) { return wy::tmem_need(n, h) <= 512; }

// Largest arity (<= 8) whose stacked FP64 triangles fit in the chunk region of an h-row leaf.
int mixed_wy_arity(int n, int h) {
    const int bytes = h * ((n + wy::kPw - 1) / wy::kPw) * 64;
    int k = 2;
    while (k < 8 && tree_ldsd(n, k + 1) * n * 8 <= bytes) ++k;
    return k;
}
int mixed_wy_ldsd(int n, int arity) { return tree_ldsd(n, arity); }
bool mixed_wy_tree_fits(int n, int h, int arity) {
    return tree_ldsd(n, arity) * n * 8 <= h * ((n + wy::kPw - 1) / wy::kPw) * 64;
}

cudaError_t mixed_wy_prepare(size_t smem_bytes) {
    const void *fns[12] = {wy_fn<float>(2), wy_fn<float>(3), wy_fn<float>(4), wy_fn<float>(5),
                           wy_fn<float>(6), wy_fn<float>(8), wy_fn<__nv_bfloat16>(2),
                           wy_fn<__nv_bfloat16>(3), wy_fn<__nv_bfloat16>(4),
                           wy_fn<__nv_bfloat16>(5), wy_fn<__nv_bfloat16>(6),
                           wy_fn<__nv_bfloat16>(8)};
    for (const void *f : fns) {
        cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem_bytes);
        if (e != cudaSuccess) return e;
        e = cudaFuncSetAttribute(f, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 (int)cudaSharedmemCarveoutMaxShared);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

int mixed_wy_blocks_per_sm(int h, size_t smem_bytes) {
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, wy_fn<float>(h / 128), wy::kThreads,
                                                      smem_bytes) != cudaSuccess)
        return 0;
    return nb;
}

cudaError_t mixed_wy_launch(const F64Args &base, const void *A, bool bf16, int ldSd,
                            size_t smem_bytes, cudaStream_t stream) {
    wy::WyArgs2 a;
    a.base = base;
    a.A = A;
    a.ldSd = ldSd;
    a.vec4 = !bf16 && (reinterpret_cast<uintptr_t>(A) % 16 == 0) && (base.lda % 4 == 0);
    // TMA loads where every leaf's rows are whole chunks (its last chunk then ends at A's last
    // row, where the TMA fills zeros)
    CUtensorMap tmap;
    std::memset(&tmap, 0, sizeof(tmap));
    a.tma = base.unit % base.h == 0 && make_tensor_map(A, bf16, base.m, base.n, base.lda, &tmap);
    const int hb = base.h / 128;
    if (bf16)
        wy_launch_t<__nv_bfloat16>(a, tmap, hb, smem_bytes, stream);
    else
        wy_launch_t<float>(a, tmap, hb, smem_bytes, stream);
    return cudaGetLastError();
}

// ---- the varlen batch (tsqr_r_batched's mixed problems up to 112 columns)
namespace {
const void *bwy_fn(bool bf16, int hb) {
    if (bf16) {
        switch (hb) {
            case 8: return (const void *)wy::tsqr_batched_wy_kernel<__nv_bfloat16, 8>;
            case 6: return (const void *)wy::tsqr_batched_wy_kernel<__nv_bfloat16, 6>;
            case 5: return (const void *)wy::tsqr_batched_wy_kernel<__nv_bfloat16, 5>;
            case 4: return (const void *)wy::tsqr_batched_wy_kernel<__nv_bfloat16, 4>;
            case 3: return (const void *)wy::tsqr_batched_wy_kernel<__nv_bfloat16, 3>;
            default: return (const void *)wy::tsqr_batched_wy_kernel<__nv_bfloat16, 2>;
        }
    }
    switch (hb) {
        case 8: return (const void *)wy::tsqr_batched_wy_kernel<float, 8>;
        case 6: return (const void *)wy::tsqr_batched_wy_kernel<float, 6>;
        case 5: return (const void *)wy::tsqr_batched_wy_kernel<float, 5>;
        case 4: return (const void *)wy::tsqr_batched_wy_kernel<float, 4>;
        case 3: return (const void *)wy::tsqr_batched_wy_kernel<float, 3>;
        default: return (const void *)wy::tsqr_batched_wy_kernel<float, 2>;
    }
}
}  // namespace

// Tensor-memory columns the batch kernel allocates for chunks of h rows and widths up to nmax.
int batched_wy_tmem_cols(int nmax, int h) { return (int)wy::tmem_cols(nmax, h); }

cudaError_t batched_wy_prepare(bool bf16, int h, size_t smem_bytes) {
    return set_smem_attrs(bwy_fn(bf16, h / 128), smem_bytes);
}

int batched_wy_blocks_per_sm(bool bf16, int h, size_t smem_bytes) {
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, bwy_fn(bf16, h / 128), wy::kThreads,
                                                      smem_bytes) != cudaSuccess)
        return 0;
    return nb;
}

cudaError_t batched_wy_launch(const BatchArgs &b, int grid, bool bf16, int h, int tcols,
                              size_t smem_bytes, cudaStream_t stream) {
    const dim3 g(grid), block(wy::kThreads);
    const int hb = h / 128;
#define TSQR_BWY(T, HBV) wy::tsqr_batched_wy_kernel<T, HBV><<<g, block, smem_bytes, stream>>>(b, tcols)
    if (bf16) {
        switch (hb) {
            case 8: TSQR_BWY(__nv_bfloat16, 8); break;
            case 6: TSQR_BWY(__nv_bfloat16, 6); break;
            case 5: TSQR_BWY(__nv_bfloat16, 5); break;
            case 4: TSQR_BWY(__nv_bfloat16, 4); break;
            case 3: TSQR_BWY(__nv_bfloat16, 3); break;
            default: TSQR_BWY(__nv_bfloat16, 2); break;
        }
    } else {
        switch (hb) {
            case 8: TSQR_BWY(float, 8); break;
            case 6: TSQR_BWY(float, 6); break;
            case 5: TSQR_BWY(float, 5); break;
            case 4: TSQR_BWY(float, 4); break;
            case 3: TSQR_BWY(float, 3); break;
            default: TSQR_BWY(float, 2); break;
        }
    }
#undef TSQR_BWY
    return cudaGetLastError();
}

}  // namespace tsqr

// Test hook (not part of the C ABI in include/tsqr.h; host only, no device call): the blocked
// leaf's shared-memory bytes for width n and chunk height h (out[0]), its tensor-memory columns
// (out[1]), and the most partial Z tiles any of its panels keeps (out[2]) against the slots
// (out[3]).  Returns 0.
extern "C" int tsqr_internal_wy_layout(int n, int h, int64_t *out) {
    out[0] = (int64_t)tsqr::mixed_wy_smem_bytes(n, h);
    out[1] = tsqr::wy::tmem_need(n, h);
    int most = 0;
    const int n8 = tsqr::wy::round_up_i(n, 8);
    for (int j0 = 0; j0 < n; j0 += tsqr::wy::kPw) {
        const int nt8 = (n8 - (j0 + tsqr::wy::kPw)) / 8;
        if (nt8 <= 0) continue;
        const int kg = tsqr::wy::kWarps / tsqr::wy::z_tile_sets(nt8);
        most = kg * nt8 > most ? kg * nt8 : most;
    }
    out[2] = most;
    out[3] = tsqr::wy::kMaxPartials;
    return 0;
}
