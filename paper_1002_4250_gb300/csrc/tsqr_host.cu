// Streaming leaf kernel (tsqr_r_host): one launch whose leaves fold A's work units while A is
// still being copied from host memory.  The copy stream copies A in P row pieces and sets
// flags[q] after piece q; leaf l takes units l, l + L, l + 2L, ... (L leaves), so every leaf
// starts on the first piece and all leaves move through the pieces together.  Before a chunk
// from a new piece is loaded the CTA waits for that piece's flag (a bounded wait: on timeout it
// records kStatusTimeoutBit and returns); the next chunk is prefetched during the current fold
// only if its piece has already arrived.  The leaves then climb the usual k-ary tree.
// TSQR allows any assignment of rows to leaves (Section 2: each row block is factorized on its
// own), so the round-robin units give a valid R; its rounding differs from tsqr_r's.
#include <cstdint>
#include <cuda_runtime.h>

#include "tsqr_fold.cuh"
#include "tsqr_internal.h"

namespace tsqr {

namespace {


// Piece 0 holds work units [0, first): the leaves' first round, so that every leaf can start
// after the smallest copy.  Piece q >= 1 holds [first + (q-1) R / (P-1), first + q R / (P-1)),
// R = nunits - first.
__device__ __forceinline__ int piece_of(const int64_t u, const int64_t nunits, const int P,
                                        const int64_t first) {
    if (u < first || P == 1) return 0;
    const int64_t r = u - first, R = nunits - first;
    const int Q = P - 1;
    int q = (int)((r * Q) / R);
    while (q + 1 < Q && ((int64_t)(q + 1) * R) / Q <= r) ++q;
    while (q > 0 && ((int64_t)q * R) / Q > r) --q;
    return 1 + q;
}

__device__ __forceinline__ unsigned int load_flag(const unsigned int *p) {
    return *reinterpret_cast<const volatile unsigned int *>(p);
}

// Whether piece q has arrived, as the whole CTA sees it; with `wait`, thread 0 polls until it
// has, at most wait_iters times with a 256 ns sleep between polls.  The copy's writes precede the flag's in stream order, and A is read through
// L2 (cp.async.cg), so the data is there once the flag is.
__device__ __forceinline__ bool piece_arrived(const unsigned int *flags, const int q,
                                              const bool wait, const long long wait_iters,
                                              unsigned int *sflag) {
    if (threadIdx.x == 0) {
        unsigned int ok = load_flag(flags + q) != 0u;
        for (long long it = 0; wait && !ok && it < wait_iters; ++it) {
            __nanosleep(256);
            ok = load_flag(flags + q) != 0u;
        }
        __threadfence();
        sflag[0] = ok;
    }
    __syncthreads();
    const bool ok = sflag[0] != 0u;
    __syncthreads();
    return ok;
}

__device__ __forceinline__ Chunk<double> unit_chunk(const F64Args &a, const int64_t u) {
    Chunk<double> c;
    const int64_t r0 = u * a.unit;
    c.src = a.A + r0;
    c.lda = a.lda;
    c.rows = (int)((a.m - r0 < a.unit) ? a.m - r0 : a.unit);
    return c;
}

}  // namespace

template <int B>
__global__ void __launch_bounds__(416, 1)
    tsqr_f64_stream_kernel(const F64Args a, const unsigned int *flags, const int pieces,
                           const int64_t first, const long long wait_iters) {
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
    unsigned int *pflag = reinterpret_cast<unsigned int *>(smem + L.scal + 1);
    for (int i = threadIdx.x; i < n * (n + 1) / 2; i += blockDim.x) Rp[i] = 0.0;
    const int leaf = blockIdx.x;
    const int64_t stride = a.nleaves;
    int64_t u = leaf;
    if (u < a.nunits) {
        if (!piece_arrived(flags, piece_of(u, a.nunits, pieces, first), true, wait_iters, pflag)) {
            if (threadIdx.x == 0 && a.status) atomicOr(a.status, kStatusTimeoutBit);
            return;
        }
        const Chunk<double> c0 = unit_chunk(a, u);
        for (int col = 0; col < n; ++col) load_column(S, a.ldS, a.hs, c0, col);
        cp_async_wait_all();
        __syncthreads();
        for (;;) {
            const int64_t nx = u + stride;
            const bool have = nx < a.nunits;
            const bool pre = have && piece_arrived(flags, piece_of(nx, a.nunits, pieces, first), false, 0,
                                                  pflag);
            Chunk<double> next;
            next.src = nullptr;
            next.lda = a.lda;
            next.rows = 0;
            if (pre) next = unit_chunk(a, nx);
            fold_leaf<double, double, B, 1, B == 1>(S, a.ldS, a.hs, Rp, f, f, seg, tot, npart, n,
                                                   next);
            if (!have) break;
            if (!pre) {
                if (!piece_arrived(flags, piece_of(nx, a.nunits, pieces, first), true, wait_iters,
                                   pflag)) {
                    if (threadIdx.x == 0 && a.status) atomicOr(a.status, kStatusTimeoutBit);
                    return;
                }
                const Chunk<double> cn = unit_chunk(a, nx);
                for (int col = 0; col < n; ++col) load_column(S, a.ldS, a.hs, cn, col);
            }
            cp_async_wait_all();
            __syncthreads();
            u = nx;
        }
    }
    climb_tree<false>(a, S, a.ldS, Rp, f, seg, tot, flag, leaf);
}

cudaError_t f64_stream_prepare(size_t smem_bytes) {
    cudaError_t e = set_smem_attrs(tsqr_f64_stream_kernel<4>, smem_bytes);
    if (e == cudaSuccess) e = set_smem_attrs(tsqr_f64_stream_kernel<3>, smem_bytes);
    if (e == cudaSuccess) e = set_smem_attrs(tsqr_f64_stream_kernel<2>, smem_bytes);
    if (e == cudaSuccess) e = set_smem_attrs(tsqr_f64_stream_kernel<1>, smem_bytes);
    return e;
}

// wait_iters: polls per wait (1 << 23 in tsqr_r_host: seconds before a timeout)
cudaError_t f64_stream_launch(const F64Args &a, const unsigned int *flags, int pieces,
                              int64_t first, int warps, size_t smem_bytes, long long wait_iters,
                              cudaStream_t stream) {
    const dim3 grid(a.nleaves), block((warps + 1) * 32);
    switch (a.blk) {
        case 4:
            tsqr_f64_stream_kernel<4><<<grid, block, smem_bytes, stream>>>(a, flags, pieces, first, wait_iters);
            break;
        case 3:
            tsqr_f64_stream_kernel<3><<<grid, block, smem_bytes, stream>>>(a, flags, pieces, first, wait_iters);
            break;
        case 2:
            tsqr_f64_stream_kernel<2><<<grid, block, smem_bytes, stream>>>(a, flags, pieces, first, wait_iters);
            break;
        default:
            tsqr_f64_stream_kernel<1><<<grid, block, smem_bytes, stream>>>(a, flags, pieces, first, wait_iters);
            break;
    }
    return cudaGetLastError();
}

}  // namespace tsqr
