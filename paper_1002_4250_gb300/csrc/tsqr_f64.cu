// FP64 kernels of libtsqr: the leaf/tree kernel of TSQR (Section 2 with the trees of
// Section 1 and Fig. 1) and a single-node kernel for the operator qr(R1, R2) of Table 3.
#include "tsqr_fold.cuh"

namespace tsqr {

template <int B>
__global__ void __launch_bounds__(416, 1) tsqr_f64_kernel(const F64Args a) {
    // one row per lane (B = 1): the software-pipelined sweep hides the shared-memory latency
    // a single block per item exposes (measured +3% at n = 64); taller lanes keep the plain
    // loop, which measured faster there
    leaf_tree_job<double, double, B, 1, B == 1>(a, a.A, a.ldS, a.ldS * a.n, blockIdx.x);
}

// The FP64 leaf is instantiated for blocks of 1, 2, 3 and 4 rows (scalar accesses).
namespace {
const void *f64_fn(int blk) {
    switch (blk) {
        case 4: return (const void *)tsqr_f64_kernel<4>;
        case 3: return (const void *)tsqr_f64_kernel<3>;
        case 2: return (const void *)tsqr_f64_kernel<2>;
        default: return (const void *)tsqr_f64_kernel<1>;
    }
}
}  // namespace

// One tree node: R = qr(R1, R2) (Table 3), optionally sign-normalized.
__global__ void __launch_bounds__(288, 1) tsqr_f64_combine_kernel(int n, const double *R1, int64_t ld1,
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
    fold_stack(S, ldS, 1, Rp, smem + L.f, smem + L.seg, smem + L.tot + seg_stride(n), n);
    if (normalize)
        store_normalized(Rp, n, R, ldr, status);
    else
        store_packed(Rp, n, R, ldr);
}

// ------------------------------------------------------------------------------------------
// host-side launchers
// ------------------------------------------------------------------------------------------
// `warps` counts the leaf kernel's bulk warps; it launches one more, the reducer warp.
size_t f64_smem_bytes(int n, int hs, int ldS, int warps) {
    return sizeof(double) * (size_t)smem_layout(n, hs, ldS, warps + 1).total;
}

cudaError_t f64_prepare(size_t smem_bytes) {
    for (int b = 1; b <= 4; ++b) {
        const cudaError_t e = set_smem_attrs(f64_fn(b), smem_bytes);
        if (e != cudaSuccess) return e;
    }
    return set_smem_attrs(tsqr_f64_combine_kernel, smem_bytes);
}

int f64_blocks_per_sm(int warps, size_t smem_bytes) {
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, f64_fn(3), (warps + 1) * 32,
                                                      smem_bytes) != cudaSuccess)
        return 0;
    return nb;
}

cudaError_t f64_launch(const F64Args &a, int warps, size_t smem_bytes, cudaStream_t stream) {
    const dim3 grid(a.nleaves), block((warps + 1) * 32);
    switch (a.blk) {
        case 4: tsqr_f64_kernel<4><<<grid, block, smem_bytes, stream>>>(a); break;
        case 3: tsqr_f64_kernel<3><<<grid, block, smem_bytes, stream>>>(a); break;
        case 2: tsqr_f64_kernel<2><<<grid, block, smem_bytes, stream>>>(a); break;
        default: tsqr_f64_kernel<1><<<grid, block, smem_bytes, stream>>>(a); break;
    }
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
