// Leaf + tree kernel launched over a range of leaves (tsqr_r_host): the leaves of one row piece
// of A, launched as soon as that piece has reached the device.  The pieces' leaves share one
// tree: a node's counter and slots persist across launches, and the last child to arrive,
// whichever launch it belongs to, combines (the root is reached in the last launch).
#include <cstdint>
#include <cuda_runtime.h>

#include "tsqr_fold.cuh"
#include "tsqr_internal.h"

namespace tsqr {

template <int B>
__global__ void __launch_bounds__(416, 1) tsqr_f64_piece_kernel(const F64Args a, const int leaf0) {
    leaf_tree_job<double, double, B, 1, B == 1>(a, a.A, a.ldS, a.ldS * a.n, leaf0 + blockIdx.x);
}

cudaError_t f64_piece_prepare(size_t smem_bytes) {
    cudaError_t e = set_smem_attrs(tsqr_f64_piece_kernel<4>, smem_bytes);
    if (e == cudaSuccess) e = set_smem_attrs(tsqr_f64_piece_kernel<3>, smem_bytes);
    if (e == cudaSuccess) e = set_smem_attrs(tsqr_f64_piece_kernel<2>, smem_bytes);
    if (e == cudaSuccess) e = set_smem_attrs(tsqr_f64_piece_kernel<1>, smem_bytes);
    return e;
}

cudaError_t f64_piece_launch(const F64Args &a, int leaf0, int leaves, int warps,
                             size_t smem_bytes, cudaStream_t stream) {
    const dim3 grid(leaves), block((warps + 1) * 32);
    switch (a.blk) {
        case 4: tsqr_f64_piece_kernel<4><<<grid, block, smem_bytes, stream>>>(a, leaf0); break;
        case 3: tsqr_f64_piece_kernel<3><<<grid, block, smem_bytes, stream>>>(a, leaf0); break;
        case 2: tsqr_f64_piece_kernel<2><<<grid, block, smem_bytes, stream>>>(a, leaf0); break;
        default: tsqr_f64_piece_kernel<1><<<grid, block, smem_bytes, stream>>>(a, leaf0); break;
    }
    return cudaGetLastError();
}

}  // namespace tsqr
