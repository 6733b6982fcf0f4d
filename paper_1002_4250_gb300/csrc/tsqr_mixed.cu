// Mixed-precision kernels of libtsqr: FP32 or BF16 A, leaf Householder folds with FP32 bulk
// arithmetic (the fused reflector update and dot products), FP64 reflector norms, scalars,
// R and tree operator (Section 2's step 1 in FP32, step 2 in FP64).  The leaf chunk lives in
// shared memory as FP32; a BF16 A is widened exactly on load.
#include "tsqr_fold.cuh"

namespace tsqr {

__global__ void __launch_bounds__(256, 1) tsqr_mixed_f32_kernel(const MixedArgs a) {
    leaf_tree_job<float, float>(a.base, static_cast<const float *>(a.A), a.ldSd, a.s_doubles,
                                blockIdx.x);
}

__global__ void __launch_bounds__(256, 1) tsqr_mixed_bf16_kernel(const MixedArgs a) {
    leaf_tree_job<float, __nv_bfloat16>(a.base, static_cast<const __nv_bfloat16 *>(a.A), a.ldSd,
                                        a.s_doubles, blockIdx.x);
}

int mixed_ldsd(int n) { return mixed_ldsd_of(n); }

int mixed_s_doubles(int n, int ldS) { return mixed_s_doubles_of(n, ldS); }

// `warps` counts bulk warps; the kernels launch one more, the reducer warp.
size_t mixed_smem_bytes(int n, int ldS, int warps) {
    return sizeof(double) * (size_t)smem_layout_s(n, mixed_s_doubles(n, ldS), warps + 1).total;
}

cudaError_t mixed_prepare(size_t smem_bytes) {
    cudaError_t e = cudaFuncSetAttribute(tsqr_mixed_f32_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem_bytes);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(tsqr_mixed_bf16_kernel,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes);
}

int mixed_blocks_per_sm(int warps, size_t smem_bytes) {
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, tsqr_mixed_f32_kernel, (warps + 1) * 32,
                                                      smem_bytes) != cudaSuccess)
        return 0;
    return nb;
}

cudaError_t mixed_launch(const MixedArgs &a, bool bf16, int warps, size_t smem_bytes,
                         cudaStream_t stream) {
    if (bf16)
        tsqr_mixed_bf16_kernel<<<a.base.nleaves, (warps + 1) * 32, smem_bytes, stream>>>(a);
    else
        tsqr_mixed_f32_kernel<<<a.base.nleaves, (warps + 1) * 32, smem_bytes, stream>>>(a);
    return cudaGetLastError();
}

}  // namespace tsqr
