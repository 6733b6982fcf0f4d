// Mixed-precision kernels of libtsqr: FP32 or BF16 A, leaf Householder folds with FP32 bulk
// arithmetic (the fused reflector update and dot products), FP64 reflector norms, scalars,
// R and tree operator (Section 2's step 1 in FP32, step 2 in FP64).  The leaf chunk lives in
// shared memory as FP32; a BF16 A is widened exactly on load.
#include "tsqr_fold.cuh"

namespace tsqr {

template <typename Tin, int B, int V>
__global__ void __launch_bounds__(416, 1) tsqr_mixed_kernel(const MixedArgs a) {
    leaf_tree_job<float, Tin, B, V, true>(a.base, static_cast<const Tin *>(a.A), a.ldSd,
                                          a.s_doubles, blockIdx.x);
}

// Instances: FP32 or BF16 input x (block, vector) in {(8,4), (6,2), (4,4), (3,1), (2,2), (1,1)}.
namespace {
template <typename Tin>
const void *mixed_fn_t(int blk, int vec) {
    switch (blk * 10 + vec) {
        case 84: return (const void *)tsqr_mixed_kernel<Tin, 8, 4>;
        case 62: return (const void *)tsqr_mixed_kernel<Tin, 6, 2>;
        case 44: return (const void *)tsqr_mixed_kernel<Tin, 4, 4>;
        case 31: return (const void *)tsqr_mixed_kernel<Tin, 3, 1>;
        case 22: return (const void *)tsqr_mixed_kernel<Tin, 2, 2>;
        default: return (const void *)tsqr_mixed_kernel<Tin, 1, 1>;
    }
}
const void *mixed_fn(bool bf16, int blk, int vec) {
    return bf16 ? mixed_fn_t<__nv_bfloat16>(blk, vec) : mixed_fn_t<float>(blk, vec);
}
constexpr int kVariants[6][2] = {{8, 4}, {6, 2}, {4, 4}, {3, 1}, {2, 2}, {1, 1}};

template <typename Tin>
void launch_t(const MixedArgs &a, int threads, size_t smem, cudaStream_t stream) {
    const dim3 grid(a.base.nleaves);
    switch (a.base.blk * 10 + a.base.vec) {
        case 84: tsqr_mixed_kernel<Tin, 8, 4><<<grid, threads, smem, stream>>>(a); break;
        case 62: tsqr_mixed_kernel<Tin, 6, 2><<<grid, threads, smem, stream>>>(a); break;
        case 44: tsqr_mixed_kernel<Tin, 4, 4><<<grid, threads, smem, stream>>>(a); break;
        case 31: tsqr_mixed_kernel<Tin, 3, 1><<<grid, threads, smem, stream>>>(a); break;
        case 22: tsqr_mixed_kernel<Tin, 2, 2><<<grid, threads, smem, stream>>>(a); break;
        default: tsqr_mixed_kernel<Tin, 1, 1><<<grid, threads, smem, stream>>>(a); break;
    }
}
}  // namespace

int mixed_s_doubles(int n, int ldS) { return (ldS * n + 1) / 2; }

// `warps` counts bulk warps; the kernels launch one more, the reducer warp.
size_t mixed_smem_bytes(int n, int ldS, int warps) {
    return sizeof(double) * (size_t)smem_layout_s(n, mixed_s_doubles_of(n, ldS, 2), warps + 1).total;
}

cudaError_t mixed_prepare(size_t smem_bytes) {
    for (const auto &v : kVariants)
        for (int bf = 0; bf < 2; ++bf) {
            const cudaError_t e = set_smem_attrs(mixed_fn(bf != 0, v[0], v[1]), smem_bytes);
            if (e != cudaSuccess) return e;
        }
    return cudaSuccess;
}

int mixed_blocks_per_sm(int warps, size_t smem_bytes) {
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, mixed_fn(false, 6, 2), (warps + 1) * 32,
                                                      smem_bytes) != cudaSuccess)
        return 0;
    return nb;
}

cudaError_t mixed_launch(const MixedArgs &a, bool bf16, int warps, size_t smem_bytes,
                         cudaStream_t stream) {
    const int threads = (warps + 1) * 32;
    if (bf16)
        launch_t<__nv_bfloat16>(a, threads, smem_bytes, stream);
    else
        launch_t<float>(a, threads, smem_bytes, stream);
    return cudaGetLastError();
}

}  // namespace tsqr
