// Varlen batched TSQR in one persistent launch: every CTA takes (problem, leaf) work items from
// a global queue, folds the leaf and climbs that problem's binary tree (Fig. 1) with the same
// "last child to arrive combines" rule as the single-matrix kernel, then takes the next item.
// Items are ordered largest first, so the queue balances uneven problems.  No CTA ever waits
// for another.
#include "tsqr_fold.cuh"

namespace tsqr {

template <typename T, typename Tin>
__device__ __forceinline__ void batched_body(const BatchArgs &b) {
    __shared__ int s_item;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_item = (int)atomicAdd(b.queue, 1u);
        __syncthreads();
        const int it = s_item;
        if (it >= b.nitems) return;
        const int2 w = b.items[it];
        const BatchProblem P = b.probs[w.x];
        F64Args a;
        a.A = static_cast<const double *>(P.A);
        a.m = P.m;
        a.lda = P.lda;
        a.n = P.n;
        a.unit = P.unit;
        a.nunits = P.nunits;
        a.nleaves = P.nleaves;
        a.arity = P.arity;
        a.h = P.h;
        a.hs = P.hs;
        a.blk = P.blk;
        a.vec = P.vec;
        a.ldS = P.ldS;
        a.slots = b.slots + P.slot_off;
        a.counters = b.counters + P.cnt_off;
        a.R = P.R;
        a.ldr = P.n;
        a.status = b.status;
        const Tin *A = static_cast<const Tin *>(P.A);
        if constexpr (sizeof(T) == 8) {
            switch (P.blk) {
                case 4: leaf_tree_job<T, Tin, 4, 1, false>(a, A, P.ldS, P.ldS * P.n, w.y, 0); break;
                case 3: leaf_tree_job<T, Tin, 3, 1, false>(a, A, P.ldS, P.ldS * P.n, w.y, 0); break;
                case 2: leaf_tree_job<T, Tin, 2, 1, false>(a, A, P.ldS, P.ldS * P.n, w.y, 0); break;
                default: leaf_tree_job<T, Tin, 1, 1, false>(a, A, P.ldS, P.ldS * P.n, w.y, 0); break;
            }
        } else {
            const int ldSd = tree_ldsd(P.n, P.arity), sd = mixed_s_doubles_of(P.n, P.ldS, P.arity);
            switch (P.blk * 10 + P.vec) {
                case 44: leaf_tree_job<T, Tin, 4, 4, true>(a, A, ldSd, sd, w.y, 0); break;
                case 22: leaf_tree_job<T, Tin, 2, 2, true>(a, A, ldSd, sd, w.y, 0); break;
                default: leaf_tree_job<T, Tin, 1, 1, true>(a, A, ldSd, sd, w.y, 0); break;
            }
        }
    }
}

__global__ void __launch_bounds__(256, 1) tsqr_batched_f64_kernel(const BatchArgs b) {
    batched_body<double, double>(b);
}
// 12 bulk warps (wide batches; FP64 here, FP32 and BF16 below): their own 416-thread bound, so
// that the 4-warp kernels keep the 256-thread bound's register budget
__global__ void __launch_bounds__(416, 1) tsqr_batched_f64w_kernel(const BatchArgs b) {
    batched_body<double, double>(b);
}
__global__ void __launch_bounds__(256, 1) tsqr_batched_f32_kernel(const BatchArgs b) {
    batched_body<float, float>(b);
}
__global__ void __launch_bounds__(256, 1) tsqr_batched_bf16_kernel(const BatchArgs b) {
    batched_body<float, __nv_bfloat16>(b);
}
__global__ void __launch_bounds__(416, 1) tsqr_batched_f32w_kernel(const BatchArgs b) {
    batched_body<float, float>(b);
}
__global__ void __launch_bounds__(416, 1) tsqr_batched_bf16w_kernel(const BatchArgs b) {
    batched_body<float, __nv_bfloat16>(b);
}

namespace {
const void *batched_fn(int dtype) {
    switch (dtype) {
        case 0: return (const void *)tsqr_batched_f64_kernel;
        case 1: return (const void *)tsqr_batched_f32_kernel;
        case 2: return (const void *)tsqr_batched_bf16_kernel;
        case 3: return (const void *)tsqr_batched_f64w_kernel;
        case 4: return (const void *)tsqr_batched_f32w_kernel;
        default: return (const void *)tsqr_batched_bf16w_kernel;
    }
}
}  // namespace

// dtype: 0 FP64, 1 FP32 (mixed), 2 BF16 (mixed); 3, 4, 5 the same with 12 bulk warps; `warps`
// counts bulk warps (+1 reducer).
cudaError_t batched_prepare(int dtype, size_t smem_bytes) {
    return set_smem_attrs(batched_fn(dtype), smem_bytes);
}

int batched_blocks_per_sm(int dtype, int warps, size_t smem_bytes) {
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, batched_fn(dtype), (warps + 1) * 32,
                                                      smem_bytes) != cudaSuccess)
        return 0;
    return nb;
}

cudaError_t batched_launch(int dtype, const BatchArgs &b, int grid, int warps, size_t smem_bytes,
                           cudaStream_t stream) {
    const int threads = (warps + 1) * 32;
    switch (dtype) {
        case 0: tsqr_batched_f64_kernel<<<grid, threads, smem_bytes, stream>>>(b); break;
        case 1: tsqr_batched_f32_kernel<<<grid, threads, smem_bytes, stream>>>(b); break;
        case 2: tsqr_batched_bf16_kernel<<<grid, threads, smem_bytes, stream>>>(b); break;
        case 3: tsqr_batched_f64w_kernel<<<grid, threads, smem_bytes, stream>>>(b); break;
        case 4: tsqr_batched_f32w_kernel<<<grid, threads, smem_bytes, stream>>>(b); break;
        default: tsqr_batched_bf16w_kernel<<<grid, threads, smem_bytes, stream>>>(b); break;
    }
    return cudaGetLastError();
}

}  // namespace tsqr
