// Declarations shared by the host API and the kernels of libtsqr (not part of the C ABI).
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "tsqr.h"
#include "tsqr_f64.cuh"

namespace tsqr {

constexpr int kStatusNonfiniteBit = 1;
constexpr int kStatusTimeoutBit = 2;  // a bounded device-side wait gave up

// Dynamic shared-memory size of a kernel, with the whole unified L1/shared array given to
// shared memory (the kernels keep their working set there and read A past L1).
template <typename F>
inline cudaError_t set_smem_attrs(F *fn, size_t smem_bytes) {
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem_bytes);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout,
                                (int)cudaSharedmemCarveoutMaxShared);
}

// FP64 path (tsqr_f64.cu)
size_t f64_smem_bytes(int n, int hs, int ldS, int warps);
cudaError_t f64_prepare(size_t smem_bytes);
int f64_blocks_per_sm(int warps, size_t smem_bytes);
cudaError_t f64_launch(const F64Args &a, int warps, size_t smem_bytes, cudaStream_t stream);
cudaError_t f64_combine_launch(int n, const double *R1, int64_t ld1, const double *R2,
                               int64_t ld2, double *R, int64_t ldr, int normalize, int warps,
                               int ldS, int hs, size_t smem_bytes, int *status,
                               cudaStream_t stream);

// Mixed path (tsqr_mixed.cu); `warps` counts bulk warps as for the FP64 path.
int mixed_s_doubles(int n, int ldS);
size_t mixed_smem_bytes(int n, int ldS, int warps);
cudaError_t mixed_prepare(size_t smem_bytes);
int mixed_blocks_per_sm(int warps, size_t smem_bytes);
cudaError_t mixed_launch(const MixedArgs &a, bool bf16, int warps, size_t smem_bytes,
                         cudaStream_t stream);

// Blocked mixed path (tsqr_mixed_wy.cu): panels of 16 columns, compact WY updates on the
// tensor cores; n <= kMixedWyMaxN, chunks of h = 256, 384, 512, 640, 768 or 1024 rows, 8 warps.
constexpr int kMixedWyMaxN = 112;
constexpr int kMixedWyHeights[6] = {1024, 768, 640, 512, 384, 256};  // tallest first
size_t mixed_wy_smem_bytes(int n, int h);
bool mixed_wy_tmem_fits(int n, int h);
int mixed_wy_arity(int n, int h);
bool mixed_wy_tree_fits(int n, int h, int arity);
cudaError_t mixed_wy_prepare(size_t smem_bytes);
int mixed_wy_blocks_per_sm(int h, size_t smem_bytes);
cudaError_t mixed_wy_launch(const F64Args &base, const void *A, bool bf16, int ldSd,
                            size_t smem_bytes, cudaStream_t stream);
// The same leaf for a varlen batch (one persistent launch; chunks of h rows for every problem;
// tensor memory of tcols columns held by every CTA).
int batched_wy_tmem_cols(int nmax, int h);
cudaError_t batched_wy_prepare(bool bf16, int h, size_t smem_bytes);
int batched_wy_blocks_per_sm(bool bf16, int h, size_t smem_bytes);
cudaError_t batched_wy_launch(const BatchArgs &b, int grid, bool bf16, int h, int tcols,
                              size_t smem_bytes, cudaStream_t stream);

// Batched path (tsqr_batched.cu); dtype 0 FP64, 1 FP32, 2 BF16; `warps` counts bulk warps.
cudaError_t batched_prepare(int dtype, size_t smem_bytes);
int batched_blocks_per_sm(int dtype, int warps, size_t smem_bytes);
cudaError_t batched_launch(int dtype, const BatchArgs &b, int grid, int warps, size_t smem_bytes,
                           cudaStream_t stream);

// Thin QR (tsqr_qr.cu)
struct QTreeArgs;
struct QLeafArgs;
size_t q_leaf_smem_bytes(int n, int qn, int ldS, int warps);
size_t q_tree_smem_bytes(int n, int arity, int qg);
cudaError_t qr_prepare(size_t factor_smem, size_t leaf_smem, size_t tree_smem);
cudaError_t qr_factor_launch(const F64Args &a, int warps, size_t smem_bytes, cudaStream_t stream);
cudaError_t q_tree_launch(const QTreeArgs &a, int grid, size_t smem_bytes, cudaStream_t stream);
cudaError_t q_leaf_launch(const QLeafArgs &a, int blk, int warps, size_t smem_bytes,
                          cudaStream_t stream);

// The AUTO plan of tsqr_r's one reduction as kernel arguments (tsqr_api.cu); A, R, workspace
// and status pointers are left for the caller.  *plan receives its public form.
tsqr_status_t f64_auto_args(int64_t m, int n, F64Args *a, int *warps, size_t *smem,
                            int64_t *nodes, tsqr_plan_t *plan);

// What tsqr_last_launch_count and tsqr_last_plan report for the calling thread (tsqr_api.cu),
// for entry points outside tsqr_api.cu.
void set_last_call(int launches, const tsqr_plan_t &plan);

// The bounded-wait test kernel (tsqr_selftest.cu): one CTA waits, at most `limit` polls, on an
// mbarrier that its own arrival completes (arrive != 0) or that nothing completes; a wait that
// runs out sets kStatusTimeoutBit in *status.  *result: 1 if the wait succeeded.  0 or 3
// (launch error).
int wait_selftest_launch(long long limit, int arrive, int *status, int *result,
                         cudaStream_t stream);

}  // namespace tsqr
