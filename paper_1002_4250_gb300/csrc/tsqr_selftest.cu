// Test hooks (not part of the C ABI in include/tsqr.h): the reflector's scalar routines
// recip_sqrt and recip on device, so that the tests can compare them with CUDA's rsqrt and
// reciprocal; and the kernels' bounded mbarrier wait, made to run out.
#include "tsqr_fold.cuh"
#include "tsqr_tc.cuh"

namespace {

__global__ void scalar_selftest_kernel(int64_t count, const double *x, double *out_rsqrt,
                                       double *out_recip) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x) {
        out_rsqrt[i] = tsqr::recip_sqrt(fabs(x[i]));
        out_recip[i] = tsqr::recip(x[i]);
    }
}

// One CTA waits, bounded by `limit` polls, on an mbarrier of count 1 as the leaf kernels wait
// for their tensor-core commits and TMA loads.  With `arrive` the CTA's own arrival completes
// the phase and the wait succeeds; without, nothing arrives, the wait gives up and, as the
// kernels do, sets the timeout bit of the status word.  result: 1 if the wait succeeded.
__global__ void wait_selftest_kernel(long long limit, int arrive, int *status, int *result) {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        tsqr::tc::mbar_init(&bar, 1);
        tsqr::tc::fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (arrive)
            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(tsqr::tc::smem_u32(&bar))
                         : "memory");
        const bool ok = tsqr::tc::mbar_wait(&bar, 0, limit);
        if (!ok && status) atomicOr(status, tsqr::kStatusTimeoutBit);
        *result = ok ? 1 : 0;
    }
}

}  // namespace

namespace tsqr {
int wait_selftest_launch(long long limit, int arrive, int *status, int *result,
                         cudaStream_t stream) {
    wait_selftest_kernel<<<1, 32, 0, stream>>>(limit, arrive, status, result);
    return cudaGetLastError() == cudaSuccess ? 0 : 3;
}
}  // namespace tsqr

extern "C" int tsqr_internal_scalar_selftest(int64_t count, const double *x, double *out_rsqrt,
                                             double *out_recip, void *stream) {
    if (count <= 0) return 0;
    scalar_selftest_kernel<<<152, 256, 0, (cudaStream_t)stream>>>(count, x, out_rsqrt, out_recip);
    return cudaGetLastError() == cudaSuccess ? 0 : 3;
}
