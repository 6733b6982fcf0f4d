// Test hook (not part of the C ABI in include/tsqr.h): evaluates the reflector's scalar
// routines recip_sqrt and recip on device so that the tests can compare them with CUDA's rsqrt
// and reciprocal.
#include "tsqr_fold.cuh"

namespace {

__global__ void scalar_selftest_kernel(int64_t count, const double *x, double *out_rsqrt,
                                       double *out_recip) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x) {
        out_rsqrt[i] = tsqr::recip_sqrt(fabs(x[i]));
        out_recip[i] = tsqr::recip(x[i]);
    }
}

}  // namespace

extern "C" int tsqr_internal_scalar_selftest(int64_t count, const double *x, double *out_rsqrt,
                                             double *out_recip, void *stream) {
    if (count <= 0) return 0;
    scalar_selftest_kernel<<<152, 256, 0, (cudaStream_t)stream>>>(count, x, out_rsqrt, out_recip);
    return cudaGetLastError() == cudaSuccess ? 0 : 3;
}
