// tsqr_r_noalloc: the FP64 R factor with the reduction tree's scratch in a fixed,
// statically allocated device array, for callers that cannot allocate device memory at call
// time.  It runs tsqr_r's kernel on the AUTO plan's one-reduction partition (never the panels).
// The device address of the array is looked up once per device and kept for the life of the
// process; it is not valid after the device has been reset.
#include <mutex>

#include "tsqr.h"
#include "tsqr_internal.h"

namespace {

// Scratch for the reduction tree: one arrival counter and one n x n FP64 slot per tree node.
// It lives in every GPU that loads the library, for the life of the process.
constexpr size_t kScratchBytes = (size_t)TSQR_NOALLOC_SCRATCH_BYTES;
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_scratch_dev[kMaxDevices] = {};

// Device address of g_scratch on the current device, looked up once per device.
tsqr_status_t scratch_address(void **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return TSQR_ERR_CUDA;
    if (dev < 0 || dev >= kMaxDevices) return TSQR_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_dev[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) return TSQR_ERR_CUDA;
        g_scratch_dev[dev] = p;
    }
    *out = g_scratch_dev[dev];
    return TSQR_SUCCESS;
}

inline size_t align256(size_t x) { return (x + 255) / 256 * 256; }

}  // namespace

extern "C" tsqr_status_t tsqr_r_noalloc(const double *A, int64_t m, int64_t n, int64_t lda,
                                        double *R, int64_t ldr, tsqr_stream_t stream) {
    tsqr::set_last_call(0, tsqr_plan_t{});
    if (m < 0 || n < 0 || lda < (m > 1 ? m : 1) || ldr < (n > 1 ? n : 1))
        return TSQR_ERR_INVALID_ARG;
    if (n > TSQR_MAX_N) return TSQR_ERR_UNSUPPORTED;
    if (n == 0) return TSQR_SUCCESS;
    if (!R || (m > 0 && !A)) return TSQR_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (m == 0)
        return cudaMemset2DAsync(R, (size_t)ldr * sizeof(double), 0, (size_t)n * sizeof(double),
                                 (size_t)n, s) == cudaSuccess ? TSQR_SUCCESS : TSQR_ERR_CUDA;
    tsqr::F64Args a;
    int warps = 0;
    size_t smem = 0;
    int64_t nodes = 0;
    tsqr_plan_t plan{};
    tsqr_status_t st = tsqr::f64_auto_args(m, (int)n, &a, &warps, &smem, &nodes, &plan);
    if (st != TSQR_SUCCESS) return st;
    const size_t cnt_bytes = align256((size_t)nodes * sizeof(unsigned int));
    const size_t need = cnt_bytes + (size_t)nodes * (size_t)n * (size_t)n * sizeof(double);
    if (need > kScratchBytes) return TSQR_ERR_UNSUPPORTED;  // the tree does not fit the array
    void *base = nullptr;
    st = scratch_address(&base);
    if (st != TSQR_SUCCESS) return st;
    if (tsqr::f64_prepare(smem) != cudaSuccess) return TSQR_ERR_CUDA;
    a.A = A;
    a.lda = lda;
    a.counters = (unsigned int *)base;
    a.slots = (double *)((char *)base + cnt_bytes);
    a.R = R;
    a.ldr = ldr;
    a.status = nullptr;
    // the counters must start at zero; the slots are always written before they are read
    if (cudaMemsetAsync(a.counters, 0, (size_t)nodes * sizeof(unsigned int), s) != cudaSuccess)
        return TSQR_ERR_CUDA;
    if (tsqr::f64_launch(a, warps, smem, s) != cudaSuccess) return TSQR_ERR_CUDA;
    tsqr::set_last_call(1, plan);
    return TSQR_SUCCESS;
}
