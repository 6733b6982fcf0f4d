// Measured pipe peaks of the GPU libtsqr runs on, for the roofline denominators of its kernels:
// FP64 DFMA, FP32 FFMA, TF32 through the warp-level mma (m16n8k8) and through the 5th-generation
// tensor core (tcgen05.mma kind::tf32, M = 128, N = 256), and BF16 through tcgen05 (kind::f16),
// the last as a cross-check against a library GEMM's throughput.  Each kernel keeps every SM
// busy with independent work for tens of milliseconds and is timed with CUDA events.
//
// Also a self-test hook of the tcgen05 operand layouts the mixed-precision leaf uses: an
// MN-major, 128-byte-swizzled A (32-row boxes of 16 columns, as a TMA box load lays them out)
// times a K-major, unswizzled B (8 x 16-byte core matrices), D in tensor memory.
#include <cstdint>
#include <cuda_runtime.h>

#include "tsqr.h"
#include "tsqr_internal.h"
#include "tsqr_tc.cuh"

namespace tsqr {
namespace {

constexpr int kChains = 8;

__global__ void __launch_bounds__(256) dfma_peak_kernel(double *sink, int iters, double b,
                                                        double c) {
    double acc[kChains];
#pragma unroll
    for (int i = 0; i < kChains; ++i) acc[i] = threadIdx.x * 1e-3 + i;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < kChains; ++i) acc[i] = fma(acc[i], b, c);
    }
    double s = 0.0;
#pragma unroll
    for (int i = 0; i < kChains; ++i) s += acc[i];
    if (s == 1234.5678) sink[threadIdx.x] = s;  // never true; keeps the chains live
}

__global__ void __launch_bounds__(256) ffma_peak_kernel(float *sink, int iters, float b,
                                                        float c) {
    float acc[kChains];
#pragma unroll
    for (int i = 0; i < kChains; ++i) acc[i] = threadIdx.x * 1e-3f + i;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < kChains; ++i) acc[i] = fmaf(acc[i], b, c);
    }
    float s = 0.0f;
#pragma unroll
    for (int i = 0; i < kChains; ++i) s += acc[i];
    if (s == 1234.5678f) sink[threadIdx.x] = s;
}

__global__ void __launch_bounds__(256) mma_tf32_peak_kernel(float *sink, int iters) {
    float a[4], b[2];
#pragma unroll
    for (int i = 0; i < 4; ++i) a[i] = tc::to_tf32(0.01f * (threadIdx.x + i));
    b[0] = tc::to_tf32(0.5f);
    b[1] = tc::to_tf32(0.25f);
    float d[kChains][4] = {};
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < kChains; ++i) tc::mma_m16n8k8(d[i], a, b);
    }
    float s = 0.0f;
#pragma unroll
    for (int i = 0; i < kChains; ++i) s += d[i][0] + d[i][1] + d[i][2] + d[i][3];
    if (s == 1234.5678f) sink[threadIdx.x] = s;
}

// One CTA per SM, 128 threads: thread 0 issues `iters` tcgen05.mma of M = 128, N = 256 and
// K = 8 (TF32) or 16 (BF16) on operands in shared memory (K-major, no swizzle: 8-row x
// 16-byte core matrices, 128 bytes apart along K and 256 bytes apart along M/N), then one
// commit; the tensor core executes one thread's mma in order and stalls its issue when its
// queue is full, so no throttling is needed.  The wait for the commit is bounded: on giving up
// the CTA records kStatusTimeoutBit.  TMEM: 256 columns.
constexpr int kPeakN = 256;

template <bool kBF16>
__global__ void __launch_bounds__(128, 1) tc05_peak_kernel(float *sink, int iters, int *status,
                                                           long long wait_limit) {
    __shared__ __align__(1024) uint32_t a_s[128 * 8];    // 128 x 32 bytes
    __shared__ __align__(1024) uint32_t b_s[kPeakN * 8]; // 256 x 32 bytes
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t tbase;
    for (int i = threadIdx.x; i < 128 * 8; i += blockDim.x)
        a_s[i] = kBF16 ? 0x3c003c00u : __float_as_uint(tc::to_tf32(0.0078125f * (i % 7)));
    for (int i = threadIdx.x; i < kPeakN * 8; i += blockDim.x)
        b_s[i] = kBF16 ? 0x3c803c80u : __float_as_uint(tc::to_tf32(0.0078125f * (i % 5)));
    if (threadIdx.x == 0) {
        tc::mbar_init(&bar, 1);
        tc::fence_mbar_init();
    }
    if (threadIdx.x < 32) {
        tc::tmem_alloc(&tbase, kPeakN);
        tc::tmem_relinquish();
    }
    tc::fence_proxy_async();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t taddr = tbase;
    bool ok = true;
    if (threadIdx.x == 0) {
        const uint64_t ad = tc::smem_desc(tc::smem_u32(a_s), 128, 256, tc::kSwNone);
        const uint64_t bd = tc::smem_desc(tc::smem_u32(b_s), 128, 256, tc::kSwNone);
        const uint32_t id = tc::instr_desc(kBF16 ? tc::kFmtBF16 : tc::kFmtTF32, 128, kPeakN,
                                           false, false);
        for (int it = 0; it < iters; ++it) {
            if (kBF16)
                tc::mma_f16(taddr, ad, bd, id, it > 0);
            else
                tc::mma_tf32(taddr, ad, bd, id, it > 0);
        }
        tc::mma_commit(&bar);
        ok = tc::mbar_wait(&bar, 0, wait_limit);
        if (!ok && status) atomicOr(status, kStatusTimeoutBit);
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    // every lane of the first warp reads one accumulator column (keeps the work live)
    if (threadIdx.x < 32) {
        float v[8];
        tc::tmem_ld8(taddr, v);
        tc::tmem_ld_wait();
        if (v[0] == 1234.5678f) sink[threadIdx.x] = v[1];
    }
    tc::fence_before_sync();
    __syncthreads();
    if (threadIdx.x < 32) tc::tmem_dealloc(taddr, kPeakN);
}

// ------------------------------------------------------------------------------------------
// tcgen05 layout self-test: D (128 x N, FP32) = A (128 x 16) * B (16 x N), TF32 inputs that
// are small integers (exact): A(i, k) = ((7 i + 3 k) mod 11) - 5, B(k, c) = ((5 k + 2 c) mod 7)
// - 3.  B is K-major, unswizzled: core matrix (c / 8, k / 4) at (c / 8) 512 + (k / 4) 128 bytes,
// row c mod 8 at 16 bytes each.  A by `variant`:
//   0: K-major, unswizzled: core matrix (i / 8, k / 4) at (i / 8) 512 + (k / 4) 128, row i mod 8
//      at 16 bytes each (LBO 128 along K, SBO 512 along M);
//   1: K-major, 128-byte swizzle: row i one 128-byte line at (i / 8) 1024 + (i mod 8) 128, unit
//      (k / 4) XOR (i mod 8) (SBO 1024 between 8-row groups; the second K step starts 32 bytes
//      in);
//   2: A in tensor memory (row i in lane i, K along 16 columns after D's), written by the
//      threads with tcgen05.st (the form the blocked mixed leaf's update uses).
// The A region is 16384 bytes, the largest extent of any variant (variant 1: 16 groups of 1024
// bytes), and B follows it.  Before the MMAs every D entry is set to -12345 (tcgen05.st), so a D
// that comes back as that value was never written.  Two MMAs (K = 8 each); D goes to global
// memory, row-major.
// ------------------------------------------------------------------------------------------
constexpr int kSelftestARegion = 16384;
__device__ __forceinline__ int a_off(int variant, int i, int k) {
    if (variant == 0) return (i / 8) * 512 + (k / 4) * 128 + (i % 8) * 16 + (k % 4) * 4;
    return (i / 8) * 1024 + (i % 8) * 128 + (((k / 4) ^ (i % 8)) << 4) + (k % 4) * 4;
}

__global__ void __launch_bounds__(128, 1) tc05_layout_selftest_kernel(float *D, int N, int variant,
                                                                      int *status,
                                                                      long long wait_limit) {
    extern __shared__ __align__(16) unsigned char dyn_raw[];
    // the 128-byte swizzle pattern repeats every 1024 bytes: operands start on that boundary
    unsigned char *dyn = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(dyn_raw) + 1023) & ~(uintptr_t)1023);
    unsigned char *a_s = dyn;                           // kSelftestARegion bytes
    unsigned char *b_s = dyn + kSelftestARegion;        // (N / 8) x 512 bytes
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t tbase;
    __shared__ int ok_s;
    if (variant != 2)
        for (int idx = threadIdx.x; idx < 128 * 16; idx += blockDim.x) {
            const int i = idx % 128, k = idx / 128;
            *reinterpret_cast<float *>(a_s + a_off(variant, i, k)) =
                (float)(((7 * i + 3 * k) % 11) - 5);
        }
    for (int idx = threadIdx.x; idx < 16 * N; idx += blockDim.x) {
        const int k = idx % 16, c = idx / 16;
        const float v = (float)(((5 * k + 2 * c) % 7) - 3);
        const int off = (c / 8) * 512 + (k / 4) * 128 + (c % 8) * 16 + (k % 4) * 4;
        *reinterpret_cast<float *>(b_s + off) = v;
    }
    if (threadIdx.x == 0) {
        tc::mbar_init(&bar, 1);
        tc::fence_mbar_init();
    }
    if (threadIdx.x < 32) {
        tc::tmem_alloc(&tbase, 512);
        tc::tmem_relinquish();
    }
    tc::fence_proxy_async();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t taddr = tbase;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t lane_base = (uint32_t)(32 * warp) << 16;
    {
        const float sentinel[8] = {-12345.f, -12345.f, -12345.f, -12345.f,
                                   -12345.f, -12345.f, -12345.f, -12345.f};
        for (int c0 = 0; c0 < N; c0 += 8) tc::tmem_st8(taddr + lane_base + (uint32_t)c0, sentinel);
        if (variant == 2) {  // this thread's row of A: columns 256 .. 271
            const int i = 32 * warp + lane;
            for (int k0 = 0; k0 < 16; k0 += 8) {
                float a[8];
#pragma unroll
                for (int q = 0; q < 8; ++q) a[q] = (float)(((7 * i + 3 * (k0 + q)) % 11) - 5);
                tc::tmem_st8(taddr + lane_base + 256u + (uint32_t)k0, a);
            }
        }
        tc::tmem_st_wait();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (threadIdx.x == 0) {
        const uint32_t id = tc::instr_desc(tc::kFmtTF32, 128, N, false, false);
        for (int s = 0; s < 2; ++s) {
            if (variant == 2) {
                const uint64_t bd = tc::smem_desc(tc::smem_u32(b_s + s * 256), 128, 512, tc::kSwNone);
                tc::mma_tf32_ts(taddr, taddr + 256u + 8u * s, bd, id, s > 0);
                continue;
            }
            const uint64_t ad =
                variant == 0 ? tc::smem_desc(tc::smem_u32(a_s + s * 256), 128, 512, tc::kSwNone)
                             : tc::smem_desc(tc::smem_u32(a_s + s * 32), 16, 1024, tc::kSw128);
            const uint64_t bd = tc::smem_desc(tc::smem_u32(b_s + s * 256), 128, 512, tc::kSwNone);
            tc::mma_tf32(taddr, ad, bd, id, s > 0);
        }
        tc::mma_commit(&bar);
        const bool ok = tc::mbar_wait(&bar, 0, wait_limit);
        ok_s = ok;
        if (!ok && status) atomicOr(status, kStatusTimeoutBit);
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (ok_s) {
        const int row = 32 * warp + lane;
        for (int c0 = 0; c0 < N; c0 += 8) {
            float v[8];
            tc::tmem_ld8(taddr + ((uint32_t)(32 * warp) << 16) + (uint32_t)c0, v);
            tc::tmem_ld_wait();
#pragma unroll
            for (int q = 0; q < 8; ++q) D[(size_t)row * N + c0 + q] = v[q];
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (threadIdx.x < 32) tc::tmem_dealloc(taddr, 512);
}

int sm_count() {
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    return v;
}

template <typename F>
float time_ms(F launch) {
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    launch();  // warm-up
    cudaEventRecord(a);
    launch();
    cudaEventRecord(b);
    cudaEventSynchronize(b);
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return ms;
}

}  // namespace
}  // namespace tsqr

using namespace tsqr;

// Measured peaks in TFLOP/s: out[0] FP64 DFMA, out[1] FP32 FFMA, out[2] TF32 warp-level mma
// (m16n8k8), out[3] TF32 tcgen05.mma, out[4] BF16 tcgen05.mma (dense; 2 flops per FMA).
// Returns TSQR_SUCCESS, TSQR_ERR_CUDA on a launch or runtime error, TSQR_ERR_TIMEOUT if a
// tensor-core wait gave up.  Synchronizes the device; takes about half a second.
extern "C" int tsqr_internal_measure_peaks(double *out, int count) {
    if (!out || count < 5) return TSQR_ERR_INVALID_ARG;
    const int sms = sm_count();
    if (sms <= 0) return TSQR_ERR_CUDA;
    void *sink = nullptr;
    int *status = nullptr;
    if (cudaMalloc(&sink, 4096) != cudaSuccess) return TSQR_ERR_ALLOC;
    if (cudaMalloc((void **)&status, sizeof(int)) != cudaSuccess) {
        cudaFree(sink);
        return TSQR_ERR_ALLOC;
    }
    cudaMemset(status, 0, sizeof(int));
    const dim3 g4(sms * 4), blk(256);
    const int it64 = 20000, it32 = 400000, itmma = 100000, ittc = 200000;
    float ms;
    ms = time_ms([&] { dfma_peak_kernel<<<g4, blk>>>((double *)sink, it64, 1.0000001, 1e-9); });
    out[0] = 2.0 * kChains * it64 * (double)g4.x * blk.x / (ms * 1e-3) / 1e12;
    ms = time_ms([&] { ffma_peak_kernel<<<g4, blk>>>((float *)sink, it32, 1.0000001f, 1e-9f); });
    out[1] = 2.0 * kChains * it32 * (double)g4.x * blk.x / (ms * 1e-3) / 1e12;
    ms = time_ms([&] { mma_tf32_peak_kernel<<<g4, blk>>>((float *)sink, itmma); });
    out[2] = 2.0 * 16 * 8 * 8 * kChains * (double)itmma * g4.x * (blk.x / 32) / (ms * 1e-3) / 1e12;
    const long long wait_limit = 1LL << 24;
    ms = time_ms([&] { tc05_peak_kernel<false><<<sms, 128>>>((float *)sink, ittc, status, wait_limit); });
    out[3] = 2.0 * 128 * kPeakN * 8 * (double)ittc * sms / (ms * 1e-3) / 1e12;
    ms = time_ms([&] { tc05_peak_kernel<true><<<sms, 128>>>((float *)sink, ittc, status, wait_limit); });
    out[4] = 2.0 * 128 * kPeakN * 16 * (double)ittc * sms / (ms * 1e-3) / 1e12;
    int st = 0;
    const cudaError_t e = cudaDeviceSynchronize();
    cudaMemcpy(&st, status, sizeof(int), cudaMemcpyDeviceToHost);
    cudaFree(sink);
    cudaFree(status);
    if (e != cudaSuccess) return TSQR_ERR_CUDA;
    return (st & kStatusTimeoutBit) ? TSQR_ERR_TIMEOUT : TSQR_SUCCESS;
}

// tcgen05 layout self-test (see tc05_layout_selftest_kernel): D is device memory of 128 x N
// floats, row-major; N a multiple of 16 in [16, 256]; variant 0..2.  Synchronizes the device.
extern "C" int tsqr_internal_tc_layout_selftest(float *D, int N, int variant) {
    if (!D || N < 16 || N > 256 || N % 16 || variant < 0 || variant > 2) return TSQR_ERR_INVALID_ARG;
    int *status = nullptr;
    if (cudaMalloc((void **)&status, sizeof(int)) != cudaSuccess) return TSQR_ERR_ALLOC;
    cudaMemset(status, 0, sizeof(int));
    const size_t smem = 1024 + (size_t)kSelftestARegion + (size_t)(N / 8) * 512;
    if (cudaFuncSetAttribute(tc05_layout_selftest_kernel,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
        cudaFree(status);
        return TSQR_ERR_CUDA;
    }
    tc05_layout_selftest_kernel<<<1, 128, smem>>>(D, N, variant, status, 1 << 22);
    const cudaError_t e = cudaDeviceSynchronize();
    int st = 0;
    cudaMemcpy(&st, status, sizeof(int), cudaMemcpyDeviceToHost);
    cudaFree(status);
    if (e != cudaSuccess) return TSQR_ERR_CUDA;
    return (st & kStatusTimeoutBit) ? TSQR_ERR_TIMEOUT : TSQR_SUCCESS;
}
