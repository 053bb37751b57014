// FP32 FMA throughput of the device: the measured denominator of the roofline
// of the greedy loop, which is bound by plain FP32 arithmetic (packed
// FFMA2/FADD2/FMUL2 and scalar compares), not by memory.
//
// Every thread runs eight independent FMA chains x <- x * m + c (m just below
// 1, so the chains settle near c / (1 - m) and never reach denormals or
// infinities), packed two lanes per FFMA2, or scalar FFMA for the second
// variant; four 256-thread CTAs per SM keep eight warps on every scheduler.
// The result is stored only if it equals a value the chains cannot reach, so
// the compiler keeps the arithmetic and the store never happens.
#include <cuda_runtime.h>

#include <cstdint>

#include "rljsde_internal.h"

namespace rljsde {
namespace {

constexpr int kPeakThreads = 256;
constexpr int kPeakCtasPerSm = 4;
constexpr int kPeakChains = 8;
constexpr int kPeakUnroll = 4;

__device__ float g_peak_sink;

template <bool PACKED>
__global__ void __launch_bounds__(kPeakThreads, kPeakCtasPerSm) fma_peak_kernel(int iters, float m, float c,
                                                                                float never)
{
    float2 x[kPeakChains];
#pragma unroll
    for (int i = 0; i < kPeakChains; ++i) x[i] = make_float2(1e-3f * threadIdx.x + i, 0.5f * i);
    const float2 m2 = make_float2(m, m), c2 = make_float2(c, c);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < kPeakUnroll; ++u) {
#pragma unroll
            for (int i = 0; i < kPeakChains; ++i) {
                if constexpr (PACKED) {
                    x[i] = __ffma2_rn(x[i], m2, c2);
                } else {
                    x[i].x = __fmaf_rn(x[i].x, m, c);
                    x[i].y = __fmaf_rn(x[i].y, m, c);
                }
            }
        }
    }
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < kPeakChains; ++i) s += x[i].x + x[i].y;
    if (s == never) g_peak_sink = s;
}

}  // namespace
}  // namespace rljsde

extern "C" int rljsde_fp32_peak(int reps, void *stream, double *tflops_out, float *ms_out)
{
    using namespace rljsde;
    if (reps < 1 || reps > 1000 || !tflops_out) return RLJSDE_ERR_INVALID_ARG;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
        return RLJSDE_ERR_CUDA;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int grid = sms * kPeakCtasPerSm, iters = 1 << 16;
    // flops of one launch: every thread, every iteration, kPeakUnroll x kPeakChains FMAs on two lanes
    const double flops = 2.0 * 2.0 * kPeakChains * kPeakUnroll * (double)iters * grid * kPeakThreads;
    cudaEvent_t a = nullptr, b = nullptr;
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) {
        if (a) cudaEventDestroy(a);
        return RLJSDE_ERR_CUDA;
    }
    float best = 1e30f;
    int st = RLJSDE_OK;
    for (int variant = 0; variant < 2 && st == RLJSDE_OK; ++variant) {
        for (int r = 0; r <= reps; ++r) {            // launch 0 warms up
            cudaEventRecord(a, s);
            if (variant == 0)
                fma_peak_kernel<true><<<grid, kPeakThreads, 0, s>>>(iters, 0.9999f, 1e-4f, -1.f);
            else
                fma_peak_kernel<false><<<grid, kPeakThreads, 0, s>>>(iters, 0.9999f, 1e-4f, -1.f);
            cudaEventRecord(b, s);
            float ms = 0.f;
            if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(b) != cudaSuccess ||
                cudaEventElapsedTime(&ms, a, b) != cudaSuccess) {
                st = RLJSDE_ERR_CUDA;
                break;
            }
            if (r > 0 && ms < best) best = ms;
        }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (st != RLJSDE_OK) return st;
    *tflops_out = flops / (best * 1e-3) / 1e12;
    if (ms_out) *ms_out = best;
    return RLJSDE_OK;
}
