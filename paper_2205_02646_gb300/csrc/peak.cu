// FP32 FMA throughput of the device: the measured denominator of the roofline
// of the greedy loop, which is bound by plain FP32 arithmetic (packed
// FFMA2/FADD2/FMUL2 and scalar compares), not by HBM; and the L2 read
// bandwidth the stored-C loop's Gram-column reads are measured against.
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

// L2 read bandwidth: a 32 MiB buffer, resident in the L2 after the warm-up
// launch, read by every SM with 16-byte non-coherent loads (the path the
// stored-C loop reads its Gram columns by), eight loads per thread in flight.
constexpr size_t kL2Bytes = (size_t)32 << 20;
constexpr int kL2Passes = 128;

__global__ void __launch_bounds__(kPeakThreads) l2_read_kernel(const float4 *__restrict__ buf, int n4, float never)
{
    const int stride = gridDim.x * blockDim.x;
    const int t0 = blockIdx.x * blockDim.x + threadIdx.x;
    float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    for (int p = 0; p < kL2Passes; ++p) {
        int i = t0;
        for (; i + 7 * stride < n4; i += 8 * stride) {
            float4 v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) v[u] = __ldg(buf + i + u * stride);
#pragma unroll
            for (int u = 0; u < 8; ++u) acc[u] += (v[u].x + v[u].y) + (v[u].z + v[u].w);
        }
        for (; i < n4; i += stride) {
            const float4 v = __ldg(buf + i);
            acc[0] += (v.x + v.y) + (v.z + v.w);
        }
    }
    float s = 0.f;
#pragma unroll
    for (int u = 0; u < 8; ++u) s += acc[u];
    if (s == never) g_peak_sink = s;
}

}  // namespace
}  // namespace rljsde

extern "C" int rljsde_l2_read_peak(int reps, void *stream, double *gbs_out, float *ms_out)
{
    using namespace rljsde;
    if (reps < 1 || reps > 1000 || !gbs_out) return RLJSDE_ERR_INVALID_ARG;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
        return RLJSDE_ERR_CUDA;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    float4 *buf = nullptr;
    if (cudaMalloc((void **)&buf, kL2Bytes) != cudaSuccess) {
        cudaGetLastError();
        return RLJSDE_ERR_OUT_OF_MEMORY;
    }
    const int n4 = (int)(kL2Bytes / sizeof(float4)), grid = sms * kPeakCtasPerSm;
    const double bytes = (double)kL2Bytes * kL2Passes;
    cudaEvent_t a = nullptr, b = nullptr;
    int st = cudaMemsetAsync(buf, 0, kL2Bytes, s) == cudaSuccess ? RLJSDE_OK : RLJSDE_ERR_CUDA;
    if (st == RLJSDE_OK && (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess))
        st = RLJSDE_ERR_CUDA;
    float best = 1e30f;
    for (int r = 0; r <= reps && st == RLJSDE_OK; ++r) {     // launch 0 warms up (and fills the L2)
        cudaEventRecord(a, s);
        l2_read_kernel<<<grid, kPeakThreads, 0, s>>>(buf, n4, -1.f);
        cudaEventRecord(b, s);
        float ms = 0.f;
        if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(b) != cudaSuccess ||
            cudaEventElapsedTime(&ms, a, b) != cudaSuccess) {
            st = RLJSDE_ERR_CUDA;
            break;
        }
        if (r > 0 && ms < best) best = ms;
    }
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    cudaStreamSynchronize(s);
    cudaFree(buf);
    if (st != RLJSDE_OK) return st;
    *gbs_out = bytes / (best * 1e-3) / 1e9;
    if (ms_out) *ms_out = best;
    return RLJSDE_OK;
}

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
