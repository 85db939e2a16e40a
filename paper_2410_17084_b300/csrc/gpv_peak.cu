// gpv_peak.cu -- arithmetic peaks of this GPU measured with the solve's own arithmetic:
// FP32 fused multiply-adds, and the float-float accumulate-form multiply-add (acc_fma, the
// inner step of the variance contraction).  Each thread runs eight independent chains so
// the pipes, not the dependencies, bound the rate; the grid fills every SM.
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/gp_voxels.h"
#include "gpv_internal.h"
#include "gpv_num.cuh"

namespace gpv {
namespace {

constexpr int kChains = 8;

__global__ void __launch_bounds__(256) k_peak_fp32(int iters, float seed, float* sink)
{
    float a[kChains], b = 1.0000001f + 1e-9f * threadIdx.x, c = 1e-7f * seed;
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = seed + k;
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int k = 0; k < kChains; ++k) a[k] = __fmaf_rn(a[k], b, c);
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += a[k];
    if (s == 1234.5f) sink[threadIdx.x] = s;  // keeps the chains alive
}

__global__ void __launch_bounds__(256) k_peak_ff(int iters, float seed, float* sink)
{
    ff acc[kChains];
    const ff y = ff_make(seed * 1e-4f, 1e-15f);
#pragma unroll
    for (int k = 0; k < kChains; ++k) acc[k] = ff_make(seed + k, 0.f);
    // each chain multiplies the running value of the next one, so no product can be
    // hoisted out of the loop (a loop-invariant product would measure only the sums)
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int k = 0; k < kChains; ++k) acc_fma(acc[k], acc[(k + 1) % kChains], y);
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += acc_norm(acc[k]).hi;
    if (s == 1234.5f) sink[threadIdx.x] = s;
}

}  // namespace
}  // namespace gpv

extern "C" int gp_voxels_measure_peak(int kind, gpv_stream_t stream, double* h_tflops)
{
    using namespace gpv;
    if ((kind != 0 && kind != 1) || !h_tflops) return GPV_EINVAL;
    int dev = 0, sms = 0;
    cudaError_t e;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) { gpv_record_cuda_error(e); return GPV_ECUDA; }
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) {
        gpv_record_cuda_error(e);
        return GPV_ECUDA;
    }
    cudaStream_t s = (cudaStream_t)stream;
    float* sink = nullptr;
    if ((e = cudaMalloc(&sink, 256 * sizeof(float))) != cudaSuccess) { gpv_record_cuda_error(e); return GPV_ECUDA; }
    const int grid = sms * 8, iters = kind == 0 ? 1 << 16 : 1 << 13;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 3.0e38f;
    for (int rep = 0; rep < 3; ++rep) {  // the first launch also loads the kernel
        cudaEventRecord(e0, s);
        if (kind == 0) k_peak_fp32<<<grid, 256, 0, s>>>(iters, 1.f + rep, sink);
        else k_peak_ff<<<grid, 256, 0, s>>>(iters, 1.f + rep, sink);
        cudaEventRecord(e1, s);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) best = ms;
    }
    e = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(sink);
    if (e != cudaSuccess) { gpv_record_cuda_error(e); return GPV_ECUDA; }
    const double ops = 2.0 * kChains * (double)iters * 256.0 * (double)grid;  // 2 flops per (float-float) FMA
    *h_tflops = ops / (best * 1e-3) / 1e12;
    return GPV_OK;
}

namespace gpv {
namespace {

// One thread waits on an mbarrier that nothing arrives at, with the library's bounded
// poll loop: the wait must give up after `polls` tries and say so.
__global__ void k_bounded_wait(uint32_t polls, int32_t* timed_out)
{
    __shared__ __align__(8) uint64_t mbar;
    const uint32_t a = static_cast<uint32_t>(__cvta_generic_to_shared(&mbar));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(a), "r"(1u) : "memory");
    bool done = false;
    for (uint32_t it = 0; it < polls && !done; ++it) {
        uint32_t d;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(d) : "r"(a), "r"(0u) : "memory");
        done = d != 0;
    }
    *timed_out = done ? 0 : 1;
}

}  // namespace
}  // namespace gpv

extern "C" int gp_voxels_selftest_bounded_wait(uint32_t polls, gpv_stream_t stream,
                                               int32_t* h_timed_out)
{
    using namespace gpv;
    if (!h_timed_out || polls == 0 || polls > (1u << 24)) return GPV_EINVAL;
    int32_t* d = nullptr;
    cudaError_t e = cudaMalloc(&d, sizeof(int32_t));
    if (e != cudaSuccess) { gpv_record_cuda_error(e); return GPV_ECUDA; }
    cudaStream_t s = (cudaStream_t)stream;
    k_bounded_wait<<<1, 1, 0, s>>>(polls, d);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(h_timed_out, d, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(d);
    if (e != cudaSuccess) { gpv_record_cuda_error(e); return GPV_ECUDA; }
    return GPV_OK;
}
