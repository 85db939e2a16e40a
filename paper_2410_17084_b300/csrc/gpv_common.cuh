// gpv_common.cuh -- device helpers shared by the solve kernels (gpv_solve.cu) and the
// full-covariance path (gpv_alg3.cu): warp/CTA reductions and the value-axis choice.
#pragma once
#include <cuda_runtime.h>

#include "gpv_init.cuh"
#include "gpv_num.cuh"

namespace gpv {

__device__ __forceinline__ float shfl_x(float x, int o) { return __shfl_xor_sync(0xffffffffu, x, o); }
__device__ __forceinline__ double shfl_x(double x, int o) { return __shfl_xor_sync(0xffffffffu, x, o); }
__device__ __forceinline__ ff shfl_x(ff x, int o)
{
    return ff_make(__shfl_xor_sync(0xffffffffu, x.hi, o), __shfl_xor_sync(0xffffffffu, x.lo, o));
}

// Sum of K values of type R over the CTA (fixed order: deterministic); every thread
// gets the totals.  red must hold K * 32 values of R.
template <class R, int K>
__device__ __forceinline__ void block_sum(R (&v)[K], R* red)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int k = 0; k < K; ++k)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[k] = v[k] + shfl_x(v[k], o);
    __syncthreads();
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < K; ++k) red[k * 32 + wid] = v[k];
    __syncthreads();
#pragma unroll
    for (int k = 0; k < K; ++k) {
        R s = red[k * 32];
        for (int w = 1; w < nw; ++w) s = s + red[k * 32 + w];
        v[k] = s;
    }
    __syncthreads();
}

// Value axis of a point set: normal = eigenvector of the smallest eigenvalue of the
// covariance; axis = argmax |normal_k| with exact ties resolved Z, then X, then Y.
// The decision needs no more than FP32: voxels whose two largest normal components
// lie within 1e-3 are axis-ambiguous by definition.
__device__ inline int value_axis_from_cov(const float c6[6])
{
    float ev[3], E[9];
    sym3_eig<float>(c6, ev, E);
    int k = 0;
    if (ev[1] < ev[k]) k = 1;
    if (ev[2] < ev[k]) k = 2;
    const float nx = fabsf(E[0 + k]), ny = fabsf(E[3 + k]), nz = fabsf(E[6 + k]);
    int ax = 2;
    float best = nz;
    if (nx > best) { ax = 0; best = nx; }
    if (ny > best) { ax = 1; }
    return ax;
}

}  // namespace gpv
