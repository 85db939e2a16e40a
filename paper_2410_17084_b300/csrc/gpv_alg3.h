// gpv_alg3.h -- launch arguments of the paper's Alg. 3 formulation (gpv_alg3.cu).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "gpv_internal.h"

namespace gpv {

struct Alg3Args {
    // inputs (CSR batch)
    const float* xyz;
    const int64_t* offsets;
    const float* centres;
    const float* lam;
    const float* sf2;
    const float* sn2;
    float size;
    int G, tau, mean_mode;
    int nmax;            // voxels with more points are reported VOX_TOO_LARGE
    int nsm;             // largest n whose ky fits shared memory
    int nlo, nhi;        // this launch of kernel A takes the voxels with nlo < n <= nhi
    int nchunk;          // voxels of this chunk (the global-memory class loops over them)
    int kp;              // row stride of the workspace operands (nmax rounded up to 32)
    int32_t v0;          // first voxel of this chunk
    // outputs
    uint8_t* axis;
    float* mean;         // [nvox, G^2]
    float* cov;          // [nvox, G^2, G^2]
    uint32_t* status;
    // per-chunk workspace
    float* ws_pb;        // k_k* big part  [chunk, G^2, kp]
    float* ws_ps;        // k_k* small part
    float* ws_fa;        // K* factors     [chunk, kp, G]
    float* ws_fb;
    float* ws_A;         // ky of the voxels beyond shared memory: [CTAs of that class, kp, kp]
    uint32_t* ws_status; // [chunk]
    int32_t* ws_n;       // [chunk]
};

// largest n whose LU fits one CTA's shared memory at grid side G
int alg3_max_n(int G);
// CTAs of the class whose ky lives in global memory (each has a kp x kp slice of ws_A)
int alg3_big_ctas();
// kernel A (by size class) for nchunk voxels from a.v0, then the tensor-core covariance
// kernel; *nlaunch = kernels queued
cudaError_t alg3_launch_chunk(const Alg3Args& a, int nchunk, cudaStream_t s, int* nlaunch);

}  // namespace gpv
