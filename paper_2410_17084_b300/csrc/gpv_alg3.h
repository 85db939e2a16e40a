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
    int kp;              // point stride of the workspace operands (nmax rounded up to 32)
    int qp;              // query rows of the k_k* workspace (G^2 rounded up to 128)
    const int32_t* vidx; // processing order of the batch's voxels (those beyond shared memory
                         // first); slot s of this chunk is voxel vidx[s0 + s]
    int32_t s0;          // first position of this chunk in vidx
    // outputs
    uint8_t* axis;
    float* mean;         // [nvox, G^2]
    float* cov;          // [nvox, G^2, G^2]
    uint32_t* status;
    // per-chunk workspace
    float* ws_pk;        // k_k* as a TF32 split pair, [chunk, qp / 128, kp / 16, 2, 128 x 16]:
                         // big then small tile, each in the K-major core-matrix layout of the
                         // tensor-core operand (columns n .. kp of the last tile are zero)
    float* ws_tf;        // K* factors per 16-point chunk, [chunk, kp / 16, 2G, 20]: rows fa(., u)
                         // then fb(., x) over the nodes, 16 points + 4 floats of padding
    float* ws_fa;        // K* factors of the global-memory class, [chunk, kp, G]
    float* ws_fb;
    float* ws_A;         // ky of the voxels beyond shared memory: [CTAs of that class, kp, kp]
    uint32_t* ws_status; // [chunk]
    int32_t* ws_n;       // [chunk]
};

// largest n whose LU fits one CTA's shared memory at grid side G
int alg3_max_n(int G);
// CTAs of the class whose ky lives in global memory (each has a kp x kp slice of ws_A)
int alg3_big_ctas();
// the processing order: voxels whose ky does not fit shared memory (nsm < n <= nmax, n >= tau)
// first, then the others; counts: two zeroed int32 counters in device memory
cudaError_t alg3_order(const int64_t* offsets, int32_t nvox, int nsm, int nmax, int tau,
                       int32_t* vidx, int32_t* counts, cudaStream_t s);
// kernel A (by size class) for nchunk voxels from position a.s0 of the order, the class
// beyond shared memory on the side stream (forked from s and joined before the covariance
// kernel), then the tensor-core covariance kernel; *nlaunch = kernels queued
cudaError_t alg3_launch_chunk(const Alg3Args& a, int nchunk, cudaStream_t s, cudaStream_t side,
                              cudaEvent_t ev_fork, cudaEvent_t ev_join, int* nlaunch);

}  // namespace gpv
