// gpv_lp.h -- launch arguments of the structure similarity loss (gpv_lp.cu).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace gpv {

struct LpArgs {
    const float* pts;     // [n, 3]
    int32_t n;
    const float* gpos;    // [m, 3]
    const float* gscale;  // [m, 3]
    int32_t m;
    float h;              // cell side of the hash grid
    // workspace
    uint32_t H;           // hash slots (power of two, >= 2 m)
    uint64_t* keys;       // [H]
    int32_t* head;        // [H]
    int32_t* next;        // [m]
    int32_t* pending;     // [n] points left to the exhaustive pass
    int32_t* counters;    // [2]: pending count, table-full flag
    uint32_t* smax;       // largest mean scale (order-preserving bits)
    double* partial;      // [nb_partial]
    int nb_partial;
    int sms;
    // outputs
    float* best;          // [n]
    int32_t* arg;         // [n]
    double* loss;         // [1]
};

cudaError_t lp_launch(const LpArgs& a, cudaStream_t s, int* nlaunch);

}  // namespace gpv
