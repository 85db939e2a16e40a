// gpv_raster.h -- launch arguments of the Gaussian rasteriser (gpv_raster.cu).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace gpv {

struct RasterCamera {
    float R[9];    // world -> camera rotation, row-major
    float t[3];    // world -> camera translation
    float fx, fy, cx, cy;
    int width, height;
    float near;
};

struct RasterArgs {
    const float* pos;      // [m, 3]
    const float* scale;    // [m, 3]
    const float* quat;     // [m, 4] (w, x, y, z)
    const float* opacity;  // [m]
    const float* color;    // [m, 3]
    int32_t m;
    RasterCamera cam;
    int tiles_x, tiles_y, ntile;
    // workspace
    float4* sp;            // [m, 3] projected splats
    int4* rect;            // [m] tile rectangle
    int32_t* tile_count;   // [ntile]
    int32_t* tile_off;     // [ntile + 1]
    int32_t* tile_cursor;  // [ntile]
    uint64_t* keys;        // [cap] (depth bits << 32 | index), per tile
    int32_t cap;
    // outputs
    float* C;              // [H, W, 3]
    float* D;              // [H, W]
    float* S;              // [H, W]
};

// projection and per-tile counts (total pairs at tile_off[ntile] afterwards)
cudaError_t raster_prepare(const RasterArgs& a, cudaStream_t s);
// lists, per-tile sort, blending
cudaError_t raster_finish(const RasterArgs& a, cudaStream_t s);

}  // namespace gpv
