// gpv_raster.cu -- alpha-blending rasterisation of 3D Gaussians (GS-LIVM Sec. 3.3, Eq. 9)
// into headless device images: colour C, depth D and silhouette S of one pinhole camera.
//
//   k_rs_pre     one thread per Gaussian (FP32): camera transform, near cull, EWA
//                projection Sigma' = J Rc Sigma Rc^T J^T + 0.3 I, conic, 3-sigma radius, the
//                rectangle of 16 x 16 tiles whose pixels it may reach; per-tile counts
//   k_rs_tscan   exclusive scan of the per-tile counts (one CTA)
//   k_rs_scatter one thread per Gaussian: key (depth bits << 32 | index) into each of its
//                tiles' lists
//   k_rs_sort    one CTA per tile: bitonic sort of the tile's keys in shared memory (a
//                global-memory bitonic pass for tiles with more than kSortSmem keys), so
//                Gaussians are blended front to back, ties by index
//   k_rs_render  one CTA per tile, one thread per pixel: batches of 256 splats staged in
//                shared memory; per pixel alpha = min(0.99, op exp(-d^T conic d / 2)) inside
//                the 3-sigma square, skipped below 1/255, blending stops before T < 1e-4;
//                the CTA leaves once every pixel is done
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "gpv_raster.h"

namespace gpv {

namespace {

constexpr int kTile = 16;
constexpr int kSortSmem = 8192;  // keys sorted in shared memory (64 KB)

__global__ void k_rs_pre(RasterArgs a)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= a.m) return;
    float4* s0 = a.sp + 3 * (int64_t)k;
    s0[0] = make_float4(0.f, 0.f, 0.f, 0.f);
    s0[1] = make_float4(0.f, 0.f, 0.f, -1.f);  // radius < 0: culled
    const RasterCamera& c = a.cam;
    const float px = a.pos[3 * k], py = a.pos[3 * k + 1], pz = a.pos[3 * k + 2];
    float t[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) t[r] = c.R[3 * r] * px + c.R[3 * r + 1] * py + c.R[3 * r + 2] * pz + c.t[r];
    // the depth that orders and culls: each operation rounded, in a fixed order, so it is
    // reproducible on any IEEE FP32 implementation
    const float zk = __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(c.R[6], px), __fmul_rn(c.R[7], py)),
                                         __fmul_rn(c.R[8], pz)), c.t[2]);
    if (!(zk > c.near)) return;
    float qw = a.quat[4 * k], qx = a.quat[4 * k + 1], qy = a.quat[4 * k + 2], qz = a.quat[4 * k + 3];
    const float qn = rsqrtf(qw * qw + qx * qx + qy * qy + qz * qz);
    qw *= qn; qx *= qn; qy *= qn; qz *= qn;
    const float R[3][3] = {
        {1.f - 2.f * (qy * qy + qz * qz), 2.f * (qx * qy - qw * qz), 2.f * (qx * qz + qw * qy)},
        {2.f * (qx * qy + qw * qz), 1.f - 2.f * (qx * qx + qz * qz), 2.f * (qy * qz - qw * qx)},
        {2.f * (qx * qz - qw * qy), 2.f * (qy * qz + qw * qx), 1.f - 2.f * (qx * qx + qy * qy)}};
    const float s2[3] = {a.scale[3 * k] * a.scale[3 * k], a.scale[3 * k + 1] * a.scale[3 * k + 1],
                         a.scale[3 * k + 2] * a.scale[3 * k + 2]};
    const float limx = 1.3f * (float)c.width / (2.f * c.fx), limy = 1.3f * (float)c.height / (2.f * c.fy);
    const float xz = fminf(fmaxf(t[0] / t[2], -limx), limx);
    const float yz = fminf(fmaxf(t[1] / t[2], -limy), limy);
    const float J[2][3] = {{c.fx / t[2], 0.f, -c.fx * xz / t[2]}, {0.f, c.fy / t[2], -c.fy * yz / t[2]}};
    // M = J Rc R (2 x 3); Sigma' = M diag(s^2) M^T
    float M[2][3];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            float acc = 0.f;
#pragma unroll
            for (int l = 0; l < 3; ++l) {
                const float jr = J[i][0] * c.R[l] + J[i][1] * c.R[3 + l] + J[i][2] * c.R[6 + l];
                acc += jr * R[l][j];
            }
            M[i][j] = acc;
        }
    const float sa = M[0][0] * M[0][0] * s2[0] + M[0][1] * M[0][1] * s2[1] + M[0][2] * M[0][2] * s2[2] + 0.3f;
    const float sb = M[0][0] * M[1][0] * s2[0] + M[0][1] * M[1][1] * s2[1] + M[0][2] * M[1][2] * s2[2];
    const float sc = M[1][0] * M[1][0] * s2[0] + M[1][1] * M[1][1] * s2[1] + M[1][2] * M[1][2] * s2[2] + 0.3f;
    const float det = sa * sc - sb * sb;
    if (!(det > 0.f)) return;
    const float mid = 0.5f * (sa + sc);
    const float lmax = mid + sqrtf(fmaxf(mid * mid - det, 0.1f));
    const float r = ceilf(3.f * sqrtf(lmax));
    const float u = c.fx * t[0] / t[2] + c.cx, v = c.fy * t[1] / t[2] + c.cy;
    // pixels x with |x + 1/2 - u| <= r, and their tiles
    const int x0 = max(0, (int)ceilf(u - r - 0.5f)), x1 = min(c.width - 1, (int)floorf(u + r - 0.5f));
    const int y0 = max(0, (int)ceilf(v - r - 0.5f)), y1 = min(c.height - 1, (int)floorf(v + r - 0.5f));
    if (x0 > x1 || y0 > y1) return;
    s0[0] = make_float4(u, v, zk, a.opacity[k]);
    s0[1] = make_float4(sc / det, -sb / det, sa / det, r);
    s0[2] = make_float4(a.color[3 * k], a.color[3 * k + 1], a.color[3 * k + 2], 0.f);
    const int tx0 = x0 / kTile, tx1 = x1 / kTile, ty0 = y0 / kTile, ty1 = y1 / kTile;
    a.rect[k] = make_int4(tx0, ty0, tx1, ty1);
    for (int ty = ty0; ty <= ty1; ++ty)
        for (int tx = tx0; tx <= tx1; ++tx) atomicAdd(&a.tile_count[ty * a.tiles_x + tx], 1);
}

// exclusive scan of ntile counts by one CTA of 1024 threads; tile_off[ntile] = total
__global__ void __launch_bounds__(1024) k_rs_tscan(const int32_t* count, int ntile, int32_t* off,
                                                   int32_t* cursor)
{
    __shared__ int32_t wsum[32];
    __shared__ int32_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int base = 0; base < ntile; base += 1024) {
        const int i = base + threadIdx.x;
        const int v = i < ntile ? count[i] : 0;
        int x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) wsum[wid] = x;
        __syncthreads();
        if (wid == 0) {
            const int w = wsum[lane];
            int wx = w;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, wx, o);
                if (lane >= o) wx += y;
            }
            wsum[lane] = wx - w;
        }
        __syncthreads();
        const int excl = carry + wsum[wid] + x - v;
        if (i < ntile) { off[i] = excl; cursor[i] = 0; }
        __syncthreads();
        if (threadIdx.x == 1023) carry = excl + v;
        __syncthreads();
    }
    if (threadIdx.x == 0) off[ntile] = carry;
}

__global__ void k_rs_scatter(RasterArgs a)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= a.m) return;
    if (a.sp[3 * (int64_t)k + 1].w < 0.f) return;
    const int4 rc = a.rect[k];
    const uint64_t key = ((uint64_t)__float_as_uint(a.sp[3 * (int64_t)k].z) << 32) | (uint32_t)k;
    for (int ty = rc.y; ty <= rc.w; ++ty)
        for (int tx = rc.x; tx <= rc.z; ++tx) {
            const int t = ty * a.tiles_x + tx;
            const int p = a.tile_off[t] + atomicAdd(&a.tile_cursor[t], 1);
            if (p < a.cap) a.keys[p] = key;
        }
}

// ascending compare-exchange: the smaller key to the lower position
__device__ __forceinline__ void cswap(uint64_t& x, uint64_t& y)
{
    if (x > y) { const uint64_t t = x; x = y; y = t; }
}

// Bitonic sort in which every compare-exchange is ascending (each merge starts by comparing
// mirrored positions), so the padding to a power of two -- keys of +infinity -- only moves
// up and never displaces a real key: the global-memory variant need not store it.
__global__ void __launch_bounds__(1024) k_rs_sort(RasterArgs a)
{
    extern __shared__ uint64_t sk[];
    const int t = blockIdx.x;
    const int beg = a.tile_off[t], cnt = a.tile_off[t + 1] - beg;
    if (cnt <= 1 || beg + cnt > a.cap) return;
    int np = 1;
    while (np < cnt) np <<= 1;
    const bool in_smem = np <= kSortSmem;
    uint64_t* k = in_smem ? sk : a.keys + beg;
    if (in_smem) {
        for (int i = threadIdx.x; i < np; i += blockDim.x) k[i] = i < cnt ? a.keys[beg + i] : ~0ull;
        __syncthreads();
    }
    auto step = [&](int lo, int hi) {
        if (in_smem) {
            cswap(k[lo], k[hi]);
        } else if (lo < cnt) {  // positions at or past cnt hold +infinity implicitly
            if (hi < cnt) {
                uint64_t x = k[lo], y = k[hi];
                cswap(x, y);
                k[lo] = x;
                k[hi] = y;
            }
        }
    };
    for (int size = 2; size <= np; size <<= 1) {
        const int half = size >> 1;
        for (int i = threadIdx.x; i < np / 2; i += blockDim.x) {
            const int blk = i / half, off = i - blk * half;
            step(blk * size + off, blk * size + size - 1 - off);
        }
        __syncthreads();
        for (int stride = half >> 1; stride > 0; stride >>= 1) {
            for (int i = threadIdx.x; i < np / 2; i += blockDim.x) {
                const int lo = 2 * i - (i & (stride - 1));
                step(lo, lo + stride);
            }
            __syncthreads();
        }
    }
    if (in_smem)
        for (int i = threadIdx.x; i < cnt; i += blockDim.x) a.keys[beg + i] = k[i];
}

__global__ void __launch_bounds__(kTile * kTile) k_rs_render(RasterArgs a)
{
    __shared__ float4 s0[kTile * kTile], s1[kTile * kTile], s2[kTile * kTile];
    const int t = blockIdx.x;
    const int tx = t % a.tiles_x, ty = t / a.tiles_x;
    const int x = tx * kTile + (threadIdx.x % kTile), y = ty * kTile + (threadIdx.x / kTile);
    const bool inside = x < a.cam.width && y < a.cam.height;
    const float pxc = x + 0.5f, pyc = y + 0.5f;
    const int beg = a.tile_off[t], cnt = min(a.tile_off[t + 1], a.cap) - beg;
    float T = 1.f, C0 = 0.f, C1 = 0.f, C2 = 0.f, Dp = 0.f, Sp = 0.f;
    bool done = !inside;
    for (int b0 = 0; b0 < cnt; b0 += kTile * kTile) {
        if (__syncthreads_and(done)) break;
        const int i = b0 + threadIdx.x;
        if (i < cnt) {
            const uint32_t k = (uint32_t)(a.keys[beg + i] & 0xFFFFFFFFull);
            s0[threadIdx.x] = a.sp[3 * (int64_t)k];
            s1[threadIdx.x] = a.sp[3 * (int64_t)k + 1];
            s2[threadIdx.x] = a.sp[3 * (int64_t)k + 2];
        }
        __syncthreads();
        const int nb = min(kTile * kTile, cnt - b0);
        for (int j = 0; j < nb && !done; ++j) {
            const float4 g0 = s0[j], g1 = s1[j];
            const float dx = pxc - g0.x, dy = pyc - g0.y;
            if (fabsf(dx) > g1.w || fabsf(dy) > g1.w) continue;
            const float power = -0.5f * (g1.x * dx * dx + g1.z * dy * dy) - g1.y * dx * dy;
            const float alpha = fminf(0.99f, g0.w * expf(power));
            if (alpha < 1.f / 255.f) continue;
            const float nt = T * (1.f - alpha);
            if (nt < 1e-4f) { done = true; break; }
            const float w = alpha * T;
            const float4 g2 = s2[j];
            C0 += g2.x * w; C1 += g2.y * w; C2 += g2.z * w;
            Dp += g0.z * w;
            Sp += w;
            T = nt;
        }
    }
    if (inside) {
        const int64_t o = (int64_t)y * a.cam.width + x;
        a.C[3 * o] = C0; a.C[3 * o + 1] = C1; a.C[3 * o + 2] = C2;
        a.D[o] = Dp;
        a.S[o] = Sp;
    }
}

}  // namespace

cudaError_t raster_prepare(const RasterArgs& a, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(a.tile_count, 0, sizeof(int32_t) * a.ntile, s);
    if (e != cudaSuccess) return e;
    if (a.m > 0) k_rs_pre<<<(a.m + 255) / 256, 256, 0, s>>>(a);
    k_rs_tscan<<<1, 1024, 0, s>>>(a.tile_count, a.ntile, a.tile_off, a.tile_cursor);
    return cudaGetLastError();
}

cudaError_t raster_finish(const RasterArgs& a, cudaStream_t s)
{
    if (a.m > 0) k_rs_scatter<<<(a.m + 255) / 256, 256, 0, s>>>(a);
    cudaError_t e = cudaFuncSetAttribute(k_rs_sort, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         kSortSmem * 8);
    if (e != cudaSuccess) return e;
    k_rs_sort<<<a.ntile, 1024, kSortSmem * 8, s>>>(a);
    k_rs_render<<<a.ntile, kTile * kTile, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace gpv
