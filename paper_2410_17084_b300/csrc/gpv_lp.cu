// gpv_lp.cu -- structure similarity loss (GS-LIVM Sec. 3.3, Eq. 11): for every point of a
// scan, min over the Gaussians k of |P_j - p_k| - mean(S_k), and the mean over the points.
//
//   k_lp_build   one thread per Gaussian: its cell floor(p / h) goes into an
//                open-addressing hash (CAS, bounded linear probing); the Gaussian is pushed
//                on the cell's list (head per slot, next per Gaussian); the largest mean
//                scale smax is kept with an order-preserving integer atomicMax.
//   k_lp_query   one thread per point: cells in Chebyshev rings r = 0, 1, ... around the
//                point's cell.  Any Gaussian in ring r + 1 or beyond is at least r h away,
//                so its value is at least r h - smax: the search stops once the best value
//                is below that bound (exact).  Points not settled within kMaxRing rings are
//                listed for the exhaustive pass.
//   k_lp_exhaust one CTA per listed point: all m Gaussians, CTA-wide minimum.
//   k_lp_mean    the mean in FP64, fixed-order per-block partial sums then one block.
// Ties between Gaussians resolve to the smallest index, so results do not depend on the
// order in which Gaussians entered the lists.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "gpv_lp.h"

namespace gpv {

namespace {

constexpr uint64_t kEmptyKey = ~0ull;
constexpr int kOff = 1 << 20;
constexpr int kMaxRing = 16;

__device__ __forceinline__ uint64_t cell_key(int x, int y, int z)
{
    const uint64_t m = 0x1FFFFFull;
    return ((uint64_t)(uint32_t)(x + kOff) & m) | (((uint64_t)(uint32_t)(y + kOff) & m) << 21) |
           (((uint64_t)(uint32_t)(z + kOff) & m) << 42);
}

__device__ __forceinline__ uint32_t cell_hash(uint64_t key, uint32_t mask)
{
    uint64_t h = key * 0x9E3779B97F4A7C15ull;
    h ^= h >> 29;
    return (uint32_t)h & mask;
}

// float <-> unsigned with the same order (for atomicMax of possibly negative values)
__device__ __forceinline__ uint32_t ord_of(float f)
{
    const uint32_t u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float float_of(uint32_t o)
{
    return __uint_as_float((o & 0x80000000u) ? (o & 0x7FFFFFFFu) : ~o);
}

__global__ void k_lp_reset(uint64_t* keys, int32_t* head, uint32_t H, uint32_t* smax, int32_t* counters)
{
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < H) { keys[i] = kEmptyKey; head[i] = -1; }
    if (i == 0) { *smax = ord_of(-3.0e38f); counters[0] = 0; counters[1] = 0; }
}

__global__ void k_lp_build(const float* gpos, const float* gscale, int32_t m, float inv_h,
                           uint64_t* keys, int32_t* head, int32_t* next, uint32_t mask,
                           uint32_t* smax, int32_t* counters)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= m) return;
    const float sb = (gscale[3 * k] + gscale[3 * k + 1] + gscale[3 * k + 2]) / 3.f;
    atomicMax(smax, ord_of(sb));
    const int cx = (int)floorf(gpos[3 * k] * inv_h), cy = (int)floorf(gpos[3 * k + 1] * inv_h),
              cz = (int)floorf(gpos[3 * k + 2] * inv_h);
    const uint64_t key = cell_key(cx, cy, cz);
    const uint32_t h0 = cell_hash(key, mask);
    int s = -1;
    for (uint32_t p = 0; p <= mask; ++p) {
        const uint32_t t = (h0 + p) & mask;
        const uint64_t cur = keys[t];
        if (cur == key) { s = (int)t; break; }
        if (cur == kEmptyKey) {
            const uint64_t old = atomicCAS((unsigned long long*)&keys[t], (unsigned long long)kEmptyKey,
                                           (unsigned long long)key);
            if (old == kEmptyKey || old == key) { s = (int)t; break; }
        }
    }
    if (s < 0) { atomicOr(counters + 1, 1); next[k] = -1; return; }  // table full
    next[k] = atomicExch(&head[s], k);
}

__device__ __forceinline__ int lookup(const uint64_t* keys, uint32_t mask, uint64_t key)
{
    const uint32_t h0 = cell_hash(key, mask);
    for (uint32_t p = 0; p <= mask; ++p) {
        const uint32_t t = (h0 + p) & mask;
        const uint64_t cur = keys[t];
        if (cur == key) return (int)t;
        if (cur == kEmptyKey) return -1;
    }
    return -1;
}

__device__ __forceinline__ void visit(const float* gpos, const float* gscale, const int32_t* next,
                                      int k, float px, float py, float pz, float& best, int& bk)
{
    for (int guard = 0; k >= 0 && guard < (1 << 30); ++guard) {
        const float dx = px - gpos[3 * k], dy = py - gpos[3 * k + 1], dz = pz - gpos[3 * k + 2];
        const float sb = (gscale[3 * k] + gscale[3 * k + 1] + gscale[3 * k + 2]) / 3.f;
        const float v = sqrtf(dx * dx + dy * dy + dz * dz) - sb;
        if (v < best || (v == best && k < bk)) { best = v; bk = k; }
        k = next[k];
    }
}

__global__ void k_lp_query(const float* pts, int32_t n, const float* gpos, const float* gscale,
                           const uint64_t* keys, const int32_t* head, const int32_t* next,
                           uint32_t mask, float h, const uint32_t* smax, float* best_out,
                           int32_t* arg_out, int32_t* pending, int32_t* counters)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const float px = pts[3 * j], py = pts[3 * j + 1], pz = pts[3 * j + 2];
    const float inv_h = 1.f / h;
    const int cx = (int)floorf(px * inv_h), cy = (int)floorf(py * inv_h), cz = (int)floorf(pz * inv_h);
    const float sm = float_of(*smax);
    float best = 3.0e38f;
    int bk = -1;
    bool done = false;
    for (int r = 0; r <= kMaxRing && !done; ++r) {
        for (int dz = -r; dz <= r; ++dz)
            for (int dy = -r; dy <= r; ++dy) {
                const bool face = (dz == -r || dz == r || dy == -r || dy == r);
                const int step = face ? 1 : 2 * r;  // inner rows: only the two ends
                for (int dx = -r; dx <= r; dx += (step > 0 ? step : 1)) {
                    const int s = lookup(keys, mask, cell_key(cx + dx, cy + dy, cz + dz));
                    if (s >= 0) visit(gpos, gscale, next, head[s], px, py, pz, best, bk);
                }
            }
        // every Gaussian beyond ring r is at least r h away
        if (bk >= 0 && best < (float)r * h - sm) done = true;
    }
    best_out[j] = best;
    arg_out[j] = bk;
    if (!done) pending[atomicAdd(counters, 1)] = j;
}

__global__ void k_lp_exhaust(const float* pts, const float* gpos, const float* gscale, int32_t m,
                             const int32_t* pending, const int32_t* counters, float* best_out,
                             int32_t* arg_out)
{
    __shared__ float sv[32];
    __shared__ int sk[32];
    const int np = counters[0];
    for (int i = blockIdx.x; i < np; i += gridDim.x) {
        const int j = pending[i];
        const float px = pts[3 * j], py = pts[3 * j + 1], pz = pts[3 * j + 2];
        float best = 3.0e38f;
        int bk = -1;
        for (int k = threadIdx.x; k < m; k += blockDim.x) {
            const float dx = px - gpos[3 * k], dy = py - gpos[3 * k + 1], dz = pz - gpos[3 * k + 2];
            const float sb = (gscale[3 * k] + gscale[3 * k + 1] + gscale[3 * k + 2]) / 3.f;
            const float v = sqrtf(dx * dx + dy * dy + dz * dz) - sb;
            if (v < best || (v == best && k < bk)) { best = v; bk = k; }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float ov = __shfl_xor_sync(0xffffffffu, best, o);
            const int ok = __shfl_xor_sync(0xffffffffu, bk, o);
            if (ok >= 0 && (bk < 0 || ov < best || (ov == best && ok < bk))) { best = ov; bk = ok; }
        }
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
        if (lane == 0) { sv[wid] = best; sk[wid] = bk; }
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int w = 1; w < nw; ++w)
                if (sk[w] >= 0 && (bk < 0 || sv[w] < best || (sv[w] == best && sk[w] < bk))) {
                    best = sv[w];
                    bk = sk[w];
                }
            best_out[j] = best;
            arg_out[j] = bk;
        }
        __syncthreads();
    }
}

constexpr int kMeanBlock = 256;

__global__ void k_lp_partial(const float* best, int32_t n, double* partial)
{
    __shared__ double s[kMeanBlock];
    double acc = 0.0;
    for (int j = blockIdx.x * kMeanBlock + threadIdx.x; j < n; j += gridDim.x * kMeanBlock)
        acc += (double)best[j];
    s[threadIdx.x] = acc;
    __syncthreads();
    for (int o = kMeanBlock / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = s[0];
}

__global__ void k_lp_final(const double* partial, int nb, int32_t n, double* loss)
{
    __shared__ double s[kMeanBlock];
    double acc = 0.0;
    for (int i = threadIdx.x; i < nb; i += kMeanBlock) acc += partial[i];
    s[threadIdx.x] = acc;
    __syncthreads();
    for (int o = kMeanBlock / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) *loss = n > 0 ? s[0] / (double)n : 0.0;
}

}  // namespace

cudaError_t lp_launch(const LpArgs& a, cudaStream_t s, int* nlaunch)
{
    const uint32_t H = a.H, mask = H - 1;
    const int blk = 256;
    k_lp_reset<<<(H + blk - 1) / blk, blk, 0, s>>>(a.keys, a.head, H, a.smax, a.counters);
    if (a.m > 0)
        k_lp_build<<<(a.m + blk - 1) / blk, blk, 0, s>>>(a.gpos, a.gscale, a.m, 1.f / a.h, a.keys,
                                                        a.head, a.next, mask, a.smax, a.counters);
    *nlaunch = a.m > 0 ? 2 : 1;
    if (a.n > 0) {
        k_lp_query<<<(a.n + blk - 1) / blk, blk, 0, s>>>(a.pts, a.n, a.gpos, a.gscale, a.keys,
                                                        a.head, a.next, mask, a.h, a.smax, a.best,
                                                        a.arg, a.pending, a.counters);
        k_lp_exhaust<<<a.sms * 4, 256, 0, s>>>(a.pts, a.gpos, a.gscale, a.m, a.pending,
                                               a.counters, a.best, a.arg);
        *nlaunch += 2;
    }
    k_lp_partial<<<a.nb_partial, kMeanBlock, 0, s>>>(a.best, a.n, a.partial);
    k_lp_final<<<1, kMeanBlock, 0, s>>>(a.partial, a.nb_partial, a.n, a.loss);
    *nlaunch += 2;
    return cudaGetLastError();
}

}  // namespace gpv
