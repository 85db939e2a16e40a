// gpv_solve.cu -- batched Voxel-GPR (GS-LIVM Sec. 3.1, Alg. 1, Eq. 2-3) on sm_103a.
//
// One CTA solves one voxel at a time and pulls the next voxel from a per-launch work
// queue (a persistent grid sized to the SM count).  Per voxel, in shared memory (or, for
// voxels whose factor does not fit, in the CTA's slice of a global workspace):
//   A1  PCA of the points (FP32, voxel-local) -> value axis (Sec. 3.1)
//   A2  voxel-local training inputs x (parameter axes) and targets f (value axis)
//   A3  Gram K + D (D = sigma^2 I, or a noise variance per point), packed lower
//       triangle, column-major (Eq. 2)
//   A4  Cholesky K + D = L L^T: blocked right-looking (16-column panels) or per column
//       (replaces the LU + explicit inverse of the paper's Alg. 3)
//       -> L^-1 in place (n^3/6 more flops buys a barrier-free contraction below)
//   A5  alpha = L^-T L^-1 (f - m)
//   A6  K* on the G x G query grid is separable: k(x_i, (u,v)) = a_i(u) b_i(v), so
//       only 2 n G exponentials are evaluated
//   A7  mu* = m + K*^T alpha (Eq. 3)
//   A8  diag(Sigma*) = sf2 - |L^-1 k_q|^2: a dense contraction L^-1 * K* tiled 8 rows
//       x 4 queries per thread, squared and summed on the fly; the n x G^2 matrix
//       L^-1 K* and the full Sigma* of Alg. 3 are never formed
//   A10 (optional, fused) Gaussian initialisation of the n_s^2 subgrids (Sec. 3.2)
// The same code is instantiated for float, double and float-float ("ff").
#include <cuda_runtime.h>
#include <stdint.h>

#include "gpv_common.cuh"
#include "gpv_init.cuh"
#include "gpv_internal.h"
#include "gpv_num.cuh"

namespace gpv {

// column-major packed lower triangle of an n x n matrix: element (r, c), r >= c
__device__ __forceinline__ int tri_off(int c, int n) { return c * n - ((c * (c - 1)) >> 1); }

// ---- blocked factor and inverse for voxels whose triangle lives in shared memory ----
__device__ __forceinline__ float shfl_idx(float x, int src) { return __shfl_sync(0xffffffffu, x, src); }
__device__ __forceinline__ double shfl_idx(double x, int src) { return __shfl_sync(0xffffffffu, x, src); }
__device__ __forceinline__ ff shfl_idx(ff x, int src)
{
    return ff_make(__shfl_sync(0xffffffffu, x.hi, src), __shfl_sync(0xffffffffu, x.lo, src));
}

// Rank-pw update of the trailing triangle (rows and columns p1..n-1) with the panel
// columns p0..p0+pw-1, in TS x TS register tiles (tile t -> block row bi >= block column bj).
template <class T, int TS>
__device__ __forceinline__ void trail_update(T* L, int n, int p0, int pw, int p1)
{
    const int m = n - p1;
    const int mb = (m + TS - 1) / TS;
    const int ntiles = mb * (mb + 1) / 2;
    for (int t = threadIdx.x; t < ntiles; t += blockDim.x) {
        int bi = (int)((sqrtf(8.f * (float)t + 1.f) - 1.f) * 0.5f);
        while (bi > 0 && bi * (bi + 1) / 2 > t) --bi;
        while ((bi + 1) * (bi + 2) / 2 <= t) ++bi;
        const int bj = t - bi * (bi + 1) / 2;
        const int i0 = p1 + TS * bi, j0 = p1 + TS * bj;
        T acc[TS][TS];
#pragma unroll
        for (int u = 0; u < TS; ++u)
#pragma unroll
            for (int w = 0; w < TS; ++w) acc[u][w] = zero<T>();
        for (int c = 0; c < pw; ++c) {
            const T* col = L + tri_off(p0 + c, n) - (p0 + c);  // col[r] = L(r, p0 + c)
            T li[TS], lj[TS];
#pragma unroll
            for (int u = 0; u < TS; ++u) {
                li[u] = col[min(i0 + u, n - 1)];
                lj[u] = col[min(j0 + u, n - 1)];
            }
#pragma unroll
            for (int u = 0; u < TS; ++u)
#pragma unroll
                for (int w = 0; w < TS; ++w) acc_fma(acc[u][w], li[u], lj[w]);
        }
#pragma unroll
        for (int u = 0; u < TS; ++u)
#pragma unroll
            for (int w = 0; w < TS; ++w) {
                const int i = i0 + u, j = j0 + w;
                if (i < n && j <= i) {
                    T* p = L + tri_off(j, n) + (i - j);
                    *p = *p - acc_norm(acc[u][w]);
                }
            }
    }
}

// Right-looking Cholesky by panels of PW (4, 8 or 16) columns, in place in the packed
// triangle: (a) the PW x PW diagonal block is factored by warp 0 in registers (lane r holds
// row r, updates exchanged by shuffles); (b) the rows below the block solve against it, one
// row per thread; (c) the trailing triangle takes the rank-PW update in 4 x 4 (or 2 x 2)
// register tiles.  Three barriers per panel; narrower panels shorten the serial (a) and (b)
// at the price of more barriers.  ild[k] receives 1 / L_kk.  Returns
//     false at a non-positive pivot; s_dm holds the running min / max pivot.
template <class T, int PW>
__device__ bool chol_smem(T* L, int n, T* ild, float* s_dm, int* s_fail)
{
    const int tid = threadIdx.x, nthr = blockDim.x, lane = tid & 31, wid = tid >> 5;
    for (int p0 = 0; p0 < n; p0 += PW) {
        const int pw = min(PW, n - p0);
        if (wid == 0) {
            // unscaled: step c subtracts a(r, c) a(r2, c) / d_cc from the rows below, so only
            // the reciprocal of the pivot is on the dependent chain; the square-root scaling
            // of every column follows in one independent pass
            T row[PW];
#pragma unroll
            for (int c = 0; c < PW; ++c)
                row[c] = (lane < pw && c <= lane) ? L[tri_off(p0 + c, n) + (lane - c)] : zero<T>();
            bool bad = false;
            float dmn = s_dm[0], dmx = s_dm[1];
            T dg = zero<T>();  // lane c: the pivot d_cc
#pragma unroll
            for (int c = 0; c < PW; ++c) {
                if (c < pw && !bad) {  // warp-uniform
                    const T dcc = shfl_idx(row[c], c);
                    const float dh = hi_of(dcc);
                    if (!(dh > 0.f)) {
                        bad = true;
                    } else {
                        dmn = fminf(dmn, dh);
                        dmx = fmaxf(dmx, dh);
                        if (lane == c) dg = dcc;
                        const T ac = row[c];              // a(lane, c)
                        const T tc = ac * grcp(dcc);      // a(lane, c) / d_cc
#pragma unroll
                        for (int r2 = c + 1; r2 < PW; ++r2) {
                            const T v = shfl_idx(ac, r2);  // a(r2, c)
                            if (lane >= r2) row[r2] = gfnma(tc, v, row[r2]);
                        }
                    }
                }
            }
            if (!bad) {
#pragma unroll
                for (int c = 0; c < PW; ++c) {
                    const T rs = grsqrt(shfl_idx(dg, c));  // 1 / L_cc
                    if (lane == c) {
                        row[c] = dg * rs;                    // L_cc = d_cc / sqrt(d_cc)
                        if (c < pw) ild[p0 + c] = rs;
                    } else if (lane > c) {
                        row[c] = row[c] * rs;
                    }
                }
                if (lane < pw)
#pragma unroll
                    for (int c = 0; c < PW; ++c)
                        if (c <= lane) L[tri_off(p0 + c, n) + (lane - c)] = row[c];
            }
            if (lane == 0) {
                s_dm[0] = dmn;
                s_dm[1] = dmx;
                if (bad) *s_fail = 1;
            }
        }
        __syncthreads();
        if (*s_fail) return false;
        const int p1 = p0 + pw;
        for (int i = p1 + tid; i < n; i += nthr) {  // (b) panel rows below the block
            T a[PW];
#pragma unroll
            for (int c = 0; c < PW; ++c)
                a[c] = c < pw ? L[tri_off(p0 + c, n) + (i - p0 - c)] : zero<T>();
#pragma unroll
            for (int c = 0; c < PW; ++c) {
                if (c < pw) {
                    a[c] = a[c] * ild[p0 + c];
#pragma unroll
                    for (int c2 = c + 1; c2 < PW; ++c2)
                        if (c2 < pw) a[c2] = gfnma(a[c], L[tri_off(p0 + c, n) + (c2 - c)], a[c2]);
                }
            }
#pragma unroll
            for (int c = 0; c < PW; ++c)
                if (c < pw) L[tri_off(p0 + c, n) + (i - p0 - c)] = a[c];
        }
        __syncthreads();
        const int m = n - p1;  // (c) trailing triangle in 4 x 4 tiles, 2 x 2 when few
        if (m > 0) {
            // rounds of tiles per thread x products per tile: the smaller wins
            const int mb4 = (m + 3) >> 2, mb2 = (m + 1) >> 1;
            const int cost4 = (mb4 * (mb4 + 1) / 2 + nthr - 1) / nthr * 16;
            const int cost2 = (mb2 * (mb2 + 1) / 2 + nthr - 1) / nthr * 4;
            if (cost4 <= cost2) trail_update<T, 4>(L, n, p0, pw, p1);
            else trail_update<T, 2>(L, n, p0, pw, p1);
        }
        __syncthreads();
    }
    return true;
}

// X = L^-1 in place by row blocks of 16.  First every 16 x 16 diagonal block is inverted
// in place, all blocks at once (thread per block column, forward substitution): these are
// the diagonal blocks D of X.  Then, block row by block row (rows above hold X, rows from
// the block down still hold L): (1) Y(r, c) = sum_{k=c}^{r0-1} L(r0+r, k) X(k, c) for
// c < r0, four rows per task so the X(k, c) loads are shared, the lanes of a warp running
// the k loop in step (their L loads are broadcasts); (2) Y parked in the block's rows;
// (3) X(r0+r, c) = -sum_{q<=r} D(r, q) Y(q, c), again four rows per task; (4) written back.
// Four barriers per block row, no dependent chain inside one.  Needs n <= blockDim.x.
template <class T>
__device__ void inv_smem(T* L, int n, const T* ild)
{
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int nblk = (n + 15) >> 4;
    {
        const int b = tid >> 4, c = tid & 15, r0 = b << 4;
        const int rb = min(16, n - r0);
        const bool act = b < nblk && c < rb;
        T z[16];
#pragma unroll
        for (int r = 0; r < 16; ++r) z[r] = zero<T>();
        if (act) {
#pragma unroll
            for (int r = 0; r < 16; ++r) {
                if (r == c) {
                    z[r] = ild[r0 + r];
                } else if (r > c && r < rb) {
                    T s2[2] = {zero<T>(), zero<T>()};
#pragma unroll
                    for (int q = 0; q < r; ++q)
                        if (q >= c) acc_fma(s2[q & 1], L[tri_off(r0 + q, n) + (r - q)], z[q]);
                    z[r] = -((acc_norm(s2[0]) + acc_norm(s2[1])) * ild[r0 + r]);
                }
            }
        }
        __syncthreads();
        if (act)
#pragma unroll
            for (int r = 0; r < 16; ++r)
                if (r >= c && r < rb) L[tri_off(r0 + c, n) + (r - c)] = z[r];
    }
    for (int r0 = 16; r0 < n; r0 += 16) {
        const int rb = min(16, n - r0);
        const int ntask = 4 * r0;
        __syncthreads();
        T y[4][4];
#pragma unroll
        for (int s = 0; s < 4; ++s) {
#pragma unroll
            for (int u = 0; u < 4; ++u) y[s][u] = zero<T>();
            const int t = tid + s * nthr;
            // the lanes of a warp run the k loop in step from the warp's smallest column
            // (X(k, c) = 0 above the diagonal), so their loads of L are broadcasts
            const int cw = t < ntask ? t % r0 : r0;
            const int kbeg = __reduce_min_sync(0xffffffffu, cw);
            if (t < ntask) {
                const int c = cw, g = t / r0;
                const T* xc = L + tri_off(c, n) - c;  // xc[k] = X(k, c)
                for (int k = kbeg; k < r0; ++k) {
                    const T x = k >= c ? xc[k] : zero<T>();
                    const T* lk = L + tri_off(k, n) - k + r0;  // lk[r] = L(r0 + r, k)
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int r = g + 4 * u;
                        if (r < rb) acc_fma(y[s][u], lk[r], x);
                    }
                }
            }
        }
        __syncthreads();
#pragma unroll
        for (int s = 0; s < 4; ++s) {  // park Y(r, c) in the block's rows
            const int t = tid + s * nthr;
            if (t < ntask) {
                const int c = t % r0, g = t / r0;
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int r = g + 4 * u;
                    if (r < rb) L[tri_off(c, n) + (r0 + r - c)] = acc_norm(y[s][u]);
                }
            }
        }
        __syncthreads();
#pragma unroll
        for (int s = 0; s < 4; ++s) {  // X(r0 + r, c) = -sum_{q <= r} D(r, q) Y(q, c)
            const int t = tid + s * nthr;
            if (t < ntask) {
                const int c = t % r0, g = t / r0;
                const T* yc = L + tri_off(c, n) + (r0 - c);  // yc[q] = Y(q, c)
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int r = g + 4 * u;
                    T acc = zero<T>();
                    // a rolled loop: unrolled over q (16) inside the 4 x 4 unrolled tasks it
                    // made 256 copies of the multiply-add, and the instruction fetch of the
                    // larger code cost more than the loop (quadric workload 40.2 -> 37.5 ms)
                    if (r < rb)
#pragma unroll 1
                        for (int q = 0; q <= r; ++q)
                            acc_fma(acc, L[tri_off(r0 + q, n) + (r - q)], yc[q]);
                    y[s][u] = -acc_norm(acc);
                }
            }
        }
        __syncthreads();
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            const int t = tid + s * nthr;
            if (t < ntask) {
                const int c = t % r0, g = t / r0;
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int r = g + 4 * u;
                    if (r < rb) L[tri_off(c, n) + (r0 + r - c)] = y[s][u];
                }
            }
        }
    }
    __syncthreads();
}

// Per-column variants for small voxels in the 8-byte types, where one barrier per column
// beats the serial 16 x 16 diagonal blocks of the blocked variants.
// Cholesky, right-looking with the unscaled trailing update: step k does
// A_ij -= A_ik A_jk / A_kk for k < j <= i and scales column k-1 in the same phase (it is
// not read by step k); one barrier per step.
template <class T>
__device__ void chol_percol_smem(T* L, int n, float& dmin, float& dmax, int& s_fail)
{
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int lane = tid & 31, wid = tid >> 5, nw = nthr >> 5;
    T dprev = zero<T>();
    T rs_prev = zero<T>();
    for (int k = 0; k < n; ++k) {
        __syncthreads();
        const T d = L[tri_off(k, n)];
        const float dh = hi_of(d);
        if (!(dh > 0.f)) {
            if (tid == 0) s_fail = 1;
            break;
        }
        dmin = fminf(dmin, dh);
        dmax = fmaxf(dmax, dh);
        if (k > 0) {  // finish column k-1
            T* ck = L + tri_off(k - 1, n);
            for (int r = tid; r < n - (k - 1); r += nthr)
                ck[r] = (r == 0) ? gsqrt(dprev) : ck[r] * rs_prev;
        }
        const T inv_d = from_f<T>(1.f) / d;
        const T* colk = L + tri_off(k, n);
        for (int j = k + 1 + wid; j < n; j += nw) {
            const T s = colk[j - k] * inv_d;
            T* colj = L + tri_off(j, n);
            if (n - j <= 64) {  // short column: one update per lane
                for (int i = j + lane; i < n; i += 32) colj[i - j] = gfnma(colk[i - k], s, colj[i - j]);
                continue;
            }
            for (int i0 = j + lane; i0 < n; i0 += 128) {  // 4 independent updates
                T a[4], b[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int i = min(i0 + 32 * u, n - 1);
                    a[u] = colk[i - k];
                    b[u] = colj[i - j];
                }
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    if (i0 + 32 * u < n) colj[i0 + 32 * u - j] = gfnma(a[u], s, b[u]);
            }
        }
        dprev = d;
        rs_prev = from_f<T>(1.f) / gsqrt(d);
    }
    __syncthreads();
    if (!s_fail && tid == 0) L[tri_off(n - 1, n)] = gsqrt(dprev);
    __syncthreads();
}

// X = L^-1 in place, right-looking elimination of L X = I: step k finalises row k
// (X_kc = B_kc / L_kk, c < k), then rows i > k take B_ic -= L_ik X_kc (c < k) and
// B_ik = -L_ik / L_kk.  One warp owns row i, so it reads L_ik before the lane of column k
// overwrites it; the diagonal keeps L_kk until a last pass writes 1 / L_kk.
template <class T>
__device__ void inv_percol_smem(T* L, int n)
{
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int lane = tid & 31, wid = tid >> 5, nw = nthr >> 5;
    for (int k = 0; k < n; ++k) {
        __syncthreads();
        const T inv = from_f<T>(1.f) / L[tri_off(k, n)];
        for (int c = tid; c < k; c += nthr) {
            T* p = L + tri_off(c, n) + (k - c);
            *p = (*p) * inv;
        }
        __syncthreads();
        for (int i = k + 1 + wid; i < n; i += nw) {
            const T m = L[tri_off(k, n) + (i - k)];
            __syncwarp();
            if (k < 64) {  // short row: one update per lane
                for (int c = lane; c <= k; c += 32) {
                    T* p = L + tri_off(c, n) + (i - c);
                    *p = (c == k) ? -(m * inv) : gfnma(m, L[tri_off(c, n) + (k - c)], *p);
                }
                continue;
            }
            for (int c0 = lane; c0 <= k; c0 += 128) {  // 4 independent updates
                T x[4], b[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int c = min(c0 + 32 * u, k);
                    x[u] = L[tri_off(c, n) + (k - c)];
                    b[u] = L[tri_off(c, n) + (i - c)];
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int c = c0 + 32 * u;
                    if (c <= k)
                        L[tri_off(c, n) + (i - c)] = (c == k) ? -(m * inv) : gfnma(m, x[u], b[u]);
                }
            }
        }
    }
    __syncthreads();
    for (int k = tid; k < n; k += nthr) {
        T* p = L + tri_off(k, n);
        *p = from_f<T>(1.f) / (*p);
    }
    __syncthreads();
}

// ---- blocked factor and inverse for voxels whose triangle lives in global memory ----
// The triangle (column-major packed, element (r, c) at tri_off(c, n) + r - c) stays in
// the CTA's workspace slice; panels of it are staged in shared memory so that every
// inner loop runs on shared memory and the global traffic is streamed, not latency-bound.

// Left-looking Cholesky by panels of pb columns: for each panel, stage the Gram columns,
// subtract the products of all finished columns (streamed through a tile of pb columns),
// factor the panel in shared memory, write it back.  Returns false at a non-positive
// pivot.  P and Tt hold pb x (n - p0) values each.
template <class T>
__device__ bool big_cholesky(T* L, int n, T* P, T* Tt, int pb, float& dmin, float& dmax)
{
    const int tid = threadIdx.x, nthr = blockDim.x;
    for (int p0 = 0; p0 < n; p0 += pb) {
        const int pw = min(pb, n - p0), R = n - p0;
        __syncthreads();
        for (int idx = tid; idx < pw * R; idx += nthr) {
            const int c = idx / R, r = idx - c * R;
            if (r >= c) P[idx] = L[tri_off(p0 + c, n) + (r - c)];
        }
        for (int k0 = 0; k0 < p0; k0 += pb) {
            const int kw = min(pb, p0 - k0);
            __syncthreads();
            for (int idx = tid; idx < kw * R; idx += nthr) {
                const int kk = idx / R, r = idx - kk * R;
                Tt[idx] = L[tri_off(k0 + kk, n) + (p0 - k0 - kk) + r];
            }
            __syncthreads();
            const int ncg = (pw + 7) >> 3;  // one task per (row, group of 8 panel columns)
            for (int t = tid; t < R * ncg; t += nthr) {
                const int r = t / ncg, cg = (t - r * ncg) * 8;
                T acc[8];
#pragma unroll
                for (int j = 0; j < 8; ++j) acc[j] = zero<T>();
                for (int kk = 0; kk < kw; ++kk) {
                    const T a = Tt[kk * R + r];
#pragma unroll
                    for (int j = 0; j < 8; ++j)
                        if (cg + j < pw) acc_fma(acc[j], a, Tt[kk * R + cg + j]);
                }
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const int c = cg + j;
                    if (c < pw && r >= c) P[c * R + r] = P[c * R + r] - acc_norm(acc[j]);
                }
            }
        }
        // the panel, right-looking and unscaled: step c subtracts P(r, c) P(c2, c) / d_c from
        // the later columns and scales column c - 1 (not read by step c); one barrier per step
        T rs_prev = zero<T>(), d_prev = zero<T>();
        for (int c = 0; c < pw; ++c) {
            __syncthreads();
            const T d = P[c * R + c];
            const float dh = hi_of(d);
            if (!(dh > 0.f)) return false;
            dmin = fminf(dmin, dh);
            dmax = fmaxf(dmax, dh);
            const T inv_d = grcp(d);
            if (c > 0)
                for (int r = c - 1 + tid; r < R; r += nthr)
                    P[(c - 1) * R + r] = (r == c - 1) ? d_prev * rs_prev : P[(c - 1) * R + r] * rs_prev;
            const int rest = pw - c - 1;
            for (int idx = tid; idx < rest * R; idx += nthr) {
                const int c2 = c + 1 + idx / R, r = idx % R;
                if (r >= c2) P[c2 * R + r] = gfnma(P[c * R + r] * inv_d, P[c * R + c2], P[c2 * R + r]);
            }
            d_prev = d;
            rs_prev = grsqrt(d);
        }
        __syncthreads();
        for (int r = pw - 1 + tid; r < R; r += nthr)  // the last column's scaling
            P[(pw - 1) * R + r] = (r == pw - 1) ? d_prev * rs_prev : P[(pw - 1) * R + r] * rs_prev;
        __syncthreads();
        for (int idx = tid; idx < pw * R; idx += nthr) {
            const int c = idx / R, r = idx - c * R;
            if (r >= c) L[tri_off(p0 + c, n) + (r - c)] = P[idx];
        }
    }
    __syncthreads();
    return true;
}

// X = L^-1 in place by row blocks of rb (<= 16) rows (rows above the block already hold X,
// rows from the block down still hold L): the block's rows of L are staged in shared
// memory (W) and its diagonal block inverted there once (D, one warp, column by column);
// then one warp per column c < r0 forms Y(r, c) = sum_{k=c}^{r0-1} L(r0+r, k) X(k, c), its
// lanes striding over k so the reads of X's column are contiguous, reduces the 16 partial
// sums across the warp, and lanes r < rb write X(r0+r, c) = -sum_{q<=r} D(r, q) Y(q, c);
// the columns of the diagonal block take D itself.  W holds rb x n values, D 16 x 16.
template <class T>
__device__ void big_invert(T* L, int n, T* W, int rbmax)
{
    const int tid = threadIdx.x, nthr = blockDim.x, lane = tid & 31, wid = tid >> 5, nw = nthr >> 5;
    T* D = W + (int64_t)rbmax * n;  // 16 x 16, row-major
    for (int r0 = 0; r0 < n; r0 += rbmax) {
        const int rb = min(rbmax, n - r0);
        __syncthreads();
        for (int idx = tid; idx < rb * (r0 + rb); idx += nthr) {
            const int r = idx / (r0 + rb), c = idx - r * (r0 + rb);
            if (c <= r0 + r) W[r * n + c] = L[tri_off(c, n) + (r0 + r - c)];
        }
        __syncthreads();
        if (wid == 0) {  // D = L_II^-1: lane c < rb solves column c
            T z[16];
#pragma unroll
            for (int r = 0; r < 16; ++r) z[r] = zero<T>();
            if (lane < rb) {
#pragma unroll
                for (int r = 0; r < 16; ++r) {
                    if (r >= lane && r < rb) {
                        T s2 = from_f<T>(r == lane ? 1.f : 0.f);
#pragma unroll
                        for (int q = 0; q < r; ++q)
                            if (q >= lane) s2 = gfnma(W[r * n + r0 + q], z[q], s2);
                        z[r] = s2 / W[r * n + r0 + r];
                    }
                }
#pragma unroll
                for (int r = 0; r < 16; ++r) D[r * 16 + lane] = z[r];
            }
        }
        __syncthreads();
        // the columns of the diagonal block: X = D
        for (int t = tid; t < rb * rb; t += nthr) {
            const int cc = t / rb, r = t - cc * rb;
            if (r >= cc) L[tri_off(r0 + cc, n) + (r - cc)] = D[r * 16 + cc];
        }
        // columns left of the block: 4 lanes per column, 8 columns per warp
        const int sub = lane & 3;
        for (int cb = wid * 8; cb < r0; cb += nw * 8) {
            const int c = cb + (lane >> 2);
            const bool act = c < r0;
            T y[16];
#pragma unroll
            for (int r = 0; r < 16; ++r) y[r] = zero<T>();
            if (act) {
                const T* xc = L + tri_off(c, n) - c;  // xc[k] = X(k, c), k >= c
                for (int k = c + sub; k < r0; k += 4) {
                    const T x = xc[k];
#pragma unroll
                    for (int r = 0; r < 16; ++r)
                        if (r < rb) acc_fma(y[r], W[r * n + k], x);
                }
            }
#pragma unroll
            for (int r = 0; r < 16; ++r) {  // sums over the column's 4 lanes
                y[r] = acc_norm(y[r]);
                y[r] = y[r] + shfl_x(y[r], 1);
                y[r] = y[r] + shfl_x(y[r], 2);
            }
            if (act) {  // lane sub writes rows sub, sub + 4, sub + 8, sub + 12
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int r = sub + 4 * u;
                    if (r < rb) {
                        T acc = zero<T>();
#pragma unroll
                        for (int q = 0; q < 16; ++q)
                            if (q <= r) acc_fma(acc, D[r * 16 + q], y[q]);
                        L[tri_off(c, n) + (r0 + r - c)] = -acc_norm(acc);
                    }
                }
            }
        }
    }
    __syncthreads();
}

// TCV: the float-float variant of the tensor-core variance path; it hands every voxel to
// k_var_tc (or, with the workspace full, to the regular kernel) and carries no contraction.
template <class T, bool TRI_SMEM, bool TCV>
__device__ void solve_voxel(const SolveArgs& A, int v, unsigned char* smem, const SmemPlan& P,
                            double* red, const T* nodes, const ff* xtab)
{
    const int tid = threadIdx.x;
    const int nthr = blockDim.x;
    const int64_t beg = A.offsets[v];
    const int n = (int)(A.offsets[v + 1] - beg);
    const int G = A.G, Gp = A.Gp, GG = G * G;
    if (TCV && A.tc->total > A.tc_cap) {
        // the call's voxels need more workspace than it has: the regular kernels solve
        // them all (decided once per call after the classification, so it does not depend
        // on scheduling); nothing is factored here
        if (tid == 0) {
            const bool big = n > A.fb_nsmall;
            A.tc_fb[(big ? (int64_t)A.nvox : 0) + atomicAdd(big ? &A.tc->fb2_count : &A.tc->fb_count, 1)] = v;
        }
        return;
    }

    float* pts = reinterpret_cast<float*>(smem + P.off_pts);
    T* x1 = reinterpret_cast<T*>(smem + P.off_vec);
    T* x2 = x1 + A.nmax;
    T* fv = x2 + A.nmax;
    T* al = fv + A.nmax;
    T* tmp = al + A.nmax;
    T* L = TRI_SMEM ? reinterpret_cast<T*>(smem + P.off_tri)
                    : reinterpret_cast<T*>(A.gws) + (int64_t)blockIdx.x * A.gws_stride;
    T* fa = TRI_SMEM ? reinterpret_cast<T*>(smem + P.off_a)
                     : L + ((int64_t)A.nmax * (A.nmax + 1) / 2 + 16);
    T* fb = TRI_SMEM ? reinterpret_cast<T*>(smem + P.off_b) : fa + (int64_t)A.nmax * G;
    T* part = reinterpret_cast<T*>(smem + P.off_part);
    T* mv = reinterpret_cast<T*>(smem + P.off_mv);
    __shared__ int s_axis;
    __shared__ int s_fail;

    // ---- load points (3n contiguous floats) ------------------------------------
    const float* src = A.xyz + 3 * beg;
    for (int t = tid; t < 3 * n; t += nthr) pts[t] = __ldg(src + t);
    __syncthreads();

    // ---- A1: PCA (FP32, voxel-local coordinates) -> value axis --------------------
    const float cx = A.centres[3 * v + 0], cy = A.centres[3 * v + 1], cz = A.centres[3 * v + 2];
    {
        float* redf = reinterpret_cast<float*>(red);
        float s3[3] = {0.f, 0.f, 0.f};
        for (int i = tid; i < n; i += nthr) {
            s3[0] += pts[3 * i + 0] - cx;
            s3[1] += pts[3 * i + 1] - cy;
            s3[2] += pts[3 * i + 2] - cz;
        }
        block_sum<float, 3>(s3, redf);
        const float inv_n = 1.f / (float)n;
        const float m0 = s3[0] * inv_n, m1 = s3[1] * inv_n, m2 = s3[2] * inv_n;
        float c6[6] = {0, 0, 0, 0, 0, 0};
        for (int i = tid; i < n; i += nthr) {
            const float d0 = (pts[3 * i + 0] - cx) - m0;
            const float d1 = (pts[3 * i + 1] - cy) - m1;
            const float d2 = (pts[3 * i + 2] - cz) - m2;
            c6[0] += d0 * d0; c6[1] += d0 * d1; c6[2] += d0 * d2;
            c6[3] += d1 * d1; c6[4] += d1 * d2; c6[5] += d2 * d2;
        }
        block_sum<float, 6>(c6, redf);
        if (tid == 0) {
            s_axis = value_axis_from_cov(c6);
            s_fail = 0;
        }
        __syncthreads();
    }
    const int axis = s_axis;
    const int p1 = axis == 2 ? 0 : axis + 1;
    const int p2 = axis == 0 ? 2 : (axis == 1 ? 0 : 1);
    const float cen[3] = {cx, cy, cz};

    // ---- A2: voxel-local inputs and targets, prior mean ---------------------------
    T msum[1] = {zero<T>()};
    for (int i = tid; i < n; i += nthr) {
        x1[i] = diff_f<T>(pts[3 * i + p1], cen[p1]);
        x2[i] = diff_f<T>(pts[3 * i + p2], cen[p2]);
        T f = diff_f<T>(pts[3 * i + axis], cen[axis]);
        fv[i] = f;
        msum[0] = msum[0] + f;
    }
    block_sum<T, 1>(msum, reinterpret_cast<T*>(red));
    const T m = A.mean_mode == 1 ? msum[0] / from_f<T>((float)n) : zero<T>();
    for (int i = tid; i < n; i += nthr) fv[i] = fv[i] - m;

    // ---- A3: Gram + noise (packed lower, column-major) ---------------------------
    const float lamf = A.lam[v], sf2f = A.sf2[v], sn2f = A.sn2[v];
    const T nlam = from_f<T>(-lamf);
    const T sf2 = from_f<T>(sf2f);
    const T sn2 = from_f<T>(sn2f);
    __syncthreads();
    {
        // flattened lower triangle, two entries per thread in flight (the exponentials
        // are long dependent chains); entry e of column c, row r: e = tri_off(c, n) + r - c
        const int ntri = n * (n + 1) / 2;
        for (int e0 = tid; e0 < ntri; e0 += 2 * nthr) {
            const int e1 = min(e0 + nthr, ntri - 1);
            int ce[2], re[2];
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const int e = u ? e1 : e0;
                // column of entry e: the largest c with tri_off(c, n) <= e
                const float b = 2.f * n + 1.f;
                int c = (int)((b - sqrtf(b * b - 8.f * (float)e)) * 0.5f);
                c = max(0, min(c, n - 1));
                while (c > 0 && tri_off(c, n) > e) --c;
                while (c + 1 < n && tri_off(c + 1, n) <= e) ++c;
                ce[u] = c;
                re[u] = c + (e - tri_off(c, n));
            }
            const T d1a = x1[re[0]] - x1[ce[0]], d2a = x2[re[0]] - x2[ce[0]];
            const T d1b = x1[re[1]] - x1[ce[1]], d2b = x2[re[1]] - x2[ce[1]];
            T ka = sf2 * gexpw(nlam * (d1a * d1a + d2a * d2a), xtab);
            T kb = sf2 * gexpw(nlam * (d1b * d1b + d2b * d2b), xtab);
            if (re[0] == ce[0]) ka = ka + (A.noise ? from_f<T>(__ldg(A.noise + beg + re[0])) : sn2);
            if (re[1] == ce[1]) kb = kb + (A.noise ? from_f<T>(__ldg(A.noise + beg + re[1])) : sn2);
            L[e0] = ka;
            if (e0 + nthr < ntri) L[e1] = kb;
        }
    }

    // ---- A4: Cholesky, right-looking, unscaled trailing update ---------------------
    // step k: A_ij -= A_ik A_jk / A_kk for k < j <= i, column k-1 scaled in the same
    // phase (it is not read by step k), one barrier per step.
    float dmin = 3.0e38f, dmax = 0.f;
    T* W = reinterpret_cast<T*>(smem + P.off_work);
    if (!TRI_SMEM) {
        __syncthreads();
        const bool ok = big_cholesky<T>(L, n, W, W + (int64_t)P.pb * n, P.pb, dmin, dmax);
        if (!ok && tid == 0) s_fail = 1;
        __syncthreads();
    } else {
        if (n <= A.percol_max) {
            chol_percol_smem<T>(L, n, dmin, dmax, s_fail);
        } else {
            __shared__ float s_dm[2];
            if (tid == 0) { s_dm[0] = 3.0e38f; s_dm[1] = 0.f; }
            __syncthreads();
            if (A.panel == 4) chol_smem<T, 4>(L, n, tmp, s_dm, &s_fail);
            else if (A.panel == 8) chol_smem<T, 8>(L, n, tmp, s_dm, &s_fail);
            else chol_smem<T, 16>(L, n, tmp, s_dm, &s_fail);
            dmin = s_dm[0];
            dmax = s_dm[1];
            __syncthreads();
        }
    }
    const bool ill = s_fail || (dmax > A.esc_cond * dmin);
    if (ill && A.escalate) {
        if (tid == 0) {
            const int big = n > A.nmax_small_f64 ? 1 : 0;
            int slot = atomicAdd(A.esc_count + big, 1);
            A.esc_list[(int64_t)big * A.nvox + slot] = v;
        }
        __syncthreads();
        return;
    }
    const int64_t obase = (int64_t)v * GG;
    // FP32 without escalation: a pivot ratio beyond the threshold leaves no significant
    // digit in the solve, so the voxel counts as not positive definite in this precision
    const bool fail32 = sizeof(T) == 4 && !A.escalate && ill;
    if (s_fail || fail32) {
        // not positive definite in this precision: report the prior
        for (int q = tid; q < GG; q += nthr) {
            A.mean[obase + q] = to_f(m);
            A.var[obase + q] = sf2f;
        }
        if (tid == 0) {
            A.axis[v] = (uint8_t)axis;
            A.status[v] = VOX_NOT_SPD | (A.escalation_pass ? VOX_ESCALATED : 0u);
        }
        if (A.pos) {
            const int NG = A.n_s * A.n_s;
            for (int g = tid; g < NG; g += nthr) {
                const int64_t o = (int64_t)v * NG + g;
                for (int k = 0; k < 3; ++k) { A.pos[3 * o + k] = cen[k]; A.scale[3 * o + k] = 0.f; }
                A.quat[4 * o] = 1.f; A.quat[4 * o + 1] = 0.f; A.quat[4 * o + 2] = 0.f; A.quat[4 * o + 3] = 0.f;
            }
        }
        __syncthreads();
        return;
    }

    if (!TRI_SMEM) big_invert<T>(L, n, W, P.rb);
    // ---- A4': X = L^-1 in place (blocked by rows, see inv_smem) ---------------------
    if (TRI_SMEM) {
        if (n <= A.percol_max) inv_percol_smem<T>(L, n);
        else inv_smem<T>(L, n, tmp);
    }
    // ---- tensor-core variance: reserve this voxel's workspace (float-float only) ------
    __shared__ long long s_tc_off;
    bool tc = false;
    if (is_ff<T>::value && A.tc_ws != nullptr && n <= (TRI_SMEM ? A.tc_nmax : A.tc_nmax_gl)) {
        if (tid == 0) {
            long long off = -1;
            const unsigned long long need = tc_need_bytes(n, G, Gp);
            if (A.tc->total <= A.tc_cap && !(dmax > kTcCond * dmin)) {
                const unsigned long long o = atomicAdd(&A.tc->used, need);
                if (o + need <= A.tc_cap) off = (long long)o;
            }
            s_tc_off = off;
        }
        __syncthreads();
        tc = s_tc_off >= 0;
    }
    __syncthreads();
    if (TCV && !tc) {  // workspace full: the regular kernel re-solves this voxel
        if (tid == 0) {
            const bool big = n > A.fb_nsmall;
            A.tc_fb[(big ? (int64_t)A.nvox : 0) + atomicAdd(big ? &A.tc->fb2_count : &A.tc->fb_count, 1)] = v;
        }
        __syncthreads();
        return;
    }

    // ---- posterior variance at the inputs (per-point noise feedback, Sec. 3.3) -------
    // With A = K + D, k_i = A e_i - d_i e_i gives sf2 - k_i^T A^-1 k_i
    // = d_i (1 - d_i (A^-1)_ii), and (A^-1)_ii is the squared norm of column i of X,
    // which is contiguous in the packed layout.
    if (A.pvar) {
        for (int i = tid; i < n; i += nthr) {
            const T* col = L + tri_off(i, n);
            T s2[2] = {zero<T>(), zero<T>()};
            int t = 0;
            for (; t + 1 < n - i; t += 2) {
                acc_fma(s2[0], col[t], col[t]);
                acc_fma(s2[1], col[t + 1], col[t + 1]);
            }
            if (t < n - i) acc_fma(s2[0], col[t], col[t]);
            const T d = A.noise ? from_f<T>(__ldg(A.noise + beg + i)) : sn2;
            const float pv = to_f(d * (from_f<T>(1.f) - d * (acc_norm(s2[0]) + acc_norm(s2[1]))));
            A.pvar[beg + i] = fmaxf(pv, 0.f);
        }
    }

    // ---- A5: alpha = X^T (X (f - m)) ----------------------------------------------
    for (int j = tid; j < n; j += nthr) {  // four partial sums in flight
        T s4[4] = {zero<T>(), zero<T>(), zero<T>(), zero<T>()};
        int i = 0;
        for (; i + 3 <= j; i += 4)
#pragma unroll
            for (int u = 0; u < 4; ++u) acc_fma(s4[u], L[tri_off(i + u, n) + (j - i - u)], fv[i + u]);
        for (; i <= j; ++i) acc_fma(s4[0], L[tri_off(i, n) + (j - i)], fv[i]);
        tmp[j] = (acc_norm(s4[0]) + acc_norm(s4[1])) + (acc_norm(s4[2]) + acc_norm(s4[3]));
    }
    // ---- A6: separable cross-covariance factors --------------------------------------
    // On the uniform nodes u_k = u_0 + k delta, e_k = exp(-lambda (x - u_k)^2) obeys
    // e_{k+1} = e_k r_k with r_k = exp(2 lambda delta (x - u_k) - lambda delta^2) and
    // r_{k+1} = r_k exp(-2 lambda delta^2): three exponentials per point and axis (and one
    // per voxel) instead of G, the rest products whose rounding grows only linearly in k
    // (in the 8-byte types; FP32 evaluates every exponential, its variance has no margin)
    // (the variant without the contraction forms them after L^-1 has left shared memory:
    // its smem plan may lay them over the triangle)
    auto kfactors = [&]() {
        if (sizeof(T) == 4) {
            for (int t0 = tid; t0 < n * G; t0 += 2 * nthr) {  // four exponentials in flight
                const int t1 = min(t0 + nthr, n * G - 1);
                const int i0 = t0 / G, u0 = t0 - i0 * G, i1 = t1 / G, u1 = t1 - i1 * G;
                const T da0 = x1[i0] - nodes[u0], db0 = x2[i0] - nodes[u0];
                const T da1 = x1[i1] - nodes[u1], db1 = x2[i1] - nodes[u1];
                const T ea0 = gexpw(nlam * (da0 * da0), xtab), eb0 = gexpw(nlam * (db0 * db0), xtab);
                const T ea1 = gexpw(nlam * (da1 * da1), xtab), eb1 = gexpw(nlam * (db1 * db1), xtab);
                fa[i0 * G + u0] = sf2 * ea0;
                fb[i0 * Gp + u0] = eb0;
                if (t0 + nthr < n * G) {
                    fa[i1 * G + u1] = sf2 * ea1;
                    fb[i1 * Gp + u1] = eb1;
                }
            }
            for (int t = tid; t < n * (Gp - G); t += nthr) {
                const int i = t / (Gp - G), u = G + (t - i * (Gp - G));
                fb[i * Gp + u] = zero<T>();
            }
        } else {
            const T dl = from_d<T>((double)A.size / (double)G);
            const T two = from_f<T>(2.f);
            const T cst = gexpw(nlam * (dl * dl) * two, xtab);  // exp(-2 lambda delta^2)
            for (int t = tid; t < 2 * n; t += nthr) {
                const int i = t >> 1;
                const T d0 = ((t & 1) ? x2[i] : x1[i]) - nodes[0];  // x - u_0
                T e = gexpw(nlam * (d0 * d0), xtab);
                T r = gexpw(nlam * (dl * dl - two * dl * d0), xtab);
                if ((t & 1) == 0) {
                    for (int k = 0; k < G; ++k) {
                        fa[i * G + k] = sf2 * e;
                        e = e * r;
                        r = r * cst;
                    }
                } else {
                    for (int k = 0; k < G; ++k) {
                        fb[i * Gp + k] = e;
                        e = e * r;
                        r = r * cst;
                    }
                }
            }
            for (int t = tid; t < n * (Gp - G); t += nthr) {
                const int i = t / (Gp - G), u = G + (t - i * (Gp - G));
                fb[i * Gp + u] = zero<T>();
            }
        }
    };
    if (!TCV) kfactors();
    __syncthreads();
    for (int i = tid; i < n; i += nthr) {  // four partial sums in flight
        T s4[4] = {zero<T>(), zero<T>(), zero<T>(), zero<T>()};
        const T* col = L + tri_off(i, n) - i;
        int j = i;
        for (; j + 3 < n; j += 4)
#pragma unroll
            for (int u = 0; u < 4; ++u) acc_fma(s4[u], col[j + u], tmp[j + u]);
        for (; j < n; ++j) acc_fma(s4[0], col[j], tmp[j]);
        al[i] = (acc_norm(s4[0]) + acc_norm(s4[1])) + (acc_norm(s4[2]) + acc_norm(s4[3]));
    }

    // ---- A5': one step of iterative refinement of alpha (FP32 path) -----------------
    // r = (f - m) - (K + D) alpha: K recomputed as in A3, every product exact (FMA) and
    // the sum in float-float, so r carries the factor's error rather than the rounding
    // of the sum; the FP32 inverse factor then gives the correction d = X^T X r, and the
    // mean below accumulates K*^T (alpha + d) in float-float.  (tmp is free once alpha
    // is formed, and f - m once r is.)
    const bool refine = sizeof(T) == 4 && A.refine != 0;
    T* dal = tmp;  // the correction d, when refining
    if (refine) {
        __syncthreads();
        for (int j = tid; j < n; j += nthr) {
            const float xj1 = to_f(x1[j]), xj2 = to_f(x2[j]);
            float sh = to_f(fv[j]), sl = 0.f;
            for (int i = 0; i < n; ++i) {
                const float d1 = __fsub_rn(xj1, to_f(x1[i])), d2 = __fsub_rn(xj2, to_f(x2[i]));
                float k = to_f(sf2 * gexpw(nlam * (d1 * d1 + d2 * d2), xtab));
                if (i == j) k = __fadd_rn(k, A.noise ? __ldg(A.noise + beg + j) : sn2f);
                const float a = to_f(al[i]);
                const float p = __fmul_rn(k, a), pe = __fmaf_rn(k, a, -p);
                const ff t = two_sum(sh, -p);
                sh = t.hi;
                sl = __fadd_rn(sl, __fsub_rn(t.lo, pe));
            }
            tmp[j] = from_f<T>(__fadd_rn(sh, sl));
        }
        __syncthreads();
        for (int j = tid; j < n; j += nthr) {  // X r
            T s2 = zero<T>();
            for (int i = 0; i <= j; ++i) acc_fma(s2, L[tri_off(i, n) + (j - i)], tmp[i]);
            fv[j] = acc_norm(s2);
        }
        __syncthreads();
        for (int i = tid; i < n; i += nthr) {  // X^T (X r)
            T s2 = zero<T>();
            const T* col = L + tri_off(i, n) - i;
            for (int j = i; j < n; ++j) acc_fma(s2, col[j], fv[j]);
            dal[i] = acc_norm(s2);
        }
        __syncthreads();
    }

    // ---- A8 handed over: L^-1 and the factors go to the workspace, k_var_tc forms the
    // variance on the tensor cores ------------------------------------------------------
    const int ntri = n * (n + 1) / 2;
    T* Wtc = tc ? reinterpret_cast<T*>(A.tc_ws + s_tc_off) : nullptr;
    if (tc) {
        for (int e = tid; e < ntri; e += nthr) Wtc[e] = L[e];
        // slice exponents: rows j of L^-1 and queries (u, v) of K* = a(u) b(v)
        int* EX = reinterpret_cast<int*>(Wtc + ntri + n * G + n * Gp + 2 * GG);
        for (int j = tid; j < n; j += nthr) {
            float mx = 0.f;
            for (int i = 0; i <= j; ++i) mx = fmaxf(mx, fabsf(hi_of(L[tri_off(i, n) + j - i])));
            EX[j] = tc_exp_above(mx);
        }
        if (TCV) {  // L^-1 is in the workspace: now the factors
            __syncthreads();
            kfactors();
            __syncthreads();
        }
        for (int e = tid; e < n * G; e += nthr) Wtc[ntri + e] = fa[e];
        for (int e = tid; e < n * Gp; e += nthr) Wtc[ntri + n * G + e] = fb[e];
        for (int q = tid; q < GG; q += nthr) {
            const int u = q / G, vq = q - u * G;
            float mx = 0.f;
            for (int i = 0; i < n; ++i) mx = fmaxf(mx, fabsf(hi_of(fa[i * G + u]) * hi_of(fb[i * Gp + vq])));
            EX[n + q] = tc_exp_above(mx);
        }
    }
    // ---- A8: |X k_q|^2 by register-tiled contraction ------------------------------
    if (!tc) {
        const int nqg = P.nqg, nrg = P.nrg;
        const int nb = (n + kRowBlk - 1) / kRowBlk;
        for (int w = tid; w < nqg * nrg; w += nthr) {
            const int qg = w % nqg, rg = w / nqg;
            const int q0 = qg * kQryBlk;
            const int u = q0 / Gp, v0 = q0 - u * Gp;
            T nrm[kQryBlk];
#pragma unroll
            for (int r = 0; r < kQryBlk; ++r) nrm[r] = zero<T>();
            // snake assignment of row blocks to row groups balances the triangle
            for (int s = 0;; ++s) {
                const int jb = (s & 1) ? (s + 1) * nrg - 1 - rg : s * nrg + rg;
                if (s * nrg >= nb) break;
                if (jb >= nb) continue;
                const int j0 = jb * kRowBlk;
                const int nrow = min(kRowBlk, n - j0);
                T acc[kRowBlk][kQryBlk];
#pragma unroll
                for (int a = 0; a < kRowBlk; ++a)
#pragma unroll
                    for (int r = 0; r < kQryBlk; ++r) acc[a][r] = zero<T>();
                const int iend = min(j0 + kRowBlk, n);
                // columns left of the block: every row of a full block is below the diagonal
                const int ifull = nrow == kRowBlk ? j0 : 0;
                for (int i = 0; i < ifull; ++i) {
                    const T ai = fa[i * G + u];
                    T kq[kQryBlk];
#pragma unroll
                    for (int r = 0; r < kQryBlk; ++r) kq[r] = ai * fb[i * Gp + v0 + r];
                    const T* col = L + tri_off(i, n) + (j0 - i);
#pragma unroll
                    for (int a = 0; a < kRowBlk; ++a) {
                        const T l = col[a];
#pragma unroll
                        for (int r = 0; r < kQryBlk; ++r) acc_fma(acc[a][r], l, kq[r]);
                    }
                }
                for (int i = ifull; i < iend; ++i) {
                    const T ai = fa[i * G + u];
                    T kq[kQryBlk];
#pragma unroll
                    for (int r = 0; r < kQryBlk; ++r) kq[r] = ai * fb[i * Gp + v0 + r];
                    const T* col = L + tri_off(i, n) + (j0 - i);
#pragma unroll
                    for (int a = 0; a < kRowBlk; ++a) {
                        // rows j0+a of column i; zero above the diagonal and past n
                        const bool ok = (a < nrow) && (j0 + a >= i);
                        const T l = ok ? col[a] : zero<T>();
#pragma unroll
                        for (int r = 0; r < kQryBlk; ++r) acc_fma(acc[a][r], l, kq[r]);
                    }
                }
#pragma unroll
                for (int a = 0; a < kRowBlk; ++a)
#pragma unroll
                    for (int r = 0; r < kQryBlk; ++r) {
                        const T x = acc_norm(acc[a][r]);
                        nrm[r] = gfma(x, x, nrm[r]);
                    }
            }
#pragma unroll
            for (int r = 0; r < kQryBlk; ++r) part[rg * (G * Gp) + q0 + r] = nrm[r];
        }
    }
    __syncthreads();

    // ---- A7 + A8 epilogue: mean and variance per query ----------------------------
    const bool want_init = A.pos != nullptr;
    for (int q = tid; q < GG; q += nthr) {
        const int u = q / G, vv = q - u * G;
        T s4[4] = {zero<T>(), zero<T>(), zero<T>(), zero<T>()};
        int i = 0;
        for (; i + 3 < n; i += 4)
#pragma unroll
            for (int w = 0; w < 4; ++w)
                acc_fma(s4[w], al[i + w] * fa[(i + w) * G + u], fb[(i + w) * Gp + vv]);
        for (; i < n; ++i) acc_fma(s4[0], al[i] * fa[i * G + u], fb[i * Gp + vv]);
        T mu = m + ((acc_norm(s4[0]) + acc_norm(s4[1])) + (acc_norm(s4[2]) + acc_norm(s4[3])));
        if (refine) {  // m + K*^T (alpha + d), float-float sum of FP32 kernel values
            ff acc = ff_make(0.f, 0.f);
            for (int i = 0; i < n; ++i) {
                const float k = __fmul_rn(to_f(fa[i * G + u]), to_f(fb[i * Gp + vv]));
                acc_fma(acc, ff_make(k, 0.f), two_sum(to_f(al[i]), to_f(dal[i])));
            }
            mu = from_f<T>(to_f(ff_make(to_f(m), 0.f) + acc_norm(acc)));
        }
        if (tc) {
            A.mean[obase + q] = to_f(mu);
            Wtc[ntri + n * G + n * Gp + q] = mu;
            continue;
        }
        T nr = zero<T>();
        for (int g = 0; g < P.nrg; ++g) nr = nr + part[g * (G * Gp) + u * Gp + vv];
        T var = sf2 - nr;
        if (!(hi_of(var) > 0.f)) var = zero<T>();
        A.mean[obase + q] = to_f(mu);
        A.var[obase + q] = to_f(var);
        if (want_init) { mv[q] = mu; mv[GG + q] = var; }
    }
    if (tid == 0) {
        A.axis[v] = (uint8_t)axis;
        uint32_t st = A.escalation_pass ? VOX_ESCALATED : 0u;
        A.status[v] = st;
    }
    if (tc) {  // queue the voxel for k_var_tc
        __syncthreads();
        if (tid == 0) {
            const int slot = atomicAdd(&A.tc->count, 1);
            A.tc_v[slot] = v;
            A.tc_off[slot] = s_tc_off;
            A.tc_off_v[v] = s_tc_off;
        }
        __syncthreads();
        return;
    }
    // ---- A10 (fused): Gaussians of the n_s x n_s subgrids ---------------------------
    if (want_init) {
        __syncthreads();
        const int NG = A.n_s * A.n_s;
        for (int g = tid; g < NG; g += nthr) {
            const int64_t o = (int64_t)v * NG + g;
            init_one_gaussian<T>(mv, mv + GG, nodes, axis, cen, A.size, G, A.n_s, A.n_r, sf2f,
                                 A.init_mode, g / A.n_s, g % A.n_s, A.pos + 3 * o,
                                 A.scale + 3 * o, A.quat + 4 * o);
        }
    }
    __syncthreads();
}

// At most 128 registers per thread at every CTA size, so that 512 threads fit an SM; the
// variant without the contraction fits in 85, so that 768 threads do.
template <class T, bool TRI_SMEM, int NT, bool TCV>
__global__ void __launch_bounds__(NT, (TCV ? 768 : 512) / NT) k_solve(SolveArgs A)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ double red[6 * 32];
    __shared__ T nodes[kMaxG];
    __shared__ ff xtab[is_ff<T>::value ? 256 : 1];  // 2^(m/256) for the float-float exp
    __shared__ int s_v;
    const SmemPlan P = smem_plan(A.nmax, A.G, A.Gp, (int)sizeof(T), TRI_SMEM, NT, TCV);
    // query grid nodes -s/2 + (u + 1/2) s / G, formed once in FP64 and rounded to T
    if (threadIdx.x < A.G)
        nodes[threadIdx.x] = from_d<T>(-0.5 * (double)A.size +
                                       ((double)threadIdx.x + 0.5) * (double)A.size / (double)A.G);
    if (is_ff<T>::value)
        for (int i = threadIdx.x; i < 256; i += blockDim.x) {
            const double t = exp2((double)i / 256.0);
            const float h = (float)t;
            xtab[i] = ff_make(h, (float)(t - (double)h));
        }
    const int total = *A.work_count;
    const int base = A.work_base ? *A.work_base : 0;
    for (;;) {
        if (threadIdx.x == 0) {
            int i = atomicAdd(A.work_next, 1);
            s_v = i < total ? A.work[base + i] : -1;
        }
        __syncthreads();
        const int v = s_v;
        __syncthreads();
        if (v < 0) break;
        solve_voxel<T, TRI_SMEM, TCV>(A, v, smem, P, red, nodes, xtab);
    }
}

// ---- size classification into buckets (device-side, no host round trip) -------
__global__ void k_classify(SolveArgs A, const int* bucket_hi, int nb, int32_t* bcount)
{
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= (A.nvox_dev ? min(*A.nvox_dev, A.nvox) : A.nvox)) return;
    const int64_t n = A.offsets[v + 1] - A.offsets[v];
    const bool skip = A.skip && A.skip[v];
    if (skip || n < A.tau || n <= 0 || n > A.max_points) {
        const int GG = A.G * A.G;
        const float sf2 = A.sf2[v];
        for (int q = 0; q < GG; ++q) {
            A.mean[(int64_t)v * GG + q] = 0.f;
            A.var[(int64_t)v * GG + q] = sf2;
        }
        A.axis[v] = 255;
        A.status[v] = skip ? VOX_CONVERGED : (n > A.max_points ? VOX_TOO_LARGE : VOX_BELOW_TAU);
        if (A.pos) {
            const int NG = A.n_s * A.n_s;
            for (int g = 0; g < NG; ++g) {
                const int64_t o = (int64_t)v * NG + g;
                for (int k = 0; k < 3; ++k) {
                    A.pos[3 * o + k] = A.centres[3 * v + k];
                    A.scale[3 * o + k] = 0.f;
                }
                A.quat[4 * o] = 1.f; A.quat[4 * o + 1] = 0.f; A.quat[4 * o + 2] = 0.f; A.quat[4 * o + 3] = 0.f;
            }
        }
        return;
    }
    int b = nb - 1;
    for (int k = 0; k < nb; ++k)
        if (n <= bucket_hi[k]) { b = k; break; }
    atomicAdd(&bcount[b], 1);
    if (A.tc_ws != nullptr && n <= max(A.tc_nmax, A.tc_nmax_gl))
        atomicAdd(&A.tc->total, (unsigned long long)tc_need_bytes((int)n, A.G, A.Gp));
}

__global__ void k_scan(int nb, const int32_t* bcount, int32_t* bbase, int32_t* bcursor,
                       int32_t* next, int32_t* esc_count)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    int s = 0;
    for (int b = 0; b < nb; ++b) {
        bbase[b] = s;
        bcursor[b] = 0;
        next[b] = 0;
        s += bcount[b];
    }
    next[nb] = 0;  // dequeue counters of the two escalation passes
    next[nb + 1] = 0;
    esc_count[0] = 0;
    esc_count[1] = 0;
}

__global__ void k_scatter(SolveArgs A, const int* bucket_hi, int nb, const int32_t* bbase,
                          int32_t* bcursor, int32_t* work)
{
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= (A.nvox_dev ? min(*A.nvox_dev, A.nvox) : A.nvox)) return;
    const int64_t n = A.offsets[v + 1] - A.offsets[v];
    if ((A.skip && A.skip[v]) || n < A.tau || n <= 0 || n > A.max_points) return;
    int b = nb - 1;
    for (int k = 0; k < nb; ++k)
        if (n <= bucket_hi[k]) { b = k; break; }
    const int slot = atomicAdd(&bcursor[b], 1);
    work[bbase[b] + slot] = v;
}

cudaError_t launch_classify(const SolveArgs& a, const int* bucket_hi, int nb, int32_t* bcount,
                            int32_t* bbase, int32_t* bcursor, int32_t* work, int32_t* next,
                            int32_t* esc_count, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(bcount, 0, sizeof(int32_t) * nb, s);
    if (e != cudaSuccess) return e;
    if (a.tc != nullptr && (e = cudaMemsetAsync(a.tc, 0, sizeof(TcCounters), s)) != cudaSuccess)
        return e;
    if (a.nvox > 0) {
        const int blk = 256, grd = (a.nvox + blk - 1) / blk;
        k_classify<<<grd, blk, 0, s>>>(a, bucket_hi, nb, bcount);
    }
    k_scan<<<1, 32, 0, s>>>(nb, bcount, bbase, bcursor, next, esc_count);
    if (a.nvox > 0) {
        const int blk = 256, grd = (a.nvox + blk - 1) / blk;
        k_scatter<<<grd, blk, 0, s>>>(a, bucket_hi, nb, bbase, bcursor, work);
    }
    return cudaGetLastError();
}

// The dynamic shared-memory limit of every instantiation is raised once, when the
// handle plans its launches (solve_occupancy), so launches stay capturable.
// CTA sizes: 128, 256 and 512 threads; the shared-memory variants (S) also 32 and 64
// for buckets of at most that many points (one warp or two per voxel)
template <class T, bool S, bool V = false>
static cudaError_t launch_t(int nthr, const SolveArgs& a, int grid, int smem, cudaStream_t s)
{
    if (nthr == 512) k_solve<T, S, 512, V><<<grid, 512, smem, s>>>(a);
    else if (nthr == 128) k_solve<T, S, 128, V><<<grid, 128, smem, s>>>(a);
    else if (S && nthr == 64) k_solve<T, S, S ? 64 : 256, V><<<grid, 64, smem, s>>>(a);
    else if (S && nthr == 32) k_solve<T, S, S ? 32 : 256, V><<<grid, 32, smem, s>>>(a);
    else k_solve<T, S, 256, V><<<grid, 256, smem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_solve(int prec, bool tri_in_smem, int nthr, const SolveArgs& a, int grid,
                         int smem, cudaStream_t s, bool tcv)
{
    if (prec == PREC_F32) return tri_in_smem ? launch_t<float, true>(nthr, a, grid, smem, s) : launch_t<float, false>(nthr, a, grid, smem, s);
    if (prec == PREC_F64) return tri_in_smem ? launch_t<double, true>(nthr, a, grid, smem, s) : launch_t<double, false>(nthr, a, grid, smem, s);
    if (tcv && tri_in_smem) return launch_t<ff, true, true>(nthr, a, grid, smem, s);
    return tri_in_smem ? launch_t<ff, true>(nthr, a, grid, smem, s) : launch_t<ff, false>(nthr, a, grid, smem, s);
}

static int tsize_of(int prec) { return prec == PREC_F32 ? 4 : 8; }

cudaError_t solve_max_smem_n(int prec, int G, int Gp, int* nmax_out, bool tcv)
{
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    const int static_bytes = 6 * 32 * 8 + 32 * 8 + 64 + 256 * 8;
    int best = 0;
    for (int n = 8; n <= 1024; n += 8) {
        SmemPlan p = smem_plan(n, G, Gp, tsize_of(prec), true, solve_threads(n, true), tcv);
        if (p.total + static_bytes <= optin) best = n;
    }
    *nmax_out = best;
    return cudaSuccess;
}

template <class T, bool S, bool V = false>
static const void* kfun(int nthr)
{
    if (S && nthr == 64) return (const void*)k_solve<T, S, S ? 64 : 256, V>;
    if (S && nthr == 32) return (const void*)k_solve<T, S, S ? 32 : 256, V>;
    return nthr == 512 ? (const void*)k_solve<T, S, 512, V>
                       : (nthr == 128 ? (const void*)k_solve<T, S, 128, V> : (const void*)k_solve<T, S, 256, V>);
}

cudaError_t solve_occupancy(int prec, bool tri_in_smem, int nthr, int smem, int* blocks_per_sm, bool tcv)
{
    const void* f;
    if (prec == PREC_F32) f = tri_in_smem ? kfun<float, true>(nthr) : kfun<float, false>(nthr);
    else if (prec == PREC_F64) f = tri_in_smem ? kfun<double, true>(nthr) : kfun<double, false>(nthr);
    else if (tcv && tri_in_smem) f = kfun<ff, true, true>(nthr);
    else f = tri_in_smem ? kfun<ff, true>(nthr) : kfun<ff, false>(nthr);
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    cudaFuncAttributes fa;
    e = cudaFuncGetAttributes(&fa, f);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             optin - (int)fa.sharedSizeBytes);
    if (e != cudaSuccess) return e;
    if (smem > optin - (int)fa.sharedSizeBytes) { *blocks_per_sm = 0; return cudaSuccess; }
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, f, nthr, smem);
}

// ---- standalone Gaussian initialisation from FP32 predictions ---------------------
__global__ void k_init(const float* mean, const float* var, const uint8_t* axis,
                       const float* centres, const float* sf2, const uint32_t* status,
                       int32_t nvox, float size, int G, int n_s, int n_r, int init_mode,
                       float* pos, float* scale, float* quat)
{
    extern __shared__ ff mvs[];  // per warp: 2 G^2 values
    __shared__ ff nodes[kMaxG];
    if (threadIdx.x < G)
        nodes[threadIdx.x] = from_d<ff>(-0.5 * (double)size +
                                        ((double)threadIdx.x + 0.5) * (double)size / (double)G);
    __syncthreads();
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nw = blockDim.x >> 5;
    const int v = blockIdx.x * nw + wid;
    if (v >= nvox) return;
    const int GG = G * G, NG = n_s * n_s;
    ff* mv = mvs + (size_t)wid * 2 * GG;
    for (int q = lane; q < GG; q += 32) {
        mv[q] = from_f<ff>(mean[(int64_t)v * GG + q]);
        mv[GG + q] = from_f<ff>(var[(int64_t)v * GG + q]);
    }
    __syncwarp();
    const bool skip = (status && (status[v] & (VOX_BELOW_TAU | VOX_NOT_SPD | VOX_TOO_LARGE))) ||
                      axis[v] > 2;
    for (int g = lane; g < NG; g += 32) {
        const int64_t o = (int64_t)v * NG + g;
        if (skip) {
            for (int k = 0; k < 3; ++k) { pos[3 * o + k] = centres[3 * v + k]; scale[3 * o + k] = 0.f; }
            quat[4 * o] = 1.f; quat[4 * o + 1] = 0.f; quat[4 * o + 2] = 0.f; quat[4 * o + 3] = 0.f;
            continue;
        }
        init_one_gaussian<ff>(mv, mv + GG, nodes, axis[v], centres + 3 * v, size, G, n_s, n_r,
                              sf2[v], init_mode, g / n_s, g % n_s, pos + 3 * o, scale + 3 * o,
                              quat + 4 * o);
    }
}

cudaError_t launch_init(const float* mean, const float* var, const uint8_t* axis,
                        const float* centres, const float* sf2, const uint32_t* status,
                        int32_t nvox, float size, int G, int n_s, int n_r, int init_mode,
                        float* pos, float* scale, float* quat, cudaStream_t s)
{
    if (nvox <= 0) return cudaSuccess;
    // one warp per voxel, its G^2 predictions staged as float-float; stay under 48 KB
    const int per_warp = 2 * G * G * (int)sizeof(ff);
    const int warps = per_warp * 4 <= 48 * 1024 ? 4 : (per_warp * 2 <= 48 * 1024 ? 2 : 1);
    const int smem = warps * per_warp;
    const int grid = (nvox + warps - 1) / warps;
    k_init<<<grid, warps * 32, smem, s>>>(mean, var, axis, centres, sf2, status, nvox, size, G,
                                          n_s, n_r, init_mode, pos, scale, quat);
    return cudaGetLastError();
}

}  // namespace gpv
