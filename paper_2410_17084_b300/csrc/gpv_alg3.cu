// gpv_alg3.cu -- the paper's own formulation of the batched solve (supplementary Alg. 3:
// add noise, LU with partial pivoting, explicit inverse, then three products giving mu*
// and the FULL posterior covariance Sigma* of the query nodes), in FP32 as the paper's
// single-precision library routines, for a CSR batch of voxels.
//
// Kernel A (k_alg3_factor, one CTA per voxel, FP32 on the CUDA cores, all in shared
// memory): value axis and local frame as the main solve (Sec. 3.1), ky = K + sigma^2 I
// (full n x n), in-place LU with partial pivoting, in-place inverse from the LU factors
// (inverse of U, then the solve with L, then the column interchanges, which are folded
// into an index map), k_k* = K*^T ky^-1 (G^2 x n) written to a workspace as a TF32
// split pair (big + small), and mu* = m + k_k* (f - m).
// Kernel B (k_alg3_cov, tcgen05 tensor cores): Sigma* = K** - k_k* K* for one 128-row x
// up-to-256-column tile of one voxel.  Operand chunks of 32 along n are staged in shared
// memory (K-major, unswizzled core matrices), three TF32 MMAs per K step (big*big +
// big*small + small*big, FP32 accumulation in tensor memory) keep FP32-level accuracy,
// the accumulator is read back with tcgen05.ld and K** is added in the epilogue.  The
// kernel is bound by the Sigma* stores (G^4 floats per voxel).
#include <cuda_runtime.h>
#include <stdint.h>

#include "gpv_alg3.h"
#include "gpv_common.cuh"
#include "gpv_umma.cuh"

namespace gpv {

namespace {

constexpr int kA3Threads = 256;
constexpr int kKC = 32;          // K chunk of the tensor-core kernel (elements)
constexpr uint32_t kWaitPolls = 1u << 26;

// shared-memory plan of kernel A (bytes) for voxels of up to nmax points
struct A3Plan {
    int off_pts, off_x1, off_x2, off_f, off_fa, off_fb, off_tmp, off_piv, off_src, off_A, total;
};

// big: ky and the K* factors live in global memory (voxels beyond shared memory)
__host__ __device__ inline A3Plan a3_plan(int nmax, int G, bool big = false)
{
    A3Plan p;
    int o = 0;
    auto take = [&](int bytes) { const int at = o; o = (o + bytes + 15) & ~15; return at; };
    p.off_pts = take(12 * nmax);
    p.off_x1 = take(4 * nmax);
    p.off_x2 = take(4 * nmax);
    p.off_f = take(4 * nmax);
    p.off_fa = take(big ? 0 : 4 * nmax * G);
    p.off_fb = take(big ? 0 : 4 * nmax * G);
    p.off_tmp = take(4 * nmax);
    p.off_piv = take(4 * nmax);
    p.off_src = take(4 * nmax);
    p.off_A = take(big ? 0 : 4 * nmax * nmax);
    p.total = o;
    return p;
}

__device__ __forceinline__ float node_pos(int i, int G, float s)
{
    return (float)(-0.5 * (double)s + ((double)i + 0.5) * (double)s / (double)G);
}

// One voxel of kernel A.  BIG: ky (row-major, stride n) and the K* factors in global
// memory (this CTA's slice of ws_A, the slot's workspace factors), the rest in shared.
template <bool BIG>
__device__ void alg3_factor_one(const Alg3Args& a, int slot, unsigned char* sm, float* red,
                                int& s_axis, int& s_fail, int& s_p, float* s_pv, int* s_pi)
{
    const int v = a.v0 + slot;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
    const int G = a.G, Q = G * G;
    const int64_t beg = a.offsets[v];
    const int n = (int)(a.offsets[v + 1] - beg);
    const bool unsolved = n < a.tau || n > a.nmax;
    // size classes: each launch takes its own range (unsolved voxels go to the first)
    if (unsolved ? a.nlo != 0 : (n <= a.nlo || n > a.nhi)) return;
    if (unsolved) {  // not processed: the prior (kernel B writes K**)
        for (int q = tid; q < Q; q += blockDim.x) a.mean[(int64_t)v * Q + q] = 0.f;
        if (tid == 0) {
            a.axis[v] = 255;
            const uint32_t st = n > a.nmax ? VOX_TOO_LARGE : VOX_BELOW_TAU;
            a.status[v] = st;
            a.ws_status[slot] = st;
            a.ws_n[slot] = n;
        }
        return;
    }
    const A3Plan P = a3_plan(a.nhi, G, BIG);
    const int Kp = a.kp;
    float* pts = reinterpret_cast<float*>(sm + P.off_pts);
    float* x1 = reinterpret_cast<float*>(sm + P.off_x1);
    float* x2 = reinterpret_cast<float*>(sm + P.off_x2);
    float* fv = reinterpret_cast<float*>(sm + P.off_f);
    float* FA = a.ws_fa + (int64_t)slot * Kp * G;  // the K* factors for kernel B
    float* FB = a.ws_fb + (int64_t)slot * Kp * G;
    float* fa = BIG ? FA : reinterpret_cast<float*>(sm + P.off_fa);
    float* fb = BIG ? FB : reinterpret_cast<float*>(sm + P.off_fb);
    float* tmp = reinterpret_cast<float*>(sm + P.off_tmp);
    int* piv = reinterpret_cast<int*>(sm + P.off_piv);
    int* src = reinterpret_cast<int*>(sm + P.off_src);
    float* A = BIG ? a.ws_A + (int64_t)blockIdx.x * Kp * Kp   // row-major, stride n
                   : reinterpret_cast<float*>(sm + P.off_A);

    for (int t = tid; t < 3 * n; t += blockDim.x) pts[t] = __ldg(a.xyz + 3 * beg + t);
    __syncthreads();
    // value axis (Sec. 3.1), as the main solve
    const float cx = a.centres[3 * v], cy = a.centres[3 * v + 1], cz = a.centres[3 * v + 2];
    {
        float s3[3] = {0.f, 0.f, 0.f};
        for (int i = tid; i < n; i += blockDim.x) {
            s3[0] += pts[3 * i] - cx; s3[1] += pts[3 * i + 1] - cy; s3[2] += pts[3 * i + 2] - cz;
        }
        block_sum<float, 3>(s3, red);
        const float inv_n = 1.f / (float)n;
        const float m0 = s3[0] * inv_n, m1 = s3[1] * inv_n, m2 = s3[2] * inv_n;
        float c6[6] = {0, 0, 0, 0, 0, 0};
        for (int i = tid; i < n; i += blockDim.x) {
            const float d0 = (pts[3 * i] - cx) - m0, d1 = (pts[3 * i + 1] - cy) - m1,
                        d2 = (pts[3 * i + 2] - cz) - m2;
            c6[0] += d0 * d0; c6[1] += d0 * d1; c6[2] += d0 * d2;
            c6[3] += d1 * d1; c6[4] += d1 * d2; c6[5] += d2 * d2;
        }
        block_sum<float, 6>(c6, red);
        if (tid == 0) { s_axis = value_axis_from_cov(c6); s_fail = 0; }
        __syncthreads();
    }
    const int axis = s_axis;
    const int p1 = axis == 2 ? 0 : axis + 1;
    const int p2 = axis == 0 ? 2 : (axis == 1 ? 0 : 1);
    const float cen[3] = {cx, cy, cz};
    float ms[1] = {0.f};
    for (int i = tid; i < n; i += blockDim.x) {
        x1[i] = pts[3 * i + p1] - cen[p1];
        x2[i] = pts[3 * i + p2] - cen[p2];
        fv[i] = pts[3 * i + axis] - cen[axis];
        ms[0] += fv[i];
    }
    block_sum<float, 1>(ms, red);
    const float m = a.mean_mode == 1 ? ms[0] / (float)n : 0.f;
    const float lam = a.lam[v], sf2 = a.sf2[v], sn2 = a.sn2[v];
    // separable cross-covariance factors: k(x_j, (u, w)) = fa[j][u] fb[j][w]
    for (int t = tid; t < n * G; t += blockDim.x) {
        const int j = t / G, u = t - j * G;
        const float nd = node_pos(u, G, a.size);
        const float d1 = x1[j] - nd, d2 = x2[j] - nd;
        fa[t] = sf2 * expf(-lam * d1 * d1);
        fb[t] = expf(-lam * d2 * d2);
    }
    // ky = K + sigma^2 I (Alg. 3, "add noise")
    for (int t = tid; t < n * n; t += blockDim.x) {
        const int i = t / n, j = t - i * n;
        const float d1 = x1[i] - x1[j], d2 = x2[i] - x2[j];
        A[t] = sf2 * expf(-lam * (d1 * d1 + d2 * d2)) + (i == j ? sn2 : 0.f);
    }
    __syncthreads();

    // ---- LU with partial pivoting, in place (row interchanges recorded in piv) -------
    for (int k = 0; k < n; ++k) {
        float best = -1.f;
        int bi = k;
        for (int i = k + tid; i < n; i += blockDim.x) {
            const float x = fabsf(A[i * n + k]);
            if (x > best) { best = x; bi = i; }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float ob = __shfl_xor_sync(0xffffffffu, best, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
        }
        if (lane == 0) { s_pv[wid] = best; s_pi[wid] = bi; }
        __syncthreads();
        if (tid == 0) {
            float b = s_pv[0];
            int ix = s_pi[0];
            for (int w = 1; w < nw; ++w)
                if (s_pv[w] > b || (s_pv[w] == b && s_pi[w] < ix)) { b = s_pv[w]; ix = s_pi[w]; }
            s_p = ix;
            piv[k] = ix;
            if (!(b > 0.f)) s_fail = 1;
        }
        __syncthreads();
        if (s_fail) break;
        const int p = s_p;
        if (p != k)
            for (int j = tid; j < n; j += blockDim.x) {
                const float t0 = A[k * n + j];
                A[k * n + j] = A[p * n + j];
                A[p * n + j] = t0;
            }
        __syncthreads();
        const float inv = 1.f / A[k * n + k];
        for (int i = k + 1 + tid; i < n; i += blockDim.x) A[i * n + k] *= inv;
        __syncthreads();
        const int r = n - k - 1;
        for (int t = tid; t < r * r; t += blockDim.x) {
            const int i = k + 1 + t / r, j = k + 1 + t % r;
            A[i * n + j] = fmaf(-A[i * n + k], A[k * n + j], A[i * n + j]);
        }
        __syncthreads();
    }
    if (s_fail) {  // singular in FP32: the prior
        for (int q = tid; q < Q; q += blockDim.x) a.mean[(int64_t)v * Q + q] = 0.f;
        if (tid == 0) {
            a.axis[v] = (uint8_t)axis;
            a.status[v] = VOX_NOT_SPD;
            a.ws_status[slot] = VOX_NOT_SPD;
            a.ws_n[slot] = n;
        }
        return;
    }
    // ---- inverse from the LU factors ----------------------------------------------
    // (a) U^-1 in place, column by column: X(i, j) = -X(j, j) sum_{k=i}^{j-1} X(i, k) U(k, j)
    for (int j = 0; j < n; ++j) {
        const float ujj = A[j * n + j];
        for (int i = tid; i < j; i += blockDim.x) {
            float s = 0.f;
            for (int k = i; k < j; ++k) s = fmaf(A[i * n + k], A[k * n + j], s);
            tmp[i] = s;
        }
        __syncthreads();
        const float xjj = 1.f / ujj;
        for (int i = tid; i < j; i += blockDim.x) A[i * n + j] = -xjj * tmp[i];
        if (tid == 0) A[j * n + j] = xjj;
        __syncthreads();
    }
    // (b) solve W L = U^-1 from the last column back: W(:, j) = X(:, j) - W(:, j+1:) L(j+1:, j)
    for (int j = n - 2; j >= 0; --j) {
        for (int i = j + 1 + tid; i < n; i += blockDim.x) tmp[i] = A[i * n + j];
        __syncthreads();
        for (int i = tid; i < n; i += blockDim.x) {
            float s = i > j ? 0.f : A[i * n + j];
            for (int k = j + 1; k < n; ++k) s = fmaf(-A[i * n + k], tmp[k], s);
            A[i * n + j] = s;
        }
        __syncthreads();
    }
    // (c) the column interchanges, applied in reverse order, as an index map:
    //     ky^-1(:, c) = W(:, src[c])
    if (tid == 0) {
        for (int c = 0; c < n; ++c) src[c] = c;
        for (int j = n - 2; j >= 0; --j) {
            const int jp = piv[j];
            if (jp != j) { const int t0 = src[j]; src[j] = src[jp]; src[jp] = t0; }
        }
    }
    __syncthreads();

    // ---- k_k* = K*^T ky^-1 (G^2 x n), written as a TF32 split pair ------------------
    float* Pb = a.ws_pb + (int64_t)slot * Q * Kp;
    float* Ps = a.ws_ps + (int64_t)slot * Q * Kp;
    {  // 4 queries x 4 columns per thread, 16 accumulators
        const int nqt = (Q + 3) >> 2, nct = (n + 3) >> 2;
        for (int t = tid; t < nqt * nct; t += blockDim.x) {
            const int qt = t / nct, ct = t - qt * nct;
            int uq[4], wq[4], sc[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int q = min(4 * qt + i, Q - 1), c = min(4 * ct + i, n - 1);
                uq[i] = q / G;
                wq[i] = q - uq[i] * G;
                sc[i] = src[c];
            }
            float acc[4][4] = {};
            for (int j = 0; j < n; ++j) {
                float kq[4], x[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    kq[i] = fa[j * G + uq[i]] * fb[j * G + wq[i]];
                    x[i] = A[j * n + sc[i]];
                }
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int k = 0; k < 4; ++k) acc[i][k] = fmaf(kq[i], x[k], acc[i][k]);
            }
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const int q = 4 * qt + i, c = 4 * ct + k;
                    if (q < Q && c < n) {
                        float bg, sl;
                        umma::tf32_split(acc[i][k], bg, sl);
                        Pb[(int64_t)q * Kp + c] = bg;
                        Ps[(int64_t)q * Kp + c] = sl;
                    }
                }
        }
    }
    // factors of K* for kernel B (already in place for BIG)
    if (!BIG)
        for (int t = tid; t < n * G; t += blockDim.x) { FA[t] = fa[t]; FB[t] = fb[t]; }
    __syncthreads();
    // ---- mu* = m + k_k* (f - m) ---------------------------------------------------------
    for (int q = tid; q < Q; q += blockDim.x) {
        float s = 0.f;
        for (int c = 0; c < n; ++c)
            s = fmaf(Pb[(int64_t)q * Kp + c] + Ps[(int64_t)q * Kp + c], fv[c] - m, s);
        a.mean[(int64_t)v * Q + q] = m + s;
    }
    if (tid == 0) {
        a.axis[v] = (uint8_t)axis;
        a.status[v] = VOX_OK;
        a.ws_status[slot] = VOX_OK;
        a.ws_n[slot] = n;
    }
}

__global__ void __launch_bounds__(kA3Threads) k_alg3_factor(Alg3Args a)
{
    extern __shared__ __align__(16) unsigned char sm[];
    __shared__ float red[6 * 32];
    __shared__ int s_axis, s_fail, s_p;
    __shared__ float s_pv[32];
    __shared__ int s_pi[32];
    alg3_factor_one<false>(a, blockIdx.x, sm, red, s_axis, s_fail, s_p, s_pv, s_pi);
}

// voxels beyond shared memory: persistent CTAs over the chunk's slots, ky in global memory
__global__ void __launch_bounds__(kA3Threads) k_alg3_factor_big(Alg3Args a)
{
    extern __shared__ __align__(16) unsigned char sm[];
    __shared__ float red[6 * 32];
    __shared__ int s_axis, s_fail, s_p;
    __shared__ float s_pv[32];
    __shared__ int s_pi[32];
    for (int slot = blockIdx.x; slot < a.nchunk; slot += gridDim.x) {
        alg3_factor_one<true>(a, slot, sm, red, s_axis, s_fail, s_p, s_pv, s_pi);
        __syncthreads();
    }
}

// Sigma* = K** - k_k* K* for rows q0 .. q0+127 and columns c0 .. c0+NN-1 of one voxel.
__global__ void __launch_bounds__(128) k_alg3_cov(Alg3Args a, int NN, uint32_t tmem_cols)
{
    extern __shared__ __align__(16) unsigned char smb[];  // unswizzled operands: 16-byte alignment
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tslot;
    __shared__ float e1[32 * 32];
    const int slot = blockIdx.z, v = a.v0 + slot;
    const int q0 = blockIdx.x * 128, c0 = blockIdx.y * 256;
    const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
    const int G = a.G, Q = G * G, Kp = a.kp;
    const float sf2 = a.sf2[v], lam = a.lam[v];
    for (int t = tid; t < G * G; t += 128) {
        const int i = t / G, j = t - i * G;
        const float d = node_pos(i, G, a.size) - node_pos(j, G, a.size);
        e1[t] = expf(-lam * d * d);
    }
    __syncthreads();
    float* cov = a.cov + (int64_t)v * Q * Q;
    const uint32_t st = a.ws_status[slot];
    const int row = q0 + 32 * w + lane;
    if (st != VOX_OK) {  // prior covariance K**
        if (row < Q) {
            const int u = row / G, x = row - u * G;
            for (int c = c0; c < min(c0 + NN, Q); ++c) {
                const int u2 = c / G, x2 = c - u2 * G;
                cov[(int64_t)row * Q + c] = sf2 * e1[u * G + u2] * e1[x * G + x2];
            }
        }
        return;
    }
    const int n = a.ws_n[slot];
    float* a_big = reinterpret_cast<float*>(smb);
    float* a_small = a_big + 128 * kKC;
    float* b_big = a_small + 128 * kKC;
    float* b_small = b_big + NN * kKC;
    if (w == 0) umma::tmem_alloc(&tslot, tmem_cols);
    if (tid == 0) {
        umma::mbar_init(&mbar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    umma::fence_before_sync();
    __syncthreads();
    umma::fence_after_sync();
    const uint32_t tmem = tslot;
    const uint32_t idesc = umma::idesc_tf32(128, NN);
    const float* Pb = a.ws_pb + (int64_t)slot * Q * Kp;
    const float* Ps = a.ws_ps + (int64_t)slot * Q * Kp;
    const float* FA = a.ws_fa + (int64_t)slot * Kp * G;
    const float* FB = a.ws_fb + (int64_t)slot * Kp * G;
    uint32_t phase = 0;
    bool ok = true;
    for (int k0 = 0; k0 < n && ok; k0 += kKC) {
        for (int t = tid; t < 128 * kKC; t += 128) {  // A = k_k* rows q0.., already split
            const int r = t / kKC, k = t - r * kKC;
            const int q = q0 + r, c = k0 + k;
            const bool in = q < Q && c < n;
            const int o = umma::kmajor_offset(r, k, kKC) >> 2;
            a_big[o] = in ? Pb[(int64_t)q * Kp + c] : 0.f;
            a_small[o] = in ? Ps[(int64_t)q * Kp + c] : 0.f;
        }
        for (int t = tid; t < NN * kKC; t += 128) {  // B = K*^T rows c0.., split here
            const int r = t / kKC, k = t - r * kKC;
            const int q = c0 + r, c = k0 + k;
            float x = 0.f;
            if (q < Q && c < n) {
                const int u = q / G, x2 = q - u * G;
                x = FA[c * G + u] * FB[c * G + x2];
            }
            float bg, sl;
            umma::tf32_split(x, bg, sl);
            const int o = umma::kmajor_offset(r, k, kKC) >> 2;
            b_big[o] = bg;
            b_small[o] = sl;
        }
        umma::fence_proxy_async_smem();
        __syncthreads();
        if (tid == 0) {
            umma::fence_after_sync();
            const uint32_t ab = umma::smem_addr(a_big), as = umma::smem_addr(a_small);
            const uint32_t bb = umma::smem_addr(b_big), bs = umma::smem_addr(b_small);
            const int sbo = (kKC / 4) * umma::kLBO;
#pragma unroll
            for (int s = 0; s < kKC / 8; ++s) {
                const uint32_t off = s * 2 * umma::kLBO;
                const uint64_t dab = umma::make_desc(ab + off, umma::kLBO, sbo);
                const uint64_t das = umma::make_desc(as + off, umma::kLBO, sbo);
                const uint64_t dbb = umma::make_desc(bb + off, umma::kLBO, sbo);
                const uint64_t dbs = umma::make_desc(bs + off, umma::kLBO, sbo);
                umma::mma_tf32(tmem, dab, dbb, idesc, k0 > 0 || s > 0);
                umma::mma_tf32(tmem, dab, dbs, idesc, true);
                umma::mma_tf32(tmem, das, dbb, idesc, true);
            }
            umma::mma_commit(&mbar);
        }
        const bool mine = umma::mbar_wait(&mbar, phase, kWaitPolls);
        phase ^= 1u;
        ok = __syncthreads_and(mine) != 0;  // the same decision in every thread
    }
    umma::fence_after_sync();
    if (!ok) {
        if (tid == 0) atomicOr(a.status + v, VOX_FAILED);
    } else {
        const int u = row / G, x = row - u * G;
        float* out = cov + (int64_t)row * Q;
        for (int cc = 0; cc < NN; cc += 16) {
            float d[16];  // every lane of the warp takes part in the load
            umma::tmem_ld16(tmem + ((uint32_t)(32 * w) << 16) + (uint32_t)cc, d);
            if (row < Q)
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    const int c = c0 + cc + i;
                    if (c < Q) {
                        const int u2 = c / G, x2 = c - u2 * G;
                        out[c] = sf2 * e1[u * G + u2] * e1[x * G + x2] - d[i];
                    }
                }
        }
    }
    umma::fence_before_sync();
    __syncthreads();
    if (w == 0) umma::tmem_free(tmem, tmem_cols);
}

}  // namespace

int alg3_max_n(int G)
{
    int dev = 0, optin = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
        return 0;
    const int static_bytes = 6 * 32 * 4 + 32 * 8 + 64;
    int best = 0;
    for (int n = 8; n <= 1024; n += 8)
        if (a3_plan(n, G).total + static_bytes <= optin) best = n;
    return best;
}

int alg3_big_ctas()
{
    int dev = 0, sms = 148;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms;
}

cudaError_t alg3_launch_chunk(const Alg3Args& a0, int nchunk, cudaStream_t s, int* nlaunch)
{
    *nlaunch = 0;
    // kernel A in three size classes, each launch with the shared memory of its largest n
    const int nsm = a0.nsm < a0.nmax ? a0.nsm : a0.nmax;  // largest n of the shared-memory classes
    const int cls[3] = {64, 128, nsm};
    cudaError_t e = cudaFuncSetAttribute(k_alg3_factor, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         a3_plan(nsm, a0.G).total);
    if (e != cudaSuccess) return e;
    int lo = 0;
    for (int c = 0; c < 3; ++c) {
        const int hi = c < 2 ? (cls[c] < nsm ? cls[c] : nsm) : nsm;
        if (hi <= lo && c > 0) continue;
        Alg3Args a = a0;
        a.nlo = lo;
        a.nhi = hi;
        const int smemA = a3_plan(hi, a.G).total;
        k_alg3_factor<<<nchunk, kA3Threads, smemA, s>>>(a);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        ++*nlaunch;
        lo = hi;
    }
    if (a0.nmax > a0.nsm) {  // voxels beyond shared memory
        Alg3Args a = a0;
        a.nlo = a0.nsm;
        a.nhi = a0.nmax;
        a.nchunk = nchunk;
        const int smemA = a3_plan(a0.nmax, a0.G, true).total;
        e = cudaFuncSetAttribute(k_alg3_factor_big, cudaFuncAttributeMaxDynamicSharedMemorySize, smemA);
        if (e != cudaSuccess) return e;
        const int grid = nchunk < alg3_big_ctas() ? nchunk : alg3_big_ctas();
        k_alg3_factor_big<<<grid, kA3Threads, smemA, s>>>(a);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        ++*nlaunch;
    }
    const Alg3Args& a = a0;
    const int Q = a.G * a.G;
    const int NN = Q >= 256 ? 256 : (Q + 15) / 16 * 16;  // columns per tile (multiple of 16)
    uint32_t cols = 32;
    while ((int)cols < NN) cols <<= 1;
    // at most 512 / cols CTAs per SM, so that tensor-memory allocations never wait
    int smemB = (2 * 128 + 2 * NN) * kKC * 4;
    const int per_sm = 233472;
    const int max_ctas = 512 / (int)cols;
    if (smemB < per_sm / (max_ctas + 1) + 16) smemB = per_sm / (max_ctas + 1) + 16;
    e = cudaFuncSetAttribute(k_alg3_cov, cudaFuncAttributeMaxDynamicSharedMemorySize, smemB);
    if (e != cudaSuccess) return e;
    dim3 grid((Q + 127) / 128, (Q + 255) / 256, nchunk);
    k_alg3_cov<<<grid, 128, smemB, s>>>(a, NN, cols);
    ++*nlaunch;
    return cudaGetLastError();
}

}  // namespace gpv
