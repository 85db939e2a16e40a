// gpv_alg3.cu -- the paper's own formulation of the batched solve (supplementary Alg. 3:
// add noise, LU with partial pivoting, explicit inverse, then three products giving mu*
// and the FULL posterior covariance Sigma* of the query nodes), in FP32 as the paper's
// single-precision library routines, for a CSR batch of voxels.
//
// Kernel A (k_alg3_factor, one CTA per voxel, FP32 on the CUDA cores, all in shared
// memory): value axis and local frame as the main solve (Sec. 3.1), ky = K + sigma^2 I
// (full n x n), in-place LU with partial pivoting, in-place inverse from the LU factors
// (inverse of U, then the solve with L, then the column interchanges, which are folded
// into an index map), k_k* = K*^T ky^-1 (G^2 x n) written to a workspace as a TF32 split
// pair in the tiles of the tensor-core operand, and mu* = m + k_k* (f - m).
// Kernel B (k_alg3_cov, tcgen05 tensor cores): Sigma* = K** - k_k* K* for one 128-row x
// up-to-128-column tile of one voxel.  k_k* arrives in chunks of 16 points by bulk copies
// (kernel A writes it in the operand's tile layout) into a three-stage ring, K*^T is
// formed from its separable factors, three TF32 MMAs per K step (big*big + big*small +
// small*big, FP32 accumulation in tensor memory) keep FP32-level accuracy, the
// accumulator is read back with tcgen05.ld and K** is added in the epilogue.  The kernel
// is bound by the Sigma* stores (G^4 floats per voxel).
#include <cuda_runtime.h>
#include <stdint.h>

#include "gpv_alg3.h"
#include "gpv_common.cuh"
#include "gpv_umma.cuh"

namespace gpv {

namespace {

constexpr int kA3Threads = 256;
constexpr int kKC = 16;          // K chunk of the tensor-core kernel (points)
constexpr int kRows = 128;       // rows of Sigma* per tile (tensor-memory lanes)
constexpr int kTfRow = 20;       // floats per factor row of a chunk: 16 points + 4 (bank spread)
constexpr int kCovStages = 3;    // operand stages of the tensor-core kernel
constexpr uint64_t kWaitNs = 2000000000ull;  // give up on an mbarrier phase after 2 s

// Index (floats) of the TF32 big part of k_k*(q, c) in one voxel's workspace (the small
// part follows at + kRows * kKC): per 128-row block and 16-column chunk a 16 KB tile,
// big part then small part, each in the K-major core-matrix layout of the tensor-core
// operand (8 rows x 4 columns per 128-byte group; groups of 4 columns of the same 8 rows
// adjacent, then the next 8 rows), so that one chunk is one bulk copy.
__host__ __device__ inline int64_t pk_index(int q, int c, int kp)
{
    const int r = q & (kRows - 1), k = c & (kKC - 1);
    return ((int64_t)(q >> 7) * (kp / kKC) + c / kKC) * (2 * kRows * kKC) + (r >> 3) * 128 +
           (k >> 2) * 32 + (r & 7) * 4 + (k & 3);
}

// shared-memory bytes of one operand stage of the tensor-core kernel: A big, A small (as
// copied), B big, B small
__host__ __device__ inline int cov_stage_bytes(int nn) { return 2 * kRows * kKC * 4 + 2 * nn * kKC * 4; }

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
                                int& s_axis, float* s_pv, int* s_pi)
{
    const int v = a.vidx[a.s0 + slot];
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
    float* FA = a.ws_fa + (int64_t)slot * Kp * G;  // working K* factors of the BIG class
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
        if (tid == 0) s_axis = value_axis_from_cov(c6);
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
    // ky = K + sigma^2 I (Alg. 3, "add noise"): a warp per row, lanes along it
    for (int i = wid; i < n; i += nw)
        for (int j = lane; j < n; j += 32) {
            const float d1 = x1[i] - x1[j], d2 = x2[i] - x2[j];
            A[i * n + j] = sf2 * expf(-lam * (d1 * d1 + d2 * d2)) + (i == j ? sn2 : 0.f);
        }
    __syncthreads();

    // ---- LU with partial pivoting, in place (row interchanges recorded in piv) -------
    bool sing = false;
    // per column k: the pivot (largest |A(i, k)|, i >= k; ties to the lowest row) by a
    // block-wide argmax, the row interchange, then the multipliers l(i) = A(i, k) / A(k, k)
    // and the rank-1 update of the trailing rows, a warp per row and lanes along it
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
        float b = s_pv[0];  // every thread reduces the warps' candidates the same way
        int p = s_pi[0];
        for (int w2 = 1; w2 < nw; ++w2)
            if (s_pv[w2] > b || (s_pv[w2] == b && s_pi[w2] < p)) { b = s_pv[w2]; p = s_pi[w2]; }
        if (!(b > 0.f)) { sing = true; break; }  // singular in FP32 (the same in every thread)
        if (tid == 0) piv[k] = p;
        if (p != k)
            for (int j = tid; j < n; j += blockDim.x) {
                const float t0 = A[k * n + j];
                A[k * n + j] = A[p * n + j];
                A[p * n + j] = t0;
            }
        __syncthreads();
        const float inv = 1.f / A[k * n + k];
        for (int i = k + 1 + wid; i < n; i += nw) {
            const float l = A[i * n + k] * inv;
            for (int j = k + 1 + lane; j < n; j += 32) A[i * n + j] = fmaf(-l, A[k * n + j], A[i * n + j]);
            __syncwarp();
            if (lane == 0) A[i * n + k] = l;
        }
        __syncthreads();
    }
    if (sing) {  // singular in FP32: the prior
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

    // ---- k_k* = K*^T ky^-1 (G^2 x n), FP32, into the tensor-core operand tiles ----------
    float* Pk = a.ws_pk + (int64_t)slot * 2 * a.qp * Kp;
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
            // columns 4ct .. 4ct+3 of a row are one 16-byte group of the tile layout
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int q = 4 * qt + i, c = 4 * ct;
                if (q < Q) {
                    float4 bg, sl;
                    umma::tf32_split(acc[i][0], bg.x, sl.x);
                    umma::tf32_split(c + 1 < n ? acc[i][1] : 0.f, bg.y, sl.y);
                    umma::tf32_split(c + 2 < n ? acc[i][2] : 0.f, bg.z, sl.z);
                    umma::tf32_split(c + 3 < n ? acc[i][3] : 0.f, bg.w, sl.w);
                    float* at = Pk + pk_index(q, c, Kp);
                    *reinterpret_cast<float4*>(at) = bg;
                    *reinterpret_cast<float4*>(at + kRows * kKC) = sl;
                }
            }
        }
        // zeros up to the end of the last 16-column tile (the tensor cores read them)
        const int c4 = 4 * nct, nz = ((n + kKC - 1) / kKC) * kKC - c4;
        if (nz > 0)
            for (int t = tid; t < Q * nz; t += blockDim.x) {
                const int q = t / nz, c = c4 + (t - q * nz);
                Pk[pk_index(q, c, Kp)] = 0.f;
                Pk[pk_index(q, c, Kp) + kRows * kKC] = 0.f;
            }
    }
    // the K* factors for the covariance kernel, per chunk of 16 points: 2G rows (fa, then
    // fb, over the nodes) of the 16 points' values, each row padded to kTfRow floats
    float* TF = a.ws_tf + (int64_t)slot * (Kp / kKC) * 2 * G * kTfRow;
    for (int t = tid; t < n * G; t += blockDim.x) {
        const int j = t / G, u = t - j * G;
        float* ch = TF + (j / kKC) * 2 * G * kTfRow + (j % kKC);
        ch[u * kTfRow] = fa[t];
        ch[(G + u) * kTfRow] = fb[t];
    }
    __syncthreads();
    // ---- mu* = m + k_k* (f - m) ---------------------------------------------------------
    for (int q = tid; q < Q; q += blockDim.x) {
        float s = 0.f;
        for (int c = 0; c < n; ++c) {
            const int64_t o = pk_index(q, c, Kp);
            s = fmaf(Pk[o] + Pk[o + kRows * kKC], fv[c] - m, s);
        }
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
    __shared__ int s_axis;
    __shared__ float s_pv[32];
    __shared__ int s_pi[32];
    alg3_factor_one<false>(a, blockIdx.x, sm, red, s_axis, s_pv, s_pi);
}

// voxels beyond shared memory: persistent CTAs over the chunk's slots, ky in global memory
__global__ void __launch_bounds__(kA3Threads) k_alg3_factor_big(Alg3Args a)
{
    extern __shared__ __align__(16) unsigned char sm[];
    __shared__ float red[6 * 32];
    __shared__ int s_axis;
    __shared__ float s_pv[32];
    __shared__ int s_pi[32];
    for (int slot = blockIdx.x; slot < a.nchunk; slot += gridDim.x) {
        alg3_factor_one<true>(a, slot, sm, red, s_axis, s_pv, s_pi);
        __syncthreads();
    }
}

// ---- small PTX wrappers of the tensor-core kernel -------------------------------------
__device__ __forceinline__ uint64_t now_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// Waits for the phase of the given parity, the thread suspended in the barrier between
// tests; false after kWaitNs without completion.
__device__ __forceinline__ bool wait_bounded(uint64_t* mbar, uint32_t parity)
{
    const uint32_t a = umma::smem_addr(mbar);
    const uint64_t t0 = now_ns();
    for (;;) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done) : "r"(a), "r"(parity), "r"(1000u) : "memory");
        if (done) return true;
        if (now_ns() - t0 > kWaitNs) return false;
    }
}
__device__ __forceinline__ void expect_tx(uint64_t* mbar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                 :: "r"(umma::smem_addr(mbar)), "r"(bytes) : "memory");
}
// bulk copy global -> shared completing on the mbarrier (16-byte aligned, size % 16 == 0)
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* mbar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
        :: "r"(umma::smem_addr(dst)), "l"(src), "r"(bytes), "r"(umma::smem_addr(mbar))
        : "memory");
}
// eight consecutive 32-bit words to global memory in one 32-byte store (32-byte aligned)
__device__ __forceinline__ void st_v8(float* p, const uint32_t* o)
{
    asm volatile("st.global.v8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};"
                 :: "l"(p), "r"(o[0]), "r"(o[1]), "r"(o[2]), "r"(o[3]), "r"(o[4]), "r"(o[5]),
                    "r"(o[6]), "r"(o[7]) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* mbar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" :: "r"(umma::smem_addr(mbar)) : "memory");
}
// barrier `id` of `count` threads that also returns whether v holds in all of them
__device__ __forceinline__ bool named_and(int id, int count, bool v)
{
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 q, %3, 0;\n\t"
        "bar.red.and.pred p, %1, %2, q;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(r) : "r"(id), "r"(count), "r"((uint32_t)v) : "memory");
    return r != 0;
}

// Sigma* = K** - k_k* K*, tiles of 128 rows x NN columns (NN a multiple of 32, at most
// 128) of every voxel of the chunk, by persistent CTAs (tiles T = blockIdx.x,
// blockIdx.x + gridDim.x, ...: the tiles of one voxel, consecutive in T, run at the same
// time on neighbouring CTAs and share their k_k* and K* reads through L2).
// Warp roles (14 warps):
//   warp 13 (one lane): per chunk of 16 points, the pre-split k_k* tile (16 KB) and the
//     chunk's 2G rows of K* factors (80 bytes each) by two bulk copies into a ring of S
//     stages, once the MMAs have released the stage ("empty");
//   warps 8-11 (operands): form K*^T (K*(k, c) = fa(k, u) fb(k, x)) for the tile's
//     columns as a TF32 split pair in the stage ("b_ready", one arrival per warp);
//   warp 12 (one lane): per chunk, the three TF32 MMAs per 8 points (big*big +
//     big*small + small*big) into one of two tensor-memory accumulators of 128 lanes x NN
//     columns, committed to the stage's "empty" barrier and, after the tile's last chunk,
//     to the accumulator's "full" barrier; waits for the epilogue to release the
//     accumulator before a tile's first MMA;
//   warps 0-7 (epilogue): the node table of K** (exp(-lam d^2) over node differences)
//     when the voxel changes, then per tile for a solved voxel the accumulator (warps w and w + 4 read lanes
//     32 (w % 4) .. and one half of the columns each, loads one group ahead), K** - it,
//     32-byte stores and the release of the accumulator; voxels without a solution
//     (status not OK) get K** alone.
// The epilogue of one tile overlaps the MMAs of the next.  Every wait gives up after
// kWaitNs (or when another role has given up): the CTA stops, the voxels of its remaining
// tiles are marked failed, copies in flight and the last MMAs are waited for (bounded)
// and the tensor memory is freed.
constexpr int kCovWarps = 14;
__host__ __device__ inline int cov3_stage_bytes(int nn, int G)
{
    return cov_stage_bytes(nn) + 2 * G * kTfRow * 4;
}
// node table of K**: [G][G + 4] floats (rows 16-byte aligned, spread over the banks), then
// the G node positions
__host__ __device__ inline int cov3_table_bytes(int G) { return ((G * (G + 4) + G) * 4 + 15) & ~15; }

struct CovShared {
    uint64_t full[kCovStages], bready[kCovStages], empty[kCovStages], acc_full[2], acc_empty[2];
    uint32_t tslot;
    int abort_tile;   // first tile not completed after a time-out (INT_MAX: none)
    int issued;       // chunks whose copies were queued (copy warp)
    int consumed;     // chunks taken by the MMA warp
    int last_mma;     // last chunk whose MMAs were committed (-1: none)
};

// waits as wait_bounded, giving up early once another role has given up
__device__ __forceinline__ bool wait_or_abort(uint64_t* mbar, uint32_t parity, volatile int* abort_tile)
{
    const uint32_t a = umma::smem_addr(mbar);
    const uint64_t t0 = now_ns();
    for (;;) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done) : "r"(a), "r"(parity), "r"(1000u) : "memory");
        if (done) return true;
        if (*abort_tile != 0x7fffffff || now_ns() - t0 > kWaitNs) return false;
    }
}
__device__ __forceinline__ void tmem_ld16_async(uint32_t taddr, uint32_t (&r)[16])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
          "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]),
          "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

__global__ void __launch_bounds__(kCovWarps * 32, 2) k_alg3_cov(Alg3Args a, int NN, int S, int ntiles)
{
    extern __shared__ __align__(128) unsigned char smb[];
    __shared__ CovShared sh;
    const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
    const int G = a.G, GS = G + 4, Q = G * G, Kp = a.kp;
    const int nrx = (Q + kRows - 1) / kRows, ncy = (Q + NN - 1) / NN, tpv = nrx * ncy;
    const int SB = cov3_stage_bytes(NN, G);
    float* e1 = reinterpret_cast<float*>(smb + S * SB);  // [G][G + 4], the epilogue's
    float* nodes = e1 + G * GS;
    constexpr uint32_t kAccCols = 128;                   // columns per accumulator
    volatile int* abort_tile = &sh.abort_tile;
    if (w == 0) umma::tmem_alloc(&sh.tslot, 2 * kAccCols);
    if (tid == 32) {
        for (int s = 0; s < kCovStages; ++s) {
            umma::mbar_init(&sh.full[s], 1);
            umma::mbar_init(&sh.bready[s], 4);
            umma::mbar_init(&sh.empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            umma::mbar_init(&sh.acc_full[b], 1);
            umma::mbar_init(&sh.acc_empty[b], 8);
        }
        sh.abort_tile = 0x7fffffff;
        sh.issued = 0;
        sh.consumed = 0;
        sh.last_mma = -1;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    for (int i = tid; i < G; i += blockDim.x) nodes[i] = node_pos(i, G, a.size);
    umma::fence_before_sync();
    __syncthreads();
    umma::fence_after_sync();
    const uint32_t tmem = sh.tslot;
    auto give_up = [&](int T) { atomicMin(&sh.abort_tile, T); };
    if (w == 13) {  // ---- copies ----------------------------------------------------------
        int gi = 0;
        for (int T = blockIdx.x; T < ntiles; T += gridDim.x) {
            if (__shfl_sync(0xffffffffu, *abort_tile, 0) != 0x7fffffff) break;
            const int slot = T / tpv, rx = (T - slot * tpv) / ncy;
            if (a.ws_status[slot] != VOX_OK) continue;
            const int nch = (a.ws_n[slot] + kKC - 1) / kKC;
            const float* src = a.ws_pk + ((int64_t)slot * 2 * a.qp + rx * 2 * kRows) * Kp;
            const float* tf = a.ws_tf + (int64_t)slot * (Kp / kKC) * 2 * G * kTfRow;
            bool ok = true;
            for (int i = 0; i < nch; ++i, ++gi) {
                const int s = gi % S, k = gi / S;
                if (k > 0) {
                    bool r = true;
                    if (lane == 0) r = wait_or_abort(&sh.empty[s], (uint32_t)(k - 1) & 1u, abort_tile);
                    ok = __shfl_sync(0xffffffffu, (int)r, 0) != 0;
                    if (!ok) break;
                }
                unsigned char* stg = smb + s * SB;
                if (lane == 0) {
                    const uint32_t tfb = 2 * G * kTfRow * 4;
                    expect_tx(&sh.full[s], 2 * kRows * kKC * 4 + tfb);
                    bulk_g2s(stg, src + (int64_t)i * 2 * kRows * kKC, 2 * kRows * kKC * 4, &sh.full[s]);
                    bulk_g2s(stg + cov_stage_bytes(NN), tf + (int64_t)i * 2 * G * kTfRow, tfb, &sh.full[s]);
                }
            }
            if (!ok) {
                if (lane == 0) give_up(T);
                break;
            }
        }
        if (lane == 0) sh.issued = gi;
    } else if (w >= 8 && w < 12) {  // ---- K*^T operand ------------------------------------
        const int pt = tid - 256;
        int gi = 0;
        for (int T = blockIdx.x; T < ntiles; T += gridDim.x) {
            if (__any_sync(0xffffffffu, *abort_tile != 0x7fffffff)) break;
            const int slot = T / tpv, cy = (T - slot * tpv) % ncy;
            if (a.ws_status[slot] != VOX_OK) continue;
            const int n = a.ws_n[slot], nch = (n + kKC - 1) / kKC, c0 = cy * NN;
            // groups of this thread: group g = 16-byte group (row r, points 4j .. 4j+3) of
            // the B operand, at byte 16 g of its buffer
            // (the point offset 4j is the same for the four groups of a thread)
            const int kg = 4 * ((pt >> 3) & 3);
            int oa[4], ob[4];
            bool gv[4], cv[4];
#pragma unroll
            for (int h = 0; h < 4; ++h) {
                const int g = pt + 128 * h;
                const int c = c0 + (g >> 5) * 8 + (g & 7);
                gv[h] = g < NN * 4;
                cv[h] = gv[h] && c < Q;
                const int u2 = cv[h] ? c / G : 0, x2 = cv[h] ? c - u2 * G : 0;
                oa[h] = u2 * kTfRow + kg;
                ob[h] = (G + x2) * kTfRow + kg;
            }
            bool ok = true;
            for (int i = 0; i < nch; ++i, ++gi) {
                const int s = gi % S;
                ok = __all_sync(0xffffffffu, wait_or_abort(&sh.full[s], (uint32_t)(gi / S) & 1u, abort_tile));
                if (!ok) break;
                unsigned char* stg = smb + s * SB;
                float* Bb = reinterpret_cast<float*>(stg + 2 * kRows * kKC * 4);
                float* Bs = Bb + NN * kKC;
                const float* tfs = Bs + NN * kKC;
#pragma unroll
                for (int h = 0; h < 4; ++h) {  // B = K*^T, zero beyond the voxel's points
                    if (!gv[h]) continue;
                    const int k = i * kKC + kg;
                    float4 pa = make_float4(0.f, 0.f, 0.f, 0.f), pb = pa;
                    if (cv[h]) {
                        pa = *reinterpret_cast<const float4*>(tfs + oa[h]);
                        pb = *reinterpret_cast<const float4*>(tfs + ob[h]);
                    }
                    float4 bg, sl;
                    umma::tf32_split(k < n ? pa.x * pb.x : 0.f, bg.x, sl.x);
                    umma::tf32_split(k + 1 < n ? pa.y * pb.y : 0.f, bg.y, sl.y);
                    umma::tf32_split(k + 2 < n ? pa.z * pb.z : 0.f, bg.z, sl.z);
                    umma::tf32_split(k + 3 < n ? pa.w * pb.w : 0.f, bg.w, sl.w);
                    const int g = pt + 128 * h;
                    reinterpret_cast<float4*>(Bb)[g] = bg;
                    reinterpret_cast<float4*>(Bs)[g] = sl;
                }
                umma::fence_proxy_async_smem();
                __syncwarp();
                if (lane == 0) mbar_arrive(&sh.bready[s]);
            }
            if (!ok) {
                if (lane == 0) give_up(T);
                break;
            }
        }
    } else if (w == 12) {  // ---- MMAs (one lane) ------------------------------------------
        if (lane == 0) {
            int gi = 0, ts = 0, last = -1;
            const uint32_t idesc = umma::idesc_tf32(kRows, NN);
            for (int T = blockIdx.x; T < ntiles; T += gridDim.x) {
                if (*abort_tile != 0x7fffffff) break;
                const int slot = T / tpv;
                if (a.ws_status[slot] != VOX_OK) continue;
                const int nch = (a.ws_n[slot] + kKC - 1) / kKC;
                const int b = ts & 1, m = ts >> 1;
                bool ok = true;
                if (m > 0)  // the epilogue has released this accumulator
                    ok = wait_or_abort(&sh.acc_empty[b], (uint32_t)(m - 1) & 1u, abort_tile);
                for (int i = 0; ok && i < nch; ++i, ++gi) {
                    const int s = gi % S;
                    const uint32_t par = (uint32_t)(gi / S) & 1u;
                    ok = wait_or_abort(&sh.bready[s], par, abort_tile) &&
                         wait_or_abort(&sh.full[s], par, abort_tile);
                    if (!ok) break;
                    umma::fence_after_sync();
                    unsigned char* stg = smb + s * SB;
                    const uint32_t ab = umma::smem_addr(stg), as = ab + kRows * kKC * 4;
                    const uint32_t bb = as + kRows * kKC * 4, bs = bb + NN * kKC * 4;
                    const uint32_t d = tmem + (uint32_t)b * kAccCols;
                    constexpr int sbo = (kKC / 4) * umma::kLBO;
#pragma unroll
                    for (int k8 = 0; k8 < kKC / 8; ++k8) {
                        const uint32_t off = k8 * 2 * umma::kLBO;
                        const uint64_t dab = umma::make_desc(ab + off, umma::kLBO, sbo);
                        const uint64_t das = umma::make_desc(as + off, umma::kLBO, sbo);
                        const uint64_t dbb = umma::make_desc(bb + off, umma::kLBO, sbo);
                        const uint64_t dbs = umma::make_desc(bs + off, umma::kLBO, sbo);
                        umma::mma_tf32(d, dab, dbb, idesc, i > 0 || k8 > 0);
                        umma::mma_tf32(d, dab, dbs, idesc, true);
                        umma::mma_tf32(d, das, dbb, idesc, true);
                    }
                    umma::mma_commit(&sh.empty[s]);
                    if (i == nch - 1) umma::mma_commit(&sh.acc_full[b]);
                    last = gi;
                }
                if (!ok) {
                    give_up(T);
                    break;
                }
                ++ts;
            }
            sh.consumed = gi;
            sh.last_mma = last;
        }
    } else {  // ---- epilogue (warps 0-7) ----------------------------------------------------
        const int q4 = w & 3, ncol = NN / 2, cbeg = (w >> 2) * ncol;
        // 32-byte stores: 16-column groups never straddle the end of a row, aligned base;
        // with G a multiple of 16 a group also stays within one row of nodes (u2 fixed)
        const bool vec = (Q & 15) == 0 && (reinterpret_cast<uintptr_t>(a.cov) & 31) == 0;
        const bool fast = vec && (G & 15) == 0;
        int ts = 0, e1_slot = -1;
        for (int T = blockIdx.x; T < ntiles; T += gridDim.x) {
            // (also: every thread is done with the node table before it is rewritten)
            if (!named_and(1, 256, *abort_tile == 0x7fffffff)) break;
            const int slot = T / tpv, rem = T - slot * tpv, rx = rem / ncy, cy = rem - rx * ncy;
            const int v = a.vidx[a.s0 + slot];
            const bool solve = a.ws_status[slot] == VOX_OK;
            const float sf2 = a.sf2[v], lam = a.lam[v];
            if (slot != e1_slot) {  // the node table of this voxel's length scale
                for (int t = tid; t < G * G; t += 256) {
                    const int i = t / G, j = t - i * G;
                    const float d = nodes[i] - nodes[j];
                    e1[i * GS + j] = expf(-lam * d * d);
                }
                e1_slot = slot;
            }
            const int b = ts & 1, m = ts >> 1;
            bool ok = true;
            if (solve) ok = wait_or_abort(&sh.acc_full[b], (uint32_t)m & 1u, abort_tile);
            if (!named_and(1, 256, ok)) {  // the same decision in every epilogue thread
                if (tid == 0) give_up(T);
                break;
            }
            if (solve) umma::fence_after_sync();
            const int row = rx * kRows + 32 * q4 + lane;
            const int u = row / G, x = row - u * G;
            float* out = a.cov + ((int64_t)v * Q + row) * Q;
            const uint32_t tb = tmem + ((uint32_t)(32 * q4) << 16) + (uint32_t)b * kAccCols + (uint32_t)cbeg;
            uint32_t r0[16], r1[16];
            if (solve) {
                tmem_ld16_async(tb, r0);
                tmem_wait_ld();
            }
            for (int cc = 0; cc < ncol; cc += 16) {
                if (!solve)  // K** alone
#pragma unroll
                    for (int t = 0; t < 16; ++t) r0[t] = 0u;
                const bool more = solve && cc + 16 < ncol;  // the next group's load in flight
                if (more) tmem_ld16_async(tb + (uint32_t)(cc + 16), r1);
                const int c = cy * NN + cbeg + cc;
                if (row < Q && c < Q) {  // Sigma* = K** - accumulator, in place in r0
                    if (fast) {
                        const int u2 = c / G, x2 = c - u2 * G;
                        const float su = sf2 * e1[u * GS + u2];
                        const float4* ex = reinterpret_cast<const float4*>(e1 + x * GS + x2);
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            const float4 e = ex[q];
                            r0[4 * q] = __float_as_uint(su * e.x - __uint_as_float(r0[4 * q]));
                            r0[4 * q + 1] = __float_as_uint(su * e.y - __uint_as_float(r0[4 * q + 1]));
                            r0[4 * q + 2] = __float_as_uint(su * e.z - __uint_as_float(r0[4 * q + 2]));
                            r0[4 * q + 3] = __float_as_uint(su * e.w - __uint_as_float(r0[4 * q + 3]));
                        }
                    } else {
                        int u2 = c / G, x2 = c - u2 * G;
#pragma unroll
                        for (int t = 0; t < 16; ++t) {
                            r0[t] = __float_as_uint(sf2 * e1[u * GS + u2] * e1[x * GS + x2] - __uint_as_float(r0[t]));
                            if (++x2 == G) { x2 = 0; ++u2; }
                        }
                    }
                    if (vec) {
                        st_v8(out + c, r0);
                        st_v8(out + c + 8, r0 + 8);
                    } else {
#pragma unroll
                        for (int t = 0; t < 16; ++t)
                            if (c + t < Q) out[c + t] = __uint_as_float(r0[t]);
                    }
                }
                __syncwarp();  // converged for the warp-wide wait
                if (more) {
                    tmem_wait_ld();
#pragma unroll
                    for (int t = 0; t < 16; ++t) r0[t] = r1[t];
                }
            }
            if (solve) {  // release the accumulator to the MMAs of the tile after next
                umma::fence_before_sync();
                __syncwarp();
                if (lane == 0) mbar_arrive(&sh.acc_empty[b]);
                ++ts;
            }
        }
    }
    __syncthreads();
    const int at = sh.abort_tile;
    if (at != 0x7fffffff) {
        // copies in flight and the last MMAs (bounded waits), then the voxels of every
        // tile of this CTA from the first one not completed are marked failed
        if (tid == 0) {
            for (int j = sh.consumed; j < sh.issued; ++j)
                wait_bounded(&sh.full[j % S], (uint32_t)(j / S) & 1u);
            if (sh.last_mma >= 0)
                wait_bounded(&sh.empty[sh.last_mma % S], (uint32_t)(sh.last_mma / S) & 1u);
        }
        for (int T = at + tid * gridDim.x; T < ntiles; T += (int)blockDim.x * gridDim.x)
            atomicOr(a.status + a.vidx[a.s0 + T / tpv], VOX_FAILED);
    }
    umma::fence_before_sync();
    __syncthreads();
    if (w == 0) umma::tmem_free(tmem, 2 * kAccCols);
}

__global__ void k_alg3_order(const int64_t* offsets, int32_t nvox, int nsm, int nmax, int tau,
                             int32_t* vidx, int32_t* counts)
{
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nvox) return;
    const int64_t n = offsets[v + 1] - offsets[v];
    if (n > nsm && n <= nmax && n >= tau) vidx[atomicAdd(counts, 1)] = v;
    else vidx[nvox - 1 - atomicAdd(counts + 1, 1)] = v;
}

}  // namespace

cudaError_t alg3_order(const int64_t* offsets, int32_t nvox, int nsm, int nmax, int tau,
                       int32_t* vidx, int32_t* counts, cudaStream_t s)
{
    if (nvox <= 0) return cudaSuccess;
    k_alg3_order<<<(nvox + 255) / 256, 256, 0, s>>>(offsets, nvox, nsm, nmax, tau, vidx, counts);
    return cudaGetLastError();
}

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

cudaError_t alg3_launch_chunk(const Alg3Args& a0, int nchunk, cudaStream_t s, cudaStream_t side,
                              cudaEvent_t ev_fork, cudaEvent_t ev_join, int* nlaunch)
{
    *nlaunch = 0;
    const bool big = a0.nmax > a0.nsm;
    cudaError_t e;
    if (big) {  // the class beyond shared memory (its voxels lead the order) on the side stream
        if ((e = cudaEventRecord(ev_fork, s)) != cudaSuccess) return e;
        if ((e = cudaStreamWaitEvent(side, ev_fork, 0)) != cudaSuccess) return e;
        Alg3Args a = a0;
        a.nlo = a0.nsm;
        a.nhi = a0.nmax;
        a.nchunk = nchunk;
        const int smemA = a3_plan(a0.nmax, a0.G, true).total;
        e = cudaFuncSetAttribute(k_alg3_factor_big, cudaFuncAttributeMaxDynamicSharedMemorySize, smemA);
        if (e != cudaSuccess) return e;
        const int grid = nchunk < alg3_big_ctas() ? nchunk : alg3_big_ctas();
        k_alg3_factor_big<<<grid, kA3Threads, smemA, side>>>(a);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        ++*nlaunch;
        if ((e = cudaEventRecord(ev_join, side)) != cudaSuccess) return e;
    }
    // kernel A in three size classes, each launch with the shared memory of its largest n
    const int nsm = a0.nsm < a0.nmax ? a0.nsm : a0.nmax;  // largest n of the shared-memory classes
    const int cls[3] = {64, 128, nsm};
    e = cudaFuncSetAttribute(k_alg3_factor, cudaFuncAttributeMaxDynamicSharedMemorySize,
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
    if (big && (e = cudaStreamWaitEvent(s, ev_join, 0)) != cudaSuccess) return e;
    const Alg3Args& a = a0;
    const int Q = a.G * a.G;
    const int NN = Q >= 128 ? 128 : (Q + 31) / 32 * 32;  // columns per tile (multiple of 32)
    const int ntiles = nchunk * ((Q + kRows - 1) / kRows) * ((Q + NN - 1) / NN);
    // two CTAs per SM (each holds 256 tensor-memory columns: two accumulators); three
    // operand stages where two such CTAs fit the SM's shared memory, else two
    const int per_sm = 233472, reserve = 1024 + (int)sizeof(CovShared) + 64;
    const int e1b = cov3_table_bytes(a.G);
    int S = kCovStages;
    if (2 * (S * cov3_stage_bytes(NN, a.G) + e1b + reserve) > per_sm) S = 2;
    int smemB = S * cov3_stage_bytes(NN, a.G) + e1b;
    if (smemB < per_sm / 3 + 16) smemB = per_sm / 3 + 16;  // never a third CTA (tensor memory)
    e = cudaFuncSetAttribute(k_alg3_cov, cudaFuncAttributeMaxDynamicSharedMemorySize, smemB);
    if (e != cudaSuccess) return e;
    const int nsms = alg3_big_ctas();  // the SM count
    const int grid = ntiles < 2 * nsms ? ntiles : 2 * nsms;
    k_alg3_cov<<<grid, kCovWarps * 32, smemB, s>>>(a, NN, S, ntiles);
    ++*nlaunch;
    return cudaGetLastError();
}

}  // namespace gpv
