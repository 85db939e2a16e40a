// gpv_vartc.cu -- diag(Sigma*) of Eq. 3 on the fifth-generation tensor cores for the
// float-float path, var_q = sf2 - |L^-1 k_q|^2, followed by the Gaussians of Sec. 3.2
// (Eq. 6-8).  The solve kernel leaves L^-1 (packed lower triangle, column-major), the
// separable cross-covariance factors a_i(u), b_i(v) and the means of each voxel in a
// workspace; this kernel forms V = L^-1 K* and its column norms.
//
// Precision.  Where points are dense, sf2 and |L^-1 k_q|^2 agree to about five digits,
// so V needs some 48 significant bits, more than any single tensor-core product
// carries.  The error-free splitting of Ozaki, Ogita, Oishi and Rump (Numer. Algorithms
// 59, 2012) gets them from BF16 products: every entry is cut into six slices of 8 bits on
// a power-of-two grid shared by its row (row j of L^-1: 2^(E_j - 1) > max_i |L^-1_ji|; the
// column of query q in K*: 2^(F_q - 1) > max_i |k_iq|).  Slice s of an entry is a multiple
// of 2^(E - 8(s+1)) of at most 2^7 grid units, so it is exactly a BF16 number, and a
// product of two slices is exact in FP32 (at most 2^14 units).  All products of one level
// l = s + t lie on one grid, and for l <= 4 the sum of their magnitudes over the pairs of
// the level and over i stays below 2^24 grid units when n < 204 (level 4: 5 * 2^14 n), so
// the tensor core's FP32 accumulation of each of these levels is exact.  Level 5 has an
// accumulator of its own too, inexact: its values stay near 2^-32 of 2^(E_j + F_q), its
// FP32 rounding far below 2^-48 of that scale.  (A level's sum is not small: it reaches
// 2^19 of its own grid, which is why every level down to 4 needs an exact accumulator.)
// Pairs with s + t > 5 are dropped (2^-48).  V = L0 + ... + L5 is assembled and squared
// in float-float.
//
// Up to 160 points levels 4 and 5 share the fifth accumulator (its rounding stays near 2^-48
// of the row scale at that size) and a pass takes 96 rows of L^-1; above, six accumulators
// of 80 columns.
//
// Organisation.  Each size bucket launches this kernel on its own stream right after its
// solve launch, over the same work list, so it runs while other buckets still factor; a CTA
// of it holds most of an SM's registers and all of its tensor memory, so on each SM the two
// kernels take turns, and this kernel's own speed adds to the step.  One persistent CTA
// per SM (512 threads) owns the tensor memory: five or six accumulators of 128 lanes (the
// queries of one M tile) x up to 96 or 80 columns (rows j of L^-1 per pass).  For each
// 16-wide chunk of i, all threads cut the A slices (K*^T: 128 queries x 16) and the B
// slices (L^-1: up to 96 rows x 16) into one of two shared-memory buffers while the tensor
// core works on the other, with the next chunk's operands already on their way from
// memory (a voxel of one pass keeps the L^-1 slices of all its chunks for its second M
// tile); after one barrier, one thread issues the 21 MMAs (kind::f16, M = 128, N = rows
// of the pass, K = 16) and commits them to the buffer's mbarrier, which each thread checks
// before it writes that buffer again.  The epilogue reads the accumulators with
// tcgen05.ld: lane = query, so each thread sums its own query's norm with no cross-thread
// reduction.  Every wait is bounded; a wait that gives up marks the voxel GPV_VOX_FAILED.
#include <cuda_runtime.h>
#include <stdint.h>

#include "gpv_init.cuh"
#include "gpv_internal.h"
#include "gpv_num.cuh"
#include "gpv_umma.cuh"

namespace gpv {
namespace {

constexpr int kVT = 512;      // threads per CTA
constexpr int kSl = 6;        // slices per operand entry
constexpr int kLv = 6;        // accumulators: levels 0 .. 5 (n > kLv5MaxN), else 0 .. 3 and 4..5
constexpr int kMT = 128;      // queries per M tile (tensor-memory lanes)
constexpr int kNJ = 80;       // rows of L^-1 per pass with six accumulators (6 * 80 <= 512)
constexpr int kNJ5 = 96;      // with five accumulators (5 * 96 <= 512)
constexpr int kLv5MaxN = 160; // up to here levels 4 and 5 share an accumulator
constexpr int kKC = 16;       // K of one MMA (BF16)
constexpr int kSliceBytes = 128 * kKC * 2;  // one slice of a 128 x 16 operand chunk
constexpr int kParts = kVT / kMT;             // threads per operand row (K chunk split)
constexpr int kKE = kKC / kParts;             // K entries per thread and chunk
constexpr uint32_t kPolls = 1u << 26;

// dynamic shared memory (bytes)
constexpr int kOffA = 0;                                   // [2][kSl] A chunks
// B chunk slots: a voxel of one pass (n <= 96) with more than one M tile keeps the slices
// of every chunk of L^-1 (at most six) for all its tiles; other voxels use two as stages
constexpr int kBSlots = 6;
static_assert(kNJ5 <= kBSlots * kKC, "a one-pass voxel has at most kBSlots chunks");
constexpr int kOffB = kOffA + 2 * kSl * kSliceBytes;       // [kBSlots][kSl] B chunks
constexpr int kOffNrm = kOffB + kBSlots * kSl * kSliceBytes;  // ff partial norms [kParts][kMT]
constexpr int kOffEnd = kOffNrm + kParts * kMT * 8;
// at least 120 KB, more than half an SM's shared memory, so that one CTA per SM holds
// the tensor memory
constexpr int kVarTcSmem = kOffEnd > 120 * 1024 ? kOffEnd : 120 * 1024;

__device__ __forceinline__ int tri_off_p(int c, int n) { return c * n - ((c * (c - 1)) >> 1); }

// Cut x = hi + lo (|x| < 2^(E-1)) into kSl slices on the grids 2^(E-8), ..., 2^(E-48):
// round to the grid by adding and subtracting 1.5 * 2^(grid exponent + 23), keep the
// exact remainder.  The first three slices come from hi alone; lo joins the remainder
// for the last three (that FP32 sum errs by at most 2^(E-49)).  Returns the FP32 bit
// patterns; each slice has at most 8 significant bits, so its upper half is its BF16.
__device__ __forceinline__ void cut_slices(float hi, float lo, int E, uint32_t (&q)[kSl])
{
    float a = hi;
#pragma unroll
    for (int s = 0; s < kSl; ++s) {
        if (s == 3) a = __fadd_rn(a, lo);
        const float sig = __uint_as_float(((uint32_t)(E - 8 * s + 15 + 127) << 23) | 0x400000u);
        const float t = __fsub_rn(__fadd_rn(a, sig), sig);
        a = __fsub_rn(a, t);
        q[s] = __float_as_uint(t);
    }
}

// Byte offset of element (r, k) of a K-major, unswizzled BF16 chunk with 16 elements per
// row: core matrices of 8 rows x 16 bytes, the two along K adjacent (LBO 128), 8-row
// groups 256 bytes apart (SBO).
__device__ __forceinline__ int kmaj16(int r, int k)
{
    return (r >> 3) * 256 + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2;
}

// Slices of NE (4 or 8) consecutive K entries of one operand row, stored in each of the
// kSl slice buffers as NE * 2 bytes of a core-matrix row.
template <int NE>
__device__ __forceinline__ void store_row(unsigned char* buf, int r, int k0, const float (&hi)[NE],
                                          const float (&lo)[NE], int E)
{
    uint32_t w[kSl][NE / 2];
#pragma unroll
    for (int p = 0; p < NE / 2; ++p) {
        uint32_t a[kSl], b[kSl];
        cut_slices(hi[2 * p], lo[2 * p], E, a);
        cut_slices(hi[2 * p + 1], lo[2 * p + 1], E, b);
#pragma unroll
        for (int s = 0; s < kSl; ++s) w[s][p] = __byte_perm(a[s], b[s], 0x7632);
    }
    const int o = kmaj16(r, k0);
#pragma unroll
    for (int s = 0; s < kSl; ++s) {
        if constexpr (NE == 8)
            *reinterpret_cast<uint4*>(buf + s * kSliceBytes + o) = make_uint4(w[s][0], w[s][1], w[s][2], w[s][3]);
        else
            *reinterpret_cast<uint2*>(buf + s * kSliceBytes + o) = make_uint2(w[s][0], w[s][1]);
    }
}

__device__ __forceinline__ void tmem_ld8_nowait(uint32_t taddr, uint32_t (&r)[8])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
          "=r"(r[6]), "=r"(r[7])
        : "r"(taddr));
}

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Ties the registers of a tcgen05.ld to a point after tcgen05.wait::ld: the compiler may
// not read them before this (ordered) statement.
__device__ __forceinline__ void reg_fence8(uint32_t (&r)[8])
{
    asm volatile(""
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]),
                   "+r"(r[6]), "+r"(r[7]));
}

// Pulls a voxel's workspace (bytes from p) toward L2 while the CTA works on another voxel.
__device__ __forceinline__ void prefetch_l2(const unsigned char* p, uint64_t bytes)
{
    for (uint64_t o = (uint64_t)threadIdx.x * 128; o < bytes; o += (uint64_t)blockDim.x * 128)
        asm volatile("prefetch.global.L2 [%0];" :: "l"(p + o));
}

// nrm += V^2 with V = l0 + ... + l5 (the levels of one entry of L^-1 K*): the exact levels
// join the leading part by TwoSum, their errors and the last level the trailing part
__device__ __forceinline__ void acc_levels(ff& nrm, float l0, float l1, float l2, float l3, float l4,
                                           float l5)
{
    const ff a = two_sum(l0, l1);
    const ff b = two_sum(a.hi, l2);
    const ff c = two_sum(b.hi, l3);
    const ff d = two_sum(c.hi, l4);
    const ff V = ff_make(d.hi, __fadd_rn(__fadd_rn(__fadd_rn(a.lo, b.lo), __fadd_rn(c.lo, d.lo)), l5));
    acc_fma(nrm, V, V);
}

__device__ void write_failed(const SolveArgs& A, int v, int GG, float sf2f)
{
    for (int q = threadIdx.x; q < GG; q += blockDim.x) A.var[(int64_t)v * GG + q] = sf2f;
    if (A.pos) {
        const int NG = A.n_s * A.n_s;
        for (int g = threadIdx.x; g < NG; g += blockDim.x) {
            const int64_t o = (int64_t)v * NG + g;
            for (int k = 0; k < 3; ++k) { A.pos[3 * o + k] = A.centres[3 * v + k]; A.scale[3 * o + k] = 0.f; }
            A.quat[4 * o] = 1.f; A.quat[4 * o + 1] = 0.f; A.quat[4 * o + 2] = 0.f; A.quat[4 * o + 3] = 0.f;
        }
    }
    if (threadIdx.x == 0) A.status[v] |= VOX_FAILED;
}

__global__ void __launch_bounds__(kVT, 1) k_var_tc(SolveArgs A)
{
    extern __shared__ __align__(16) unsigned char sm[];
    __shared__ __align__(8) uint64_t mbar[2];
    __shared__ uint32_t tslot;
    __shared__ int s_item, s_next;
    __shared__ int s_broken;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // the voxels of one size bucket (the solve launch's own work list)
    const int32_t* work = A.work + (A.work_base ? *A.work_base : 0);
    const int count = *A.work_count;
    if (count == 0) return;
    ff* nrm2 = reinterpret_cast<ff*>(sm + kOffNrm);
    const int G = A.G, Gp = A.Gp, GG = G * G;
    if (warp == 0) umma::tmem_alloc(&tslot, 512);
    if (tid == 0) {
        umma::mbar_init(&mbar[0], 1);
        umma::mbar_init(&mbar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_broken = 0;
    }
    umma::fence_before_sync();
    __syncthreads();
    umma::fence_after_sync();
    const uint32_t tmem = tslot;
    const uint32_t abase = umma::smem_addr(sm + kOffA), bbase = umma::smem_addr(sm + kOffB);
    uint32_t uses[2] = {0u, 0u};  // commits issued per buffer (identical in every thread)
    int chunk = 0;
    if (tid == 0) s_item = atomicAdd(A.work_next, 1);
    __syncthreads();

    for (;;) {
        const int it = s_item;
        if (it >= count) break;
        if (tid == 0) s_next = atomicAdd(A.work_next, 1);  // one voxel ahead
        const int v = work[it];
        const long long off = A.tc_off_v[v];
        const int n = (int)(A.offsets[v + 1] - A.offsets[v]);
        const float sf2f = A.sf2[v];
        __syncthreads();
        {   // the next voxel's workspace travels to L2 meanwhile
            const int nx = s_next;
            if (nx < count) {
                const int vn = work[nx];
                const long long on = A.tc_off_v[vn];
                const int nn = (int)(A.offsets[vn + 1] - A.offsets[vn]);
                if (on >= 0) prefetch_l2(A.tc_ws + on, tc_need_bytes(nn, G, Gp));
            }
        }
        if (off < 0) {  // not handed over: escalated, not SPD, or re-solved by the regular kernel
            __syncthreads();
            if (tid == 0) s_item = s_next;
            __syncthreads();
            continue;
        }
        if (s_broken) {
            write_failed(A, v, GG, sf2f);
            __syncthreads();
            if (tid == 0) s_item = s_next;
            __syncthreads();
            continue;
        }
        const int ntri = n * (n + 1) / 2;
        const ff* X = reinterpret_cast<const ff*>(A.tc_ws + off);
        const ff* FA = X + ntri;
        const ff* FB = FA + n * G;
        const ff* MU = FB + n * Gp;
        ff* VAR = const_cast<ff*>(MU) + GG;
        const int* EX = reinterpret_cast<const int*>(VAR + GG);  // slice exponents: rows of
        const int* FQ = EX + n;                                  // L^-1, then the queries
        bool failed = false;
        const int r = tid & (kMT - 1), h = tid >> 7;  // operand row, part of the K chunk
        // up to kLv5MaxN points levels 4 and 5 share an accumulator (their FP32 rounding stays
        // near 2^-48 of the row scale) and a pass takes 96 rows; above, level 4 is exact too
        const int nlv = n > kLv5MaxN ? kLv : kLv - 1;
        const int njp = n > kLv5MaxN ? kNJ : kNJ5;
        // one pass and several M tiles: L^-1 is cut once, during the first tile
        const bool keepB = n <= njp && GG > kMT;
        for (int mt = 0; mt * kMT < GG && !failed; ++mt) {
            const bool cutB = !keepB || mt == 0;
            const int q = mt * kMT + r;
            const bool qv = q < GG;
            const int u = qv ? q / G : 0, w = qv ? q - u * G : 0;
            const int F = qv ? FQ[q] : 0;
            ff nrm = zero<ff>();
            for (int j0 = 0; j0 < n && !failed; j0 += njp) {
                const int nj = min(njp, n - j0), Np = (nj + 15) & ~15;
                const int nkc = (min(n, j0 + nj) + kKC - 1) / kKC;  // rows j < j0 + nj need i <= j
                const int j = j0 + r;
                const int Ej = j < n ? EX[j] : 0;
                uint32_t started = 0u;  // accumulators written in this pass (thread 0)
                // operands of a chunk, loaded one chunk ahead: their latency overlaps the
                // barrier and the MMA issue of the chunk before
                ff pa[kKE], pb[kKE], px[kKE];
                auto load_chunk = [&](int kc) {
                    const int i0 = kc * kKC + kKE * h;
#pragma unroll
                    for (int e = 0; e < kKE; ++e) {
                        const int i = i0 + e;
                        const bool ia = qv && i < n;
                        pa[e] = ia ? FA[i * G + u] : zero<ff>();
                        pb[e] = ia ? FB[i * Gp + w] : zero<ff>();
                        px[e] = (cutB && j < n && i <= j) ? X[tri_off_p(i, n) + j - i] : zero<ff>();
                    }
                };
                load_chunk(0);
                for (int kc = 0; kc < nkc; ++kc) {
                    const int b = chunk & 1;
                    // each thread sees for itself that the MMAs which last read this buffer
                    // are done before it writes there; a wait that gave up skips the writes
                    // and is shared at the barrier below
                    bool bad = false;
                    if (uses[b] > 0) bad = !umma::mbar_wait(&mbar[b], (uses[b] - 1) & 1, kPolls);
                    unsigned char* abuf = sm + kOffA + b * kSl * kSliceBytes;
                    const int bs = keepB ? kc : b;  // B slot: its earlier readers finished
                    unsigned char* bbuf = sm + kOffB + bs * kSl * kSliceBytes;  // by the last pass end
                    if (!bad) {
                        {   // A: k(x_i, q) = a_i(u) b_i(v) for the 128 queries of the tile
                            float hi[kKE], lo[kKE];
#pragma unroll
                            for (int e = 0; e < kKE; ++e) {
                                const ff k = pa[e] * pb[e];  // zero past n and past G^2
                                hi[e] = k.hi;
                                lo[e] = k.lo;
                            }
                            store_row<kKE>(abuf, r, kKE * h, hi, lo, F);
                        }
                        if (cutB) {   // B: row j of L^-1, zero above the diagonal and past n
                            float hi[kKE], lo[kKE];
#pragma unroll
                            for (int e = 0; e < kKE; ++e) {
                                hi[e] = px[e].hi;
                                lo[e] = px[e].lo;
                            }
                            store_row<kKE>(bbuf, r, kKE * h, hi, lo, Ej);
                        }
                    }
                    if (kc + 1 < nkc) load_chunk(kc + 1);
                    umma::fence_proxy_async_smem();
                    if (__syncthreads_or(bad)) { failed = true; break; }
                    if (tid == 0) {
                        umma::fence_after_sync();
                        const uint32_t idesc = umma::idesc_bf16(kMT, Np);
                        const uint32_t a0 = abase + b * kSl * kSliceBytes;
                        const uint32_t b0 = bbase + bs * kSl * kSliceBytes;
#pragma unroll
                        for (int s = 0; s < kSl; ++s)
#pragma unroll
                            for (int t = 0; s + t < kSl; ++t) {
                                const int lv = min(s + t, nlv - 1);
                                const bool acc = (started >> lv) & 1u;
                                started |= 1u << lv;
                                umma::mma_bf16(tmem + lv * njp, umma::make_desc(a0 + t * kSliceBytes, 128, 256),
                                               umma::make_desc(b0 + s * kSliceBytes, 128, 256), idesc, acc);
                            }
                        umma::mma_commit(&mbar[b]);
                    }
                    ++uses[b];
                    ++chunk;
                }
                if (failed) break;
                {   // all MMAs of the pass are done once its last commit has arrived
                    const int lb = (chunk - 1) & 1;
                    const bool ok = umma::mbar_wait(&mbar[lb], (uses[lb] - 1) & 1, kPolls);
                    if (__syncthreads_or(!ok)) { failed = true; break; }
                }
                umma::fence_after_sync();
                {   // epilogue: warps w, w + 4, .. read lanes 32 (w % 4) ..; 8-column units round robin
                    const int grp = warp >> 2;
                    const uint32_t lane_base = (uint32_t)(32 * (warp & 3)) << 16;
                    const int U = Np / 8;
                    for (int uu = grp; uu < U; uu += kParts) {
                        uint32_t l[kLv][8];
#pragma unroll
                        for (int lv = 0; lv < kLv; ++lv) {
                            if (lv < nlv) {
                                tmem_ld8_nowait(tmem + lane_base + lv * njp + uu * 8, l[lv]);
                            } else {
#pragma unroll
                                for (int c = 0; c < 8; ++c) l[lv][c] = 0u;
                            }
                        }
                        tmem_wait_ld();
#pragma unroll
                        for (int lv = 0; lv < kLv; ++lv) reg_fence8(l[lv]);
#pragma unroll
                        for (int c = 0; c < 8; ++c)
                            if (j0 + uu * 8 + c < n)
                                acc_levels(nrm, __uint_as_float(l[0][c]), __uint_as_float(l[1][c]),
                                           __uint_as_float(l[2][c]), __uint_as_float(l[3][c]),
                                           __uint_as_float(l[4][c]), __uint_as_float(l[5][c]));
                    }
                }
                umma::fence_before_sync();
                __syncthreads();
            }
            if (failed) break;
            // the two column halves of each query -> variance
            {
                const int row = 32 * (warp & 3) + lane, grp = warp >> 2;
                nrm2[grp * kMT + row] = acc_norm(nrm);
                __syncthreads();
                if (tid < kMT) {
                    const int qq = mt * kMT + tid;
                    if (qq < GG) {
                        ff tot = nrm2[tid];
#pragma unroll
                        for (int g = 1; g < kParts; ++g) tot = tot + nrm2[g * kMT + tid];
                        ff var = from_f<ff>(sf2f) - tot;
                        if (!(var.hi > 0.f)) var = zero<ff>();
                        A.var[(int64_t)v * GG + qq] = to_f(var);
                        VAR[qq] = var;  // for the Gaussians (k_init_tc)
                    }
                }
                __syncthreads();
            }
        }
        if (failed) {
            if (tid == 0) s_broken = 1;
            __syncthreads();
            write_failed(A, v, GG, sf2f);
            __syncthreads();
            if (tid == 0) s_item = s_next;
            __syncthreads();
            continue;
        }
        __syncthreads();
        if (tid == 0) s_item = s_next;
        __syncthreads();
    }
    // a pass that gave up may have MMAs in flight: wait for them (bounded) before freeing
    if (s_broken) {
        for (int b = 0; b < 2; ++b)
            if (uses[b] > 0) umma::mbar_wait(&mbar[b], (uses[b] - 1) & 1, kPolls);
    }
    umma::fence_before_sync();
    __syncthreads();
    umma::fence_after_sync();
    if (warp == 0) umma::tmem_free(tmem, 512);
}

// ---- A10: Gaussians of the n_s x n_s subgrids (Eq. 6-8) of the voxels k_var_tc served:
// one warp per voxel, lanes over the Gaussians, the float-float means and variances read
// from the workspace (many warps per SM hide the latency of the small eigenproblems).
__global__ void __launch_bounds__(256) k_init_tc(SolveArgs A)
{
    __shared__ ff nodes[kMaxG];
    const int G = A.G, Gp = A.Gp, GG = G * G, NG = A.n_s * A.n_s;
    if (threadIdx.x < G)
        nodes[threadIdx.x] = from_d<ff>(-0.5 * (double)A.size + ((double)threadIdx.x + 0.5) * (double)A.size / (double)G);
    __syncthreads();
    const int count = A.tc->count;
    const int lane = threadIdx.x & 31;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int it = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; it < count; it += nwarps) {
        const int v = A.tc_v[it];
        if (A.status[v] & VOX_FAILED) continue;  // k_var_tc wrote the prior and default Gaussians
        const int n = (int)(A.offsets[v + 1] - A.offsets[v]);
        const ff* MU = reinterpret_cast<const ff*>(A.tc_ws + A.tc_off[it]) + n * (n + 1) / 2 + n * G + n * Gp;
        const int axis = A.axis[v];
        const float sf2f = A.sf2[v];
        for (int g = lane; g < NG; g += 32) {
            const int64_t o = (int64_t)v * NG + g;
            init_one_gaussian<ff>(MU, MU + GG, nodes, axis, A.centres + 3 * v, A.size, G, A.n_s, A.n_r,
                                  sf2f, A.init_mode, g / A.n_s, g % A.n_s, A.pos + 3 * o, A.scale + 3 * o,
                                  A.quat + 4 * o);
        }
    }
}

}  // namespace

cudaError_t launch_init_tc(const SolveArgs& a, int sms, cudaStream_t s)
{
    k_init_tc<<<sms * 4, 256, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t var_tc_prepare()
{
    return cudaFuncSetAttribute(k_var_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, kVarTcSmem);
}

cudaError_t launch_var_tc(const SolveArgs& a, int sms, cudaStream_t s)
{
    k_var_tc<<<sms, kVT, kVarTcSmem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace gpv
