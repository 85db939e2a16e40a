// gpv_tall.cu -- Voxel-GPR of large voxels (GS-LIVM Sec. 3.1, Alg. 1, Eq. 2-3) as one
// blocked Cholesky of a tall matrix whose trailing updates run on the fifth-generation
// tensor cores (tcgen05) as exact BF16 slice products.
//
// The matrix.  For a voxel of n points (padded to np, a multiple of 32, by identity rows)
// and Q = G^2 query nodes, the rows of
//          M = [ K + D ]   np x np, lower triangle   (Gram + noise, Eq. 2)
//              [ K*^T  ]   Q  x np                    (cross-covariance, Eq. 2)
// are factored through their first np columns: rows 0..np-1 become L (K + D = L L^T) and
// the query rows become V = K*^T L^-T, so that
//          var_q = sf2 - |V_q|^2     and     mu_q = m + V_q . z,   z = L^-1 (f - m)
// (Eq. 3, diagonal of Sigma* only).  Neither L^-1 nor the full Sigma* of the paper's
// Alg. 3 is formed: the explicit inverse is n^3/3 flops the method does not need, which
// at G = 9 is more than the triangular solve it would replace.
//
// The factor (left-looking, panels of 32 columns).  Panel p (columns c0 = 32 p ..
// c0 + 31) of every row r >= c0 is
//          P[r, :] = M[r, panel] - sum_{k < c0} L[r, k] L[panel, k]
// a GEMM of the rows (M tiles of 128) against the panel's own rows (N = 32) over all
// earlier columns, which the tensor cores do; then the 32 x 32 diagonal block is factored
// (128 threads, right-looking, one named barrier per column in float-float and per two
// columns in FP32) and inverted by blocks, every row solves against it (L[r, panel] =
// P[r, :] L_pp^-T as dot products with the block inverse), z is extended, and each query
// row adds its new entries to the running sums |V_q|^2 and V_q . z.  The entries of M
// come from K + D, formed once per voxel, and from the separable node factors of K*.
//
// Precision.  Each finished entry of L and V is cut into NSL slices of 8 bits on a
// power-of-two grid fixed per row by a bound on the row's norm (Gram row r:
// |L_r|^2 = A_rr; query row: |V_q|^2 = sf2 - var_q <= sf2), the scheme of Ozaki, Ogita,
// Oishi and Rump (Numer. Algorithms 59, 2012).  A slice is exactly a BF16 number and a
// product of two slices is exact in FP32.  The products of one level l = s + t share one
// grid, and level l has its own FP32 accumulator in tensor memory: by Cauchy-Schwarz
// over the row norms, level 0 stays below 2^14 grid units and level 1 below 2^20 for any
// K; the levels of remainder slices (products of up to 2^14 units, signs close to
// random) grow like sqrt(K) 2^14 / 3 (2^17.4 at K = 1024, against 2^24 for exactness).
// With six slices levels 4 and 5 share one accumulator: level 5 then rounds to the FP32
// grid of the level-4 sum, an error below 2^-45 of |L_r| |L_c| even when every rounding
// has the same sign, where the float-float working type holds about 2^-44.
// The mixed path uses NSL = 6 (48 bits, 21 products per element); the FP32 path NSL = 4
// (32 bits, 10 products: the fixed-point grid of a row then resolves entries well below
// the row's norm to about FP32's own precision).  Five slices (40 bits) kept the mean and
// variance far inside their tolerances and were 7% faster on the stress workload, but the
// Gaussian scales of the escalation workload's flat voxels (smallest scale near 1e-4 m)
// then moved by 1.8e-4 relative, above the 1e-4 of the initialisation: six it is.  Pairs
// with s + t >= NSL are dropped (below 2^-8 NSL of the row scale).  The diagonal-block
// factor, the solves against it and the running sums are in the working type (float-float
// or FP32) on the CUDA cores.
//
// Organisation.  One persistent CTA per SM (384 threads); one launch drains every size
// bucket above the threshold, largest voxels first.  Per voxel all threads first form
// K + D (stored per panel, column by column) and the separable K* node factors.  Warp 0
// loads operand chunks (one 128 x 32 tile of each A slice, one 32 x 32 tile of each B
// slice, contiguous in the slice store) with cp.async.bulk into a ring of shared-memory
// stages (two of 60 KB in float-float, three of 40 KB in FP32), each completing on an
// mbarrier; one thread of warp 1 issues the MMAs (M = 128, K = 16, kind::f16) of a tile
// into one of three accumulator sets (one 32-column accumulator per level, side by side)
// and commits: per A slice s one MMA takes the B slices of levels s .. nlv-1 side by side
// (N up to 160), the pairs of the shared last accumulator follow one by one (11 MMAs per
// K step in float-float instead of 21, 4 in FP32 instead of 10: the A tile is read from
// shared memory once per slice, not once per pair).  Tile 0 of a panel, whose diagonal
// block every other row waits for, has all but its last chunk accumulated in set 2 during
// the previous panel; the other tiles alternate between sets 0 and 1.  Warps 4..7 and
// 8..11 take the even and odd tiles: they read the levels with tcgen05.ld (lane = row),
// form P in the working type, solve, cut and store the slices.  Every mbarrier wait
// suspends in the barrier between tests and gives up after 2 s; a wait that gives up marks
// the voxel GPV_VOX_FAILED and the CTA stops.
#include <cuda_runtime.h>
#include <stdint.h>

#include "gpv_common.cuh"
#include "gpv_init.cuh"
#include "gpv_internal.h"
#include "gpv_num.cuh"
#include "gpv_umma.cuh"

namespace gpv {
namespace {

constexpr int kT = 384;        // threads per CTA
constexpr int kBP = 32;        // panel width = MMA N
constexpr int kMT = 128;       // rows per M tile
constexpr int kNSt = 3;        // most operand stages of a plan
constexpr uint64_t kWaitNs = 2000000000ull;  // a wait gives up after 2 s
constexpr uint32_t kHintNs = 1000;            // suspend-time hint of one barrier test
constexpr int kSlA = kMT * kBP * 2;  // bytes of one slice of a 128 x 32 A tile
constexpr int kSlB = kBP * kBP * 2;  // bytes of one slice of a 32 x 32 B tile
constexpr int kGrpBytes = 512;       // one 8-row group of a 32-column panel slice

template <int NSL> struct Plan {
    static constexpr int stage = NSL * (kSlA + kSlB);
    // accumulators per set: one per level, except that with six slices levels 4 and 5
    // share the last one
    static constexpr int nlv = NSL == 6 ? 5 : NSL;
    static constexpr int set_cols = nlv * kBP;  // tensor-memory columns of one set
    static constexpr int tmem_cols = 512;       // three sets
    static_assert(3 * set_cols <= tmem_cols, "tensor memory");
    // operand stages: two for float-float (measured faster than three: 1.32 against
    // 1.36 ms per 512-point voxel and SM), three for FP32
    static constexpr int nst = NSL == 6 ? 2 : 3;
    static_assert(nst <= kNSt, "stages");
};

constexpr int kLs = kBP + 1;  // row stride of the diagonal-block buffers (bank spread)

// dynamic shared memory: [stages][x1, x2: np each][Lkk, D: 32 x 33 each][rd, zp: 32]
// [T: 16 x 16, the products of the blocked inverse]
__host__ __device__ inline int tall_smem_bytes(int nsl, int npmax, int tsize)
{
    int o = (nsl == 6 ? 2 : 3) * nsl * (kSlA + kSlB);
    o += 2 * npmax * tsize;
    o += (2 * kBP * kLs + 2 * kBP + 256) * tsize;
    return (o + 15) & ~15;
}

// ---- small PTX wrappers -------------------------------------------------------------
__device__ __forceinline__ void mbar_expect_tx(uint64_t* mbar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                 :: "r"(umma::smem_addr(mbar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// Waits for the phase of the given parity.  Between tests the thread is suspended in the
// barrier (up to kHintNs, or until the phase completes), so waiting warps leave the issue
// slots to the warps that work; false after kWaitNs without completion.
__device__ __forceinline__ bool wait_phase(uint64_t* mbar, uint32_t parity)
{
    const uint32_t a = umma::smem_addr(mbar);
    const uint64_t t0 = global_ns();
    for (;;) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done) : "r"(a), "r"(parity), "r"(kHintNs) : "memory");
        if (done) return true;
        if (global_ns() - t0 > kWaitNs) return false;
    }
}
__device__ __forceinline__ void mbar_arrive(uint64_t* mbar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" :: "r"(umma::smem_addr(mbar)) : "memory");
}
// bulk copy global -> shared, completing bytes on the mbarrier (16-byte aligned, size % 16 == 0)
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* mbar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
        :: "r"(umma::smem_addr(dst)), "l"(src), "r"(bytes), "r"(umma::smem_addr(mbar))
        : "memory");
}
__device__ __forceinline__ void fence_async_global()
{
    asm volatile("fence.proxy.async.global;" ::: "memory");
}
__device__ __forceinline__ void named_sync(int id, int count)
{
    asm volatile("bar.sync %0, %1;" :: "r"(id), "r"(count) : "memory");
}
__device__ __forceinline__ void named_arrive(int id, int count)
{
    asm volatile("bar.arrive %0, %1;" :: "r"(id), "r"(count) : "memory");
}
__device__ __forceinline__ void tmem_ld16_nowait(uint32_t taddr, uint32_t (&r)[16])
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

// x += y (y a float) with an unnormalised float-float accumulator
__device__ __forceinline__ void add_f(float& x, float y) { x = __fadd_rn(x, y); }
__device__ __forceinline__ void add_f(ff& x, float y)
{
    const ff s = two_sum(x.hi, y);
    x.hi = s.hi;
    x.lo = __fadd_rn(x.lo, s.lo);
}
__device__ __forceinline__ int vload(const int& x) { return *(const volatile int*)&x; }
__device__ __forceinline__ void vstore(int& x, int y) { *(volatile int*)&x = y; }

__device__ __forceinline__ float lo_of(float) { return 0.f; }
__device__ __forceinline__ float lo_of(ff x) { return x.lo; }

// Slices of x (|x| < 2^(E-1)) on the grids 2^(E-8), ..., 2^(E-8 NSL): round to the grid by
// adding and subtracting 1.5 * 2^(grid exponent + 23), keep the exact remainder; the low
// part of a float-float value joins the remainder after the third slice (that FP32 sum
// errs by at most 2^(E-49)).  Returns the BF16 bit patterns (upper halves: every slice
// has at most 8 significant bits).
template <int NSL, class T>
__device__ __forceinline__ void cut(T x, int E, uint32_t (&q)[NSL])
{
    float a = hi_of(x);
    const float lo = lo_of(x);
#pragma unroll
    for (int s = 0; s < NSL; ++s) {
        if (s == 3) a = __fadd_rn(a, lo);
        const float sig = __uint_as_float(((uint32_t)(E - 8 * s + 15 + 127) << 23) | 0x400000u);
        const float t = __fsub_rn(__fadd_rn(a, sig), sig);
        a = __fsub_rn(a, t);
        q[s] = __float_as_uint(t) >> 16;
    }
}

// Byte offset of (panel p, slice s, 8-row group g) in the slice store; within it, row
// r % 8 and column c (of the panel) sit at (c / 8) * 128 + (r % 8) * 16 + (c % 8) * 2:
// core matrices of 8 rows x 16 bytes, K-major, so a 16-group A tile and a 4-group B tile
// are contiguous and land in shared memory in the layout the MMA reads (LBO 128, SBO 512).
__device__ __forceinline__ int64_t sl_off(int p, int s, int g, int nsl, int RG)
{
    return ((int64_t)(p * nsl + s) * RG + g) * kGrpBytes;
}

struct Sh {  // static shared state
    uint64_t full[kNSt], empty[kNSt], acc_full[3], acc_empty[3];
    uint32_t tmem;
    int v, abort, broken, fail;
    float dmin, dmax;
    int axis;
};

}  // namespace

// Entries of K + D kept per panel: rows c0 .. np-1 of panel p, 32 values each, column by
// column (entry (r, c0 + j) at j (np - c0) + r - c0), so that a warp reading one column for
// 32 consecutive rows reads contiguous memory.
__host__ __device__ inline int64_t tall_gram_off(int p, int np)
{
    return (int64_t)kBP * ((int64_t)p * np - (int64_t)kBP * p * (p - 1) / 2);
}
__host__ __device__ inline int64_t tall_gram_elems(int np) { return tall_gram_off(np / kBP, np); }

// Workspace of one CTA: slice store, per-row running sums, node factors, K + D.
__host__ __device__ inline int tall_np(int n) { return (n + kBP - 1) / kBP * kBP; }
__host__ __device__ inline int tall_rg(int np, int Q) { return (np + Q + kMT + 7) / 8; }
__host__ __device__ inline int64_t tall_ws_bytes(int nsl, int nmax, int G, int tsize)
{
    const int np = tall_np(nmax), Q = G * G;
    const int64_t sl = (int64_t)(np / kBP) * nsl * tall_rg(np, Q) * kGrpBytes;
    const int64_t rs = (int64_t)2 * (np + Q) * tsize;   // running sums w, s2 per row
    const int64_t ab = (int64_t)2 * np * G * tsize;     // node factors a(u), b(v)
    const int64_t gr = tall_gram_elems(np) * tsize;     // K + D, panel by panel
    const int64_t yE = (int64_t)np * (tsize + 4);       // targets f - m, row exponents
    return (sl + rs + ab + gr + yE + 255) & ~(int64_t)255;
}

namespace {

template <class T, int NSL>
__global__ void __launch_bounds__(kT, 1) k_tall(SolveArgs A, unsigned char* ws, int64_t ws_stride,
                                                int npmax)
{
    extern __shared__ __align__(128) unsigned char sm[];
    __shared__ Sh sh;
    __shared__ double red[6 * 32];
    __shared__ T nodes[kMaxG];
    __shared__ ff xtab[is_ff<T>::value ? 256 : 1];
    using P = Plan<NSL>;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int G = A.G, Q = G * G;
    unsigned char* wsb = ws + (int64_t)blockIdx.x * ws_stride;

    T* x1 = reinterpret_cast<T*>(sm + P::nst * P::stage);
    T* x2 = x1 + npmax;
    T* Lkk = x2 + npmax;       // L of the diagonal block, 32 x 33, row-major
    T* Dm = Lkk + kBP * kLs;   // its inverse (lower triangle, zeros above)
    T* rd = Dm + kBP * kLs;    // 1 / L_jj
    T* zp = rd + kBP;          // z of the panel
    T* Tb = zp + kBP;          // 16 x 16 products of the blocked inverse

    // entries (i, m), m <= i, of the diagonal block's trailing triangles in the order
    // e = w (w + 1) / 2 + u, w = 31 - m, u = 31 - i: the update of step k is the prefix
    // e < (31 - k)(32 - k) / 2, so a thread keeps the entries e = ri + 128 c at every step
    __shared__ uint16_t tri[kBP * (kBP - 1) / 2];
    for (int e = tid; e < kBP * (kBP - 1) / 2; e += kT) {
        int w = (int)((sqrtf(8.f * (float)e + 1.f) - 1.f) * 0.5f);
        while ((w + 1) * (w + 2) / 2 <= e) ++w;
        while (w * (w + 1) / 2 > e) --w;
        const int u = e - w * (w + 1) / 2;
        tri[e] = (uint16_t)(((kBP - 1 - u) << 8) | (kBP - 1 - w));
    }

    if (threadIdx.x < G)
        nodes[threadIdx.x] = from_d<T>(-0.5 * (double)A.size +
                                       ((double)threadIdx.x + 0.5) * (double)A.size / (double)G);
    if (is_ff<T>::value)
        for (int i = tid; i < 256; i += kT) {
            const double t = exp2((double)i / 256.0);
            const float h = (float)t;
            xtab[i] = ff_make(h, (float)(t - (double)h));
        }
    if (tid == 0) {
        for (int i = 0; i < P::nst; ++i) { umma::mbar_init(&sh.full[i], 1); umma::mbar_init(&sh.empty[i], 1); }
        for (int i = 0; i < 3; ++i) { umma::mbar_init(&sh.acc_full[i], 1); umma::mbar_init(&sh.acc_empty[i], 4); }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        sh.broken = 0;
    }
    if (warp == 2) umma::tmem_alloc(&sh.tmem, P::tmem_cols);
    umma::fence_before_sync();
    __syncthreads();
    umma::fence_after_sync();
    const uint32_t tmem = sh.tmem;

    // pipeline counters (each role keeps its own copy of the common schedule)
    uint32_t cnt = 0;               // operand chunks (producer, MMA issuer)
    uint32_t use[3] = {0, 0, 0};    // completed tiles per accumulator set (MMA issuer, epilogue)
    const uint32_t idesc = umma::idesc_bf16(kMT, kBP);

    int q = (A.nqueues > 1 ? A.nqueues : 1) - 1;  // queue being drained (largest voxels first)
    for (;;) {
        if (tid == 0) {
            int vv = -1;
            for (; q >= 0; --q) {
                const int i = atomicAdd(A.work_next + q, 1);
                if (i < A.work_count[q]) {
                    vv = A.work[(A.work_base ? A.work_base[q] : 0) + i];
                    break;
                }
            }
            sh.v = vv;
            sh.abort = 0;
            sh.fail = 0;
            sh.dmin = 3.0e38f;
            sh.dmax = 0.f;
        }
        __syncthreads();
        const int v = sh.v;
        if (v < 0 || vload(sh.broken)) break;

        // ---- A1/A2: points, value axis, local inputs and targets (all threads) ----------
        const int64_t beg = A.offsets[v];
        const int n = (int)(A.offsets[v + 1] - beg);
        const int np = tall_np(n), NP = np / kBP, R = np + Q, RG = tall_rg(np, Q);
        const float* src = A.xyz + 3 * beg;
        const float cx = A.centres[3 * v + 0], cy = A.centres[3 * v + 1], cz = A.centres[3 * v + 2];
        {
            float* redf = reinterpret_cast<float*>(red);
            float s3[3] = {0.f, 0.f, 0.f};
            for (int i = tid; i < n; i += kT) {
                s3[0] += __ldg(src + 3 * i) - cx;
                s3[1] += __ldg(src + 3 * i + 1) - cy;
                s3[2] += __ldg(src + 3 * i + 2) - cz;
            }
            block_sum<float, 3>(s3, redf);
            const float inv_n = 1.f / (float)n;
            const float m0 = s3[0] * inv_n, m1 = s3[1] * inv_n, m2 = s3[2] * inv_n;
            float c6[6] = {0, 0, 0, 0, 0, 0};
            for (int i = tid; i < n; i += kT) {
                const float d0 = (__ldg(src + 3 * i) - cx) - m0;
                const float d1 = (__ldg(src + 3 * i + 1) - cy) - m1;
                const float d2 = (__ldg(src + 3 * i + 2) - cz) - m2;
                c6[0] += d0 * d0; c6[1] += d0 * d1; c6[2] += d0 * d2;
                c6[3] += d1 * d1; c6[4] += d1 * d2; c6[5] += d2 * d2;
            }
            block_sum<float, 6>(c6, redf);
            if (tid == 0) sh.axis = value_axis_from_cov(c6);
            __syncthreads();
        }
        const int axis = sh.axis;
        const int pa1 = axis == 2 ? 0 : axis + 1;
        const int pa2 = axis == 0 ? 2 : (axis == 1 ? 0 : 1);
        const float cen[3] = {cx, cy, cz};
        const float lamf = A.lam[v], sf2f = A.sf2[v], sn2f = A.sn2[v];
        // global part of the workspace: slices, running sums (w: the partial products
        // L z of Gram rows and V . z of query rows; s2: |V_q|^2), the node factors
        // a_i(u) = sf2 exp(-lambda (x_i - u)^2), b_i(v) = exp(-lambda (y_i - v)^2), K + D by
        // panels, the targets f - m and the row exponents
        unsigned char* sl = wsb;
        T* rs = reinterpret_cast<T*>(wsb + (int64_t)NP * NSL * RG * kGrpBytes);
        T* fa = rs + 2 * (int64_t)R;
        T* fb = fa + (int64_t)np * G;
        T* gram = fb + (int64_t)np * G;
        T* yv = gram + tall_gram_elems(np);
        int* Eg = reinterpret_cast<int*>(yv + np);
        const T nlam = from_f<T>(-lamf), sf2 = from_f<T>(sf2f);
        T msum[1] = {zero<T>()};
        float nmin = 3.0e38f;
        for (int i = tid; i < np; i += kT) {
            if (i < n) {
                x1[i] = diff_f<T>(__ldg(src + 3 * i + pa1), cen[pa1]);
                x2[i] = diff_f<T>(__ldg(src + 3 * i + pa2), cen[pa2]);
                const T f = diff_f<T>(__ldg(src + 3 * i + axis), cen[axis]);
                yv[i] = f;
                msum[0] = msum[0] + f;
                const float d = A.noise ? __ldg(A.noise + beg + i) : sn2f;
                Eg[i] = tc_exp_above(sqrtf(sf2f + d));
            } else {  // identity padding rows
                x1[i] = zero<T>();
                x2[i] = zero<T>();
                yv[i] = zero<T>();
                Eg[i] = tc_exp_above(1.f);
            }
        }
        block_sum<T, 1>(msum, reinterpret_cast<T*>(red));
        const T m = A.mean_mode == 1 ? msum[0] / from_f<T>((float)n) : zero<T>();
        for (int i = tid; i < n; i += kT) yv[i] = yv[i] - m;
        const int EV = tc_exp_above(sqrtf(sf2f));
        (void)nmin;
        for (int i = tid; i < 2 * R; i += kT) rs[i] = zero<T>();
        __syncthreads();
        for (int t = tid; t < np * G; t += kT) {
            const int i = t / G, u = t - i * G;
            if (i < n) {
                const T da = x1[i] - nodes[u], db = x2[i] - nodes[u];
                fa[t] = sf2 * gexpw(nlam * (da * da), xtab);
                fb[t] = gexpw(nlam * (db * db), xtab);
            } else {
                fa[t] = zero<T>();
                fb[t] = zero<T>();
            }
        }
        // A3: K + D (lower triangle; identity on the padding), stored panel by panel and
        // column by column within a panel
        for (int pp = 0; pp < NP; ++pp) {
            const int cc0 = pp * kBP, rows = np - cc0;
            T* gp = gram + tall_gram_off(pp, np);
            for (int e = tid; e < rows * kBP; e += kT) {
                const int jc = e / rows;
                const int r = cc0 + (e - jc * rows), c = cc0 + jc;
                T o;
                if (c > r) o = zero<T>();
                else if (r >= n || c >= n) o = from_f<T>(r == c ? 1.f : 0.f);
                else {
                    const T d1 = x1[r] - x1[c], d2 = x2[r] - x2[c];
                    o = sf2 * gexpw(nlam * (d1 * d1 + d2 * d2), xtab);
                    if (r == c) o = o + from_f<T>(A.noise ? __ldg(A.noise + beg + r) : sn2f);
                }
                gp[e] = o;
            }
        }
        __syncthreads();

        // ---- A3-A8: panels ------------------------------------------------------------
        for (int p = 0; p < NP; ++p) {
            const int c0 = p * kBP;
            const int T_ = (R - c0 + kMT - 1) / kMT;  // M tiles of this panel
            // Work of the tensor cores in this panel, in order (items it = 0 .. T_):
            //   it = 0       tile 0, chunk p - 1 only: chunks 0 .. p-2 were accumulated into
            //                set 2 during the previous panel (its diagonal block is the
            //                critical path of the panel, so only one chunk waits for it);
            //   1 <= it < T_ tile it, chunks 0 .. p-1, into set it & 1;
            //   it = T_      tile 0 of the next panel (rows c0 + 32 ..), chunks 0 .. p-1,
            //                into set 2, once this panel's tile 0 has been read.
            const int nch = (p > 0 ? 1 : 0) + (T_ - 1) * p + (p + 1 < NP ? p : 0);
            if (warp == 0 && nch > 0) {
                // producer
                if (lane == 0) {
                    uint32_t c2 = cnt;
                    for (int it = 0; it <= T_; ++it) {
                        int ga = (c0 + kMT * it) >> 3, gb = c0 >> 3, j0 = 0;
                        if (it == 0) j0 = p - 1;
                        else if (it == T_) ga = gb = (c0 + kBP) >> 3;
                        if (it == T_ && p + 1 >= NP) break;
                        for (int j = max(j0, 0); j < p; ++j, ++c2) {
                            const int st = c2 % P::nst;
                            const uint32_t rnd = c2 / P::nst;
                            if (rnd > 0 && !vload(sh.broken) &&
                                !wait_phase(&sh.empty[st], (rnd - 1) & 1))
                                vstore(sh.broken, 1);
                            if (vload(sh.broken)) continue;
                            unsigned char* dst = sm + st * P::stage;
                            mbar_expect_tx(&sh.full[st], P::stage);
#pragma unroll
                            for (int s = 0; s < NSL; ++s) {
                                bulk_g2s(dst + s * kSlA, sl + sl_off(j, s, ga, NSL, RG), kSlA, &sh.full[st]);
                                bulk_g2s(dst + NSL * kSlA + s * kSlB, sl + sl_off(j, s, gb, NSL, RG),
                                         kSlB, &sh.full[st]);
                            }
                        }
                    }
                }
                __syncwarp();
                cnt += (uint32_t)nch;
            } else if (warp == 1 && nch > 0) {
                // MMA issuer
                if (lane == 0) {
                    uint32_t c2 = cnt;
                    for (int it = 0; it <= T_; ++it) {
                        if (it == T_ && p + 1 >= NP) break;
                        const int set = (it == 0 || it == T_) ? 2 : (it & 1);
                        const int j0 = it == 0 ? p - 1 : 0;
                        if (j0 < 0 || j0 >= p) continue;  // nothing to multiply (panel 0)
                        // a fresh accumulation waits until the set's last tile was read
                        const bool fresh = it != 0 || p == 1;
                        if (it != 0 && use[set] > 0 && !vload(sh.broken) &&
                            !wait_phase(&sh.acc_empty[set], (use[set] - 1) & 1))
                            vstore(sh.broken, 1);
                        umma::fence_after_sync();
                        const uint32_t dacc = tmem + set * P::set_cols;
                        for (int j = j0; j < p; ++j, ++c2) {
                            const int st = c2 % P::nst;
                            if (!vload(sh.broken) && !wait_phase(&sh.full[st], (c2 / P::nst) & 1))
                                vstore(sh.broken, 1);
                            umma::fence_after_sync();
                            if (!vload(sh.broken)) {
                                const uint32_t a0 = umma::smem_addr(sm + st * P::stage);
                                const uint32_t b0 = a0 + NSL * kSlA;
                                const bool first = fresh && j == j0;
                                // per A slice s one MMA over the B slices 0 .. nlv-1-s side by
                                // side (N = (nlv - s) 32; they are contiguous in the stage with
                                // the 8-row-group stride of one slice), writing the levels
                                // s .. nlv-1, which lie side by side in tensor memory; the pairs
                                // of the shared last accumulator (s + s2 >= nlv) one by one
#pragma unroll
                                for (int ks = 0; ks < 2; ++ks)
#pragma unroll
                                    for (int s = 0; s < NSL; ++s) {
                                        const uint64_t ad = umma::make_desc(a0 + s * kSlA + ks * 256, 128, 512);
                                        if (s < P::nlv) {
                                            const uint64_t bd = umma::make_desc(b0 + ks * 256, 128, 512);
                                            umma::mma_bf16(dacc + s * kBP, ad, bd,
                                                           umma::idesc_bf16(kMT, (P::nlv - s) * kBP),
                                                           !(first && ks == 0 && s == 0));
                                        }
#pragma unroll
                                        for (int s2 = (P::nlv - s > 0 ? P::nlv - s : 0); s2 < NSL - s; ++s2) {
                                            const uint64_t bd = umma::make_desc(b0 + s2 * kSlB + ks * 256, 128, 512);
                                            umma::mma_bf16(dacc + (P::nlv - 1) * kBP, ad, bd, idesc, true);
                                        }
                                    }
                            }
                            umma::mma_commit(&sh.empty[st]);
                        }
                        if (it < T_) {  // the tile is complete: hand it to its epilogue group
                            umma::mma_commit(&sh.acc_full[set]);
                            ++use[set];
                        }
                    }
                }
                __syncwarp();
                cnt += (uint32_t)nch;
            } else if (warp >= 4) {
                // epilogue groups: warps 4..7 take the even tiles, 8..11 the odd ones
                const int grp = (warp - 4) >> 2, qd = warp & 3;
                const int ri = 32 * qd + lane;  // row within the tile = tensor-memory lane
                for (int t = grp; t < T_; t += 2) {
                    const int r = c0 + kMT * t + ri;
                    const bool valid = r < R;
                    T row[kBP];
                    // P = M[r, panel] - sum_{k < c0} L[r, k] L[panel, k]
                    const int Er = valid ? (r < np ? Eg[r] : EV) : 0;
                    if (p > 0) {
                        const int set = t == 0 ? 2 : (t & 1);
                        if (!vload(sh.broken) && !wait_phase(&sh.acc_full[set], use[set] & 1))
                            vstore(sh.broken, 1);
                        umma::fence_after_sync();
                        const uint32_t tb = tmem + ((uint32_t)(32 * qd) << 16) + set * P::set_cols;
                        // the levels hold the products' values (the slices keep their
                        // magnitudes); summed into the working type, largest level first
#pragma unroll
                        for (int h = 0; h < 2; ++h) {
                            {
                                uint32_t lv[16];
                                tmem_ld16_nowait(tb + 16 * h, lv);
                                tmem_wait_ld();
#pragma unroll
                                for (int jj = 0; jj < 16; ++jj) row[16 * h + jj] = from_f<T>(__uint_as_float(lv[jj]));
                            }
                            // the later levels in a rolled loop: the epilogue's instruction
                            // footprint, not its operation count, bounds it (measured 4% faster
                            // on the stress workload than the unrolled loop)
#pragma unroll 1
                            for (int l = 1; l < P::nlv; ++l) {
                                uint32_t lv[16];
                                tmem_ld16_nowait(tb + l * kBP + 16 * h, lv);
                                tmem_wait_ld();
#pragma unroll
                                for (int jj = 0; jj < 16; ++jj) add_f(row[16 * h + jj], __uint_as_float(lv[jj]));
                            }
                        }
                        umma::fence_before_sync();
                        __syncwarp();
                        if (lane == 0) mbar_arrive(&sh.acc_empty[set]);
                        ++use[set];
                    } else {
#pragma unroll
                        for (int j = 0; j < kBP; ++j) row[j] = zero<T>();
                    }
                    if (valid) {  // P = M[r, panel] - (the products of the earlier columns)
                        if (r < np) {
                            const T* gp = gram + tall_gram_off(p, np) + (r - c0);
                            const int64_t rows = np - c0;
#pragma unroll
                            for (int j = 0; j < kBP; ++j) row[j] = gp[j * rows] - row[j];
                        } else {  // cross-covariance of query q = (u, v)
                            const int q = r - np, uu = q / G, vv = q - uu * G;
#pragma unroll
                            for (int j = 0; j < kBP; ++j)
                                row[j] = fa[(int64_t)(c0 + j) * G + uu] * fb[(int64_t)(c0 + j) * G + vv] - row[j];
                        }
                    }
                    const bool diag = t == 0 && qd == 0;  // warp 4: the rows of the diagonal block
                    if (t == 0) {
                        // ---- group A (128 threads): factor the diagonal block, invert it, z of
                        // the panel; warp 4 holds its rows -------------------------------------
                        if (diag) {
#pragma unroll
                            for (int j = 0; j < kBP; ++j) Lkk[lane * kLs + j] = row[j];
                            zp[lane] = yv[c0 + lane] - rs[2 * (c0 + lane)];
                        }
                        named_sync(1, 128);
                        float dmn = 3.0e38f, dmx = 0.f;
                        int bad = 0;
                        // FP32 is bound by the barriers of the column steps: two columns per
                        // step; float-float by the arithmetic's latency: one (measured: FP32
                        // 0.52 against 0.54 ms per 512-point voxel and SM with two; float-float
                        // 3-6% slower with two)
                        if constexpr (sizeof(T) == 4) {
                            // right-looking, two columns and one barrier per step: step k forms the
                            // 2 x 2 pivot block of columns k, k+1 (every thread, redundantly), scales
                            // columns k-2, k-1 (their readers are past the barrier) and updates the
                            // trailing triangle by both columns, in the order and roundings of two
                            // one-column steps: L_ik = A_ik / L_kk, L_i,k+1 = (A_i,k+1 - L_ik L_k+1,k)
                            // / L_k+1,k+1, A_im -= L_ik L_mk, then A_im -= L_i,k+1 L_m,k+1.  As in
                            // the float-float factor below, a thread's trailing entries stay in
                            // registers; an entry goes to shared memory after its last update,
                            // the step before its column is one of the pivot pair (m = k + 2 or
                            // k + 3; measured 2% faster on the FP32 stress workload)
                            int eim[4];
                            T xr[4];
#pragma unroll
                            for (int c = 0; c < 4; ++c) {
                                const int e = ri + 128 * c;
                                eim[c] = e < kBP * (kBP - 1) / 2 ? (int)tri[e] : 0;
                                xr[c] = Lkk[(eim[c] >> 8) * kLs + (eim[c] & 255)];
                            }
                            T d0p = zero<T>(), d1p = zero<T>(), il0p = zero<T>(), il1p = zero<T>(), l10p = zero<T>();
                            for (int k = 0; k < kBP; k += 2) {
                                const T d0 = Lkk[k * kLs + k];
                                const T il0 = grsqrt(d0);  // 1 / L_kk
                                const T l10 = Lkk[(k + 1) * kLs + k] * il0;
                                const T d1 = gfnma(l10, l10, Lkk[(k + 1) * kLs + k + 1]);
                                const T il1 = grsqrt(d1);  // 1 / L_k+1,k+1
                                if (ri == 0) {
    #pragma unroll
                                    for (int u = 0; u < 2; ++u) {
                                        if (c0 + k + u < n) {
                                            const float dh = hi_of(u ? d1 : d0);
                                            if (!(dh > 0.f)) bad = 1;
                                            dmn = fminf(dmn, dh);
                                            dmx = fmaxf(dmx, dh);
                                        }
                                    }
                                }
                                if (k > 0) {
                                    if (ri >= k && ri < kBP) {
                                        const T li0 = Lkk[ri * kLs + k - 2] * il0p;
                                        const T a1 = Lkk[ri * kLs + k - 1];
                                        Lkk[ri * kLs + k - 2] = li0;
                                        Lkk[ri * kLs + k - 1] = gfnma(li0, l10p, a1) * il1p;
                                    } else if (ri == k - 2) {
                                        Lkk[(k - 2) * kLs + k - 2] = d0p * il0p;
                                        Lkk[(k - 1) * kLs + k - 2] = l10p;
                                        Lkk[(k - 1) * kLs + k - 1] = d1p * il1p;
                                        rd[k - 2] = il0p;
                                        rd[k - 1] = il1p;
                                    }
                                }
                                const int sz = kBP - 2 - k, cntk = sz * (sz + 1) / 2;  // entries, m >= k + 2
#pragma unroll
                                for (int c = 0; c < 4; ++c) {
                                    const int i = eim[c] >> 8, m = eim[c] & 255;
                                    const T li0 = Lkk[i * kLs + k] * il0, lm0 = Lkk[m * kLs + k] * il0;
                                    const T li1 = gfnma(li0, l10, Lkk[i * kLs + k + 1]) * il1;
                                    const T lm1 = gfnma(lm0, l10, Lkk[m * kLs + k + 1]) * il1;
                                    const T nx = gfnma(li1, lm1, gfnma(li0, lm0, xr[c]));
                                    xr[c] = ri + 128 * c < cntk ? nx : xr[c];
                                }
#pragma unroll
                                for (int c = 0; c < 4; ++c) {
                                    const int m = eim[c] & 255;
                                    if (ri + 128 * c < cntk && (m == k + 2 || m == k + 3))
                                        Lkk[(eim[c] >> 8) * kLs + m] = xr[c];
                                }
                                d0p = d0;
                                d1p = d1;
                                il0p = il0;
                                il1p = il1;
                                l10p = l10;
                                named_sync(1, 128);
                            }
                            if (ri == kBP - 2) {  // the last pivot block
                                Lkk[(kBP - 2) * kLs + kBP - 2] = d0p * il0p;
                                Lkk[(kBP - 1) * kLs + kBP - 2] = l10p;
                                Lkk[(kBP - 1) * kLs + kBP - 1] = d1p * il1p;
                                rd[kBP - 2] = il0p;
                                rd[kBP - 1] = il1p;
                            }
                            named_sync(1, 128);
                        } else {
                            // right-looking, one column and one barrier per step: step k scales
                            // column k - 1 (its readers are past the barrier) and updates the
                            // trailing triangle with L_ik L_mk = (A_ik / L_kk)(A_mk / L_kk).  A
                            // thread's trailing entries (e = ri + 128 c, the same at every step)
                            // stay in registers; an entry is stored to shared memory after its
                            // last update (step m - 1), where the next step reads it as part of
                            // its column (measured 2.5% faster on the stress workload than
                            // updating the entries in shared memory)
                            int eim[4];
                            T xr[4];
#pragma unroll
                            for (int c = 0; c < 4; ++c) {
                                const int e = ri + 128 * c;
                                eim[c] = e < kBP * (kBP - 1) / 2 ? (int)tri[e] : 0;
                                xr[c] = Lkk[(eim[c] >> 8) * kLs + (eim[c] & 255)];
                            }
                            T dprev = zero<T>(), ilprev = zero<T>();
                            for (int k = 0; k < kBP; ++k) {
                                const T d = Lkk[k * kLs + k];
                                if (ri == 0 && c0 + k < n) {
                                    const float dh = hi_of(d);
                                    if (!(dh > 0.f)) bad = 1;
                                    dmn = fminf(dmn, dh);
                                    dmx = fmaxf(dmx, dh);
                                }
                                const T il = grsqrt(d);  // 1 / L_kk
                                if (k > 0) {
                                    if (ri >= k && ri < kBP) Lkk[ri * kLs + k - 1] = Lkk[ri * kLs + k - 1] * ilprev;
                                    else if (ri == k - 1) { Lkk[(k - 1) * kLs + k - 1] = dprev * ilprev; rd[k - 1] = ilprev; }
                                }
                                const int sz = kBP - 1 - k, cntk = sz * (sz + 1) / 2;
                                // all four updates without branches (a select keeps the entries
                                // already final), so their dependency chains interleave
#pragma unroll
                                for (int c = 0; c < 4; ++c) {
                                    const int i = eim[c] >> 8, m = eim[c] & 255;
                                    const T nx = gfnma(Lkk[i * kLs + k] * il, Lkk[m * kLs + k] * il, xr[c]);
                                    xr[c] = ri + 128 * c < cntk ? nx : xr[c];
                                }
#pragma unroll
                                for (int c = 0; c < 4; ++c)
                                    if (ri + 128 * c < cntk && (eim[c] & 255) == k + 1)
                                        Lkk[(eim[c] >> 8) * kLs + k + 1] = xr[c];
                                dprev = d;
                                ilprev = il;
                                named_sync(1, 128);
                            }
                            if (ri == kBP - 1) { Lkk[(kBP - 1) * kLs + kBP - 1] = dprev * ilprev; rd[kBP - 1] = ilprev; }
                            named_sync(1, 128);
                        }
                        // D = L_pp^-1 by blocks: the eight 4 x 4 diagonal blocks directly, then
                        // three levels D21 = -D22 (L21 D11) doubling the block size; zeros above
                        for (int e = ri; e < kBP * kBP; e += 128) {
                            const int i = e >> 5, j = e & 31;
                            if (j > i || (i >> 2) != (j >> 2)) Dm[i * kLs + j] = zero<T>();
                        }
                        if (ri < 8) {
                            const int o = 4 * ri;
                            for (int j = 0; j < 4; ++j) {
                                Dm[(o + j) * kLs + o + j] = rd[o + j];
                                for (int i = j + 1; i < 4; ++i) {
                                    T acc = zero<T>();
                                    for (int k = j; k < i; ++k)
                                        acc_fma(acc, Lkk[(o + i) * kLs + o + k], Dm[(o + k) * kLs + o + j]);
                                    Dm[(o + i) * kLs + o + j] = -(acc_norm(acc) * rd[o + i]);
                                }
                            }
                        }
                        named_sync(1, 128);
                        for (int h = 4; h < kBP; h *= 2) {
                            const int E = (kBP / (2 * h)) * h * h;
                            for (int e = ri; e < E; e += 128) {  // T = L21 D11
                                const int bb = e / (h * h), i = (e / h) % h, j = e % h, o = 2 * h * bb;
                                T acc = zero<T>();
                                for (int k = j; k < h; ++k)
                                    acc_fma(acc, Lkk[(o + h + i) * kLs + o + k], Dm[(o + k) * kLs + o + j]);
                                Tb[e] = acc_norm(acc);
                            }
                            named_sync(1, 128);
                            for (int e = ri; e < E; e += 128) {  // D21 = -D22 T
                                const int bb = e / (h * h), i = (e / h) % h, j = e % h, o = 2 * h * bb;
                                T acc = zero<T>();
                                for (int k = 0; k <= i; ++k)
                                    acc_fma(acc, Dm[(o + h + i) * kLs + o + h + k], Tb[bb * h * h + k * h + j]);
                                Dm[(o + h + i) * kLs + o + j] = -acc_norm(acc);
                            }
                            named_sync(1, 128);
                        }
                        // z_p = D (y_p - w_p)
                        T zl = zero<T>();
                        if (ri < kBP)
                            for (int k = 0; k <= ri; ++k) acc_fma(zl, Dm[ri * kLs + k], zp[k]);
                        named_sync(1, 128);
                        if (ri < kBP) zp[ri] = acc_norm(zl);
                        if (ri == 0) {
                            if (bad) sh.fail = 1;
                            sh.dmin = fminf(sh.dmin, dmn);
                            sh.dmax = fmaxf(sh.dmax, dmx);
                        }
                        __threadfence_block();
                        named_sync(1, 128);
                        if (diag && T_ > 1) named_arrive(2, 160);  // the odd tiles' group may go on
                    } else if (t == 1) {
                        named_sync(2, 160);
                    }
                    // ---- L[r, panel] = P[r, :] D^T (the diagonal rows take L_pp itself), the
                    // running sums, the slices: two columns per step ------------------------
                    if (valid) {
                        T w = rs[2 * (int64_t)r], s2 = rs[2 * (int64_t)r + 1];
                        const bool qrow = r >= np;
                        const int g = r >> 3;
                        unsigned char* base = sl + sl_off(p, 0, g, NSL, RG) + (r & 7) * 16;
                        const int64_t sstride = (int64_t)RG * kGrpBytes;  // next slice
                        // D is lower triangular: the dot products of columns j, j + 1 stop at
                        // column j + 1.  Float-float: one rolled loop over the column pairs,
                        // the dot products unrolled over all 32 columns and left at j + 1
                        // (the exact triangle with the smallest instruction footprint; 12%
                        // faster on the stress workload than blocks of 8 columns, each
                        // unrolled to its block's end).  FP32: blocks of 8 columns, each dot
                        // product unrolled to its block's last column (the exit test costs
                        // more than the single FMAs it saves).
                        constexpr int kRB = is_ff<T>::value ? kBP : 8;
#pragma unroll
                        for (int jb = 0; jb < kBP / kRB; ++jb) {
                            for (int j = kRB * jb; j < kRB * jb + kRB; j += 2) {
                                T l0, l1;
                                if (diag) {
                                    l0 = j <= lane ? Lkk[lane * kLs + j] : zero<T>();
                                    l1 = j + 1 <= lane ? Lkk[lane * kLs + j + 1] : zero<T>();
                                } else {
                                    T a0 = zero<T>(), a1 = zero<T>();
                                    const T* d0 = Dm + j * kLs;
                                    const T* d1 = d0 + kLs;
#pragma unroll
                                    for (int k = 0; k < kRB * jb + kRB; ++k) {
                                        if (is_ff<T>::value && k > j + 1) break;
                                        acc_fma(a0, row[k], d0[k]);
                                        acc_fma(a1, row[k], d1[k]);
                                    }
                                    l0 = acc_norm(a0);
                                    l1 = acc_norm(a1);
                                    acc_fma(w, l0, zp[j]);
                                    acc_fma(w, l1, zp[j + 1]);
                                    if (qrow) {
                                        acc_fma(s2, l0, l0);
                                        acc_fma(s2, l1, l1);
                                    }
                                }
                                uint32_t qa[NSL], qb[NSL];
                                cut<NSL, T>(l0, Er, qa);
                                cut<NSL, T>(l1, Er, qb);
                                unsigned char* o = base + (j >> 3) * 128 + (j & 7) * 2;
#pragma unroll
                                for (int ss = 0; ss < NSL; ++ss)
                                    *reinterpret_cast<uint32_t*>(o + ss * sstride) = qa[ss] | (qb[ss] << 16);
                            }
                        }
                        if (!diag) {
                            rs[2 * (int64_t)r] = acc_norm(w);
                            rs[2 * (int64_t)r + 1] = acc_norm(s2);
                        }
                    }
                    fence_async_global();
                }
            }
            __syncthreads();
            // conditioning check of the mixed path after each panel's pivots
            if (tid == 0 && !sh.abort) {
                const bool ill = sh.fail || (sh.dmax > A.esc_cond * sh.dmin);
                if (ill && A.escalate) sh.abort = 1;
                else if (sh.fail || (sizeof(T) == 4 && !A.escalate && ill)) sh.abort = 2;  // FP32: as above
                if (vload(sh.broken)) sh.abort = 3;
            }
            __syncthreads();
            if (sh.abort) break;
        }

        // ---- outputs ------------------------------------------------------------------
        const int64_t obase = (int64_t)v * Q;
        const int ab = sh.abort;
        if (ab == 1) {  // badly conditioned: the FP64 pass re-solves the voxel
            if (tid == 0) {
                const int big = n > A.nmax_small_f64 ? 1 : 0;
                const int slot = atomicAdd(A.esc_count + big, 1);
                A.esc_list[(int64_t)big * A.nvox + slot] = v;
            }
        } else if (ab >= 2) {  // not positive definite in this precision, or a wait gave up
            for (int q = tid; q < Q; q += kT) {
                A.mean[obase + q] = to_f(m);
                A.var[obase + q] = sf2f;
            }
            if (A.pos) {
                const int NG = A.n_s * A.n_s;
                for (int g = tid; g < NG; g += kT) {
                    const int64_t o = (int64_t)v * NG + g;
                    for (int k = 0; k < 3; ++k) { A.pos[3 * o + k] = cen[k]; A.scale[3 * o + k] = 0.f; }
                    A.quat[4 * o] = 1.f; A.quat[4 * o + 1] = 0.f; A.quat[4 * o + 2] = 0.f; A.quat[4 * o + 3] = 0.f;
                }
            }
            if (tid == 0) {
                A.axis[v] = (uint8_t)axis;
                A.status[v] = (ab == 3 ? VOX_FAILED : VOX_NOT_SPD) | (A.escalation_pass ? VOX_ESCALATED : 0u);
            }
        } else {
            // mu_q = m + V_q . z, var_q = sf2 - |V_q|^2; predictions staged for the init
            T* mv = reinterpret_cast<T*>(sm);  // the operand stages are idle now
            for (int q = tid; q < Q; q += kT) {
                const T mu = m + rs[2 * (int64_t)(np + q)];
                T var = sf2 - rs[2 * (int64_t)(np + q) + 1];
                if (!(hi_of(var) > 0.f)) var = zero<T>();
                A.mean[obase + q] = to_f(mu);
                A.var[obase + q] = to_f(var);
                mv[q] = mu;
                mv[Q + q] = var;
            }
            if (tid == 0) {
                A.axis[v] = (uint8_t)axis;
                A.status[v] = A.escalation_pass ? VOX_ESCALATED : 0u;
            }
            if (A.pos) {
                __syncthreads();
                const int NG = A.n_s * A.n_s;
                for (int g = tid; g < NG; g += kT) {
                    const int64_t o = (int64_t)v * NG + g;
                    init_one_gaussian<T>(mv, mv + Q, nodes, axis, cen, A.size, G, A.n_s, A.n_r, sf2f,
                                         A.init_mode, g / A.n_s, g % A.n_s, A.pos + 3 * o,
                                         A.scale + 3 * o, A.quat + 4 * o);
                }
            }
        }
        __syncthreads();
    }
    // every MMA this CTA issued has completed (each tile's epilogue waited for it)
    umma::fence_before_sync();
    __syncthreads();
    if (warp == 2) umma::tmem_free(tmem, P::tmem_cols);
}

}  // namespace

int tall_smem(int prec, int npmax)
{
    return prec == PREC_F32 ? tall_smem_bytes(4, npmax, 4) : tall_smem_bytes(6, npmax, 8);
}

int64_t tall_ws_stride(int prec, int nmax, int G)
{
    return prec == PREC_F32 ? tall_ws_bytes(4, nmax, G, 4) : tall_ws_bytes(6, nmax, G, 8);
}

cudaError_t tall_prepare(int prec, int npmax)
{
    const int bytes = tall_smem(prec, npmax);
    return prec == PREC_F32
               ? cudaFuncSetAttribute(k_tall<float, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes)
               : cudaFuncSetAttribute(k_tall<ff, 6>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

cudaError_t launch_tall(int prec, const SolveArgs& a, unsigned char* ws, int64_t ws_stride, int npmax,
                        int grid, cudaStream_t s)
{
    const int bytes = tall_smem(prec, npmax);
    if (prec == PREC_F32) k_tall<float, 4><<<grid, kT, bytes, s>>>(a, ws, ws_stride, npmax);
    else k_tall<ff, 6><<<grid, kT, bytes, s>>>(a, ws, ws_stride, npmax);
    return cudaGetLastError();
}

}  // namespace gpv
