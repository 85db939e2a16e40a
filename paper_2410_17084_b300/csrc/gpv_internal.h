// gpv_internal.h -- launch arguments shared by the C-ABI layer and the kernels.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace gpv {

enum Prec { PREC_F32 = 0, PREC_FF = 1, PREC_F64 = 2 };

// Per-voxel status bits (mirrors include/gp_voxels.h)
enum : uint32_t {
    VOX_OK = 0,
    VOX_BELOW_TAU = 1u,
    VOX_ESCALATED = 2u,
    VOX_NOT_SPD = 4u,
    VOX_TRUNCATED = 8u,
    VOX_TOO_LARGE = 16u,
    VOX_CONVERGED = 32u,
    VOX_FAILED = 64u,
};

constexpr int kThreads = 512;   // largest CTA size of the solve kernels
constexpr int kRowBlk = 8;      // rows of L^-1 per register tile
constexpr int kQryBlk = 4;      // queries per register tile
constexpr int kMaxG = 32;       // largest query grid side
constexpr int kNumBuckets = 12; // size buckets of the batched launch

// Device counters of the tensor-core variance of one solve call: total = workspace bytes
// all eligible voxels would need (summed when the call classifies its voxels; the call
// takes the tensor-core variance only if it fits tc_cap, so the choice does not depend on
// scheduling), used = bytes handed out, count = voxels queued, next = dequeue counter.
struct TcCounters {
    unsigned long long total, used;
    int32_t count, next;
    int32_t fb_count, fb_next;  // voxels the tensor-core solve variant could not hand over
    int32_t fb2_count, fb2_next;  // the same, too large for the shared-memory kernels
};

struct SolveArgs {
    // inputs (CSR batch of voxels)
    const float* xyz;
    const int64_t* offsets;
    const float* centres;
    const float* lam;
    const float* sf2;
    const float* sn2;
    const float* noise;         // per-point noise variance (replaces sn2 on the diagonal), or null
    const uint8_t* skip;        // per-voxel: nonzero = converged, not solved (or null)
    int32_t nvox;               // rows of the outputs (stride of the escalation lists)
    const int32_t* nvox_dev;    // device count of rows to solve (serving), or null
    float size;
    int G, Gp, n_s, n_r, tau, mean_mode, init_mode;
    float esc_cond;
    int escalate;        // 1: badly conditioned voxels go to esc_list instead of being solved
    int escalation_pass; // 1: this launch re-solves escalated voxels (sets VOX_ESCALATED)
    int refine;          // FP32: one step of iterative refinement of alpha (float-float residual)
    // outputs
    uint8_t* axis;
    float* mean;
    float* var;
    uint32_t* status;
    float* pos;
    float* scale;
    float* quat;
    float* pvar;                // per-point posterior variance at the inputs, or null
    // work queue of this launch
    const int32_t* work;
    const int32_t* work_base;   // device: first entry of this launch in work[] (or null)
    const int32_t* work_count;
    int32_t* work_next;
    int nqueues;                // the tall-matrix kernel drains queues nqueues-1 .. 0 of the
                                // consecutive base/count/next arrays (0 or 1: one queue)
    int32_t* esc_list;
    int32_t* esc_count;
    // global-memory workspace for factors that do not fit shared memory
    void* gws;
    int64_t gws_stride;  // elements of the working type per CTA
    int nmax;            // largest n handled by this launch
    int max_points;      // voxels with more points are reported VOX_TOO_LARGE
    int nmax_small_f64;  // escalated voxels up to this n take the shared-memory FP64 pass
    int percol_max;      // shared-memory voxels up to this n use the per-column factor/inverse
    int panel;           // panel width of the blocked factor: 4, 8 or 16
    // tensor-core variance (float-float, shared-memory factor): the solve kernel leaves
    // L^-1, the cross-covariance factors and the mean of each voxel in tc_ws and k_var_tc
    // forms diag(Sigma*) and the Gaussians from them.  Null tc_ws: the solve kernel
    // forms them itself.
    unsigned char* tc_ws;
    uint64_t tc_cap;     // bytes of tc_ws
    TcCounters* tc;
    int32_t* tc_v;       // voxels queued for k_var_tc (one entry per voxel at most)
    int64_t* tc_off;     // their byte offsets in tc_ws
    int32_t* tc_fb;      // voxels re-solved by the regular kernel (workspace full): n <=
                         // fb_nsmall at [0, nvox), larger ones at [nvox, 2 nvox)
    int fb_nsmall;       // largest n of the shared-memory re-solve
    long long* tc_off_v; // per output row: workspace byte offset, -1 if not handed over
    int tc_nmax;         // largest n that takes the tensor-core variance (factor in shared memory)
    int tc_nmax_gl;      // the same for voxels whose factor lives in the global workspace
};

// Conditioning limit of the tensor-core variance: voxels whose pivot ratio
// (max L_ii / min L_ii)^2 exceeds it keep the float-float contraction on the CUDA cores.
// The slices share one exponent per row of L^-1 and per query, so entries far below their
// row's largest carry fewer bits than in float-float; the worst voxels of the workloads
// stay under 1e4, the 1e5 limit leaves a factor of ten.
constexpr float kTcCond = 1e5f;

// Largest n of the tensor-core variance for voxels whose factor lives in the global
// workspace: the four exact levels 0-3 stay exact for n < 256 (4 x 2^14 n); level 4 is
// exact by the worst-case bound only to n < 204, above that its sum would have to gather
// 5 n products of up to 2^14 units with one sign (the low slices are close to uniformly
// distributed, their sums stay near 2^18 units) to round.
constexpr int kTcMaxNGl = 255;

// Largest n of the tensor-core variance with the factor in shared memory (the variant's
// smaller plan fits about 224 points at G = 16); the exactness of the levels is as for
// the workspace voxels below.
constexpr int kTcMaxN = 224;

// Workspace bytes of one voxel: packed L^-1, the factors (n G and n Gp), the G^2 means
// and the G^2 variances, float-float, then the slice exponents of the n rows of L^-1 and
// of the G^2 queries (int32), rounded up to 16 bytes.
__host__ __device__ inline uint64_t tc_need_bytes(int n, int G, int Gp)
{
    const uint64_t e = (uint64_t)n * (n + 1) / 2 + (uint64_t)n * G + (uint64_t)n * Gp + 2 * (uint64_t)G * G;
    return (8 * e + 4 * ((uint64_t)n + (uint64_t)G * G) + 15) & ~(uint64_t)15;
}

// Shared-memory plan of one CTA (bytes), identical on host and device.
// Elements of the working type in one CTA's global-workspace slice (factor + factors).
__host__ __device__ inline int64_t gws_slice_elems(int nmax, int G, int Gp)
{
    return (int64_t)nmax * (nmax + 1) / 2 + 16 + (int64_t)nmax * G + (int64_t)nmax * Gp + 16;
}

struct SmemPlan {
    int off_pts, off_vec, off_tri, off_a, off_b, off_part, off_mv, off_work, total;
    int nrg, nqg;
    int pb, rb;  // panel width of the blocked factor, row block of the blocked inverse
};

// Shared memory of the workspace variant (factor in global memory): its panel buffers
// take what the other regions leave of this budget.
constexpr int kBigSmem = 216 * 1024;

__host__ __device__ inline int align16(int x) { return (x + 15) & ~15; }

// tcv: the solve variant that hands the variance to k_var_tc (no contraction partials,
// no staged predictions).
__host__ __device__ inline SmemPlan smem_plan(int nmax, int G, int Gp, int tsize, bool tri_in_smem,
                                              int nthr, bool tcv = false)
{
    SmemPlan p;
    int nqg = (G * Gp) / kQryBlk;
    int nrg = nqg >= nthr ? 1 : nthr / nqg;
    p.nqg = nqg;
    p.nrg = nrg;
    int o = 0;
    p.off_pts = o; o = align16(o + 12 * nmax);
    p.off_vec = o; o = align16(o + 5 * nmax * tsize);
    p.off_tri = o;
    // +16 elements of slack: masked tile loads near the end of the triangle stay inside
    if (tri_in_smem) o = align16(o + (int)(((int64_t)nmax * (nmax + 1) / 2 + 16) * tsize));
    // the cross-covariance factors live next to the triangle: in shared memory, or in
    // the CTA's slice of the global workspace
    // the variant without the contraction forms the factors after L^-1 has been handed
    // over, so where they fit they lie over the triangle
    const int64_t tri_bytes = ((int64_t)nmax * (nmax + 1) / 2 + 16) * tsize;
    const bool overlay = tcv && tri_in_smem &&
                         (int64_t)align16(nmax * G * tsize) + (int64_t)nmax * Gp * tsize <= tri_bytes;
    if (overlay) {
        p.off_a = p.off_tri;
        p.off_b = p.off_tri + align16(nmax * G * tsize);
    } else {
        p.off_a = o;
        if (tri_in_smem) o = align16(o + nmax * G * tsize);
        p.off_b = o;
        if (tri_in_smem) o = align16(o + nmax * Gp * tsize);
    }
    p.off_part = o; if (!tcv) o = align16(o + nrg * G * Gp * tsize);
    p.off_mv = o; if (!tcv) o = align16(o + 2 * G * G * 8);
    p.off_work = o;
    p.pb = 0;
    p.rb = 0;
    if (!tri_in_smem) {
        const int work = kBigSmem - o;
        int pb = work > 0 ? work / (2 * nmax * tsize) : 0;
        // the inverse stages rb rows of the factor and a 16 x 16 block
        int rb = work > 256 * tsize ? (work - 256 * tsize) / (nmax * tsize) : 0;
        pb = (pb > 32 ? 32 : pb) & ~3;
        rb = (rb > 16 ? 16 : rb) & ~3;
        p.pb = pb;
        p.rb = rb;
        const int need_f = 2 * pb * nmax * tsize, need_i = (rb * nmax + 256) * tsize;
        const int need = need_f > need_i ? need_f : need_i;
        o = align16(o + need);
    }
    p.total = o;
    return p;
}

// Text of a CUDA error for gp_voxels_last_error() (gpv_api.cu)
void gpv_record_cuda_error(cudaError_t e);

// Default CTA size of a launch: small voxels are bound by the latency of their barriers
// and gain from several CTAs per SM; from 128 points on (and for the workspace variant)
// shared memory allows one CTA per SM, which then gets 16 warps.  The shared-memory
// variants need n <= CTA size.  gp_voxels_autotune may choose another per bucket.
inline int solve_threads(int nmax, bool tri_in_smem) { return (!tri_in_smem || nmax >= 128) ? 512 : 256; }
// Default per-column (rather than blocked) factor and inverse: 8-byte types up to 96 points.
inline int default_percol_max(int tsize) { return tsize == 8 ? 96 : 0; }
// Default CTA size and panel width of a shared-memory bucket of at most hi points.  The
// FP32 shapes are those gp_voxels_autotune picks on the stress, quadric and escalation
// batches: one warp per voxel up to 32 points when the grid has at most 128 queries, two
// up to 48, 128 threads up to 64, 256 up to 160; 4-column panels for 65..96 points, 8 for
// 97..160.  factor_panel > 0 fixes the panel width.
inline void default_bucket_shape(int prec, int hi, int G, int factor_panel, int* nthr, int* panel)
{
    *nthr = solve_threads(hi, true);
    *panel = factor_panel > 0 ? factor_panel : 16;
    if (prec == PREC_F32 && hi <= 160) {
        const bool fewq = G * G <= 128;
        *nthr = fewq && hi <= 32 ? 32 : (fewq && hi <= 48 ? 64 : (hi <= 64 ? 128 : 256));
        if (factor_panel == 0) *panel = hi <= 64 ? 16 : (hi <= 96 ? 4 : 8);
    }
}

// Launchers (gpv_solve.cu)
cudaError_t launch_classify(const SolveArgs& a, const int* bucket_hi, int nb, int32_t* bcount,
                            int32_t* bbase, int32_t* bcursor, int32_t* work, int32_t* next,
                            int32_t* esc_count, cudaStream_t s);
// tcv: the float-float shared-memory variant that hands the variance to k_var_tc
cudaError_t launch_solve(int prec, bool tri_in_smem, int nthr, const SolveArgs& a, int grid, int smem,
                         cudaStream_t s, bool tcv = false);
cudaError_t solve_max_smem_n(int prec, int G, int Gp, int* nmax_out, bool tcv = false);
cudaError_t solve_occupancy(int prec, bool tri_in_smem, int nthr, int smem, int* blocks_per_sm,
                            bool tcv = false);
cudaError_t launch_var_tc(const SolveArgs& a, int sms, cudaStream_t s);
// Large voxels: blocked Cholesky of the tall matrix [K + D; K*^T] on the tensor cores
// (gpv_tall.cu).  prec PREC_FF (six BF16 slices) or PREC_F32 (four); npmax = largest n
// of the launch rounded up to 32; ws holds one slice store of tall_ws_stride() bytes per
// CTA; grid = CTAs (one per SM).
int tall_smem(int prec, int npmax);
int64_t tall_ws_stride(int prec, int nmax, int G);
cudaError_t tall_prepare(int prec, int npmax);
cudaError_t launch_tall(int prec, const SolveArgs& a, unsigned char* ws, int64_t ws_stride, int npmax,
                        int grid, cudaStream_t s);
cudaError_t launch_init_tc(const SolveArgs& a, int sms, cudaStream_t s);
cudaError_t var_tc_prepare();
cudaError_t launch_init(const float* mean, const float* var, const uint8_t* axis,
                        const float* centres, const float* sf2, const uint32_t* status,
                        int32_t nvox, float size, int G, int n_s, int n_r, int init_mode,
                        float* pos, float* scale, float* quat, cudaStream_t s);

}  // namespace gpv
