// gpv_api.cu -- the C ABI of include/gp_voxels.h: handle life cycle, the batched
// solve (size buckets on forked streams, persistent CTAs, FP64 escalation pass) and
// the standalone Gaussian initialisation.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "../../include/gp_voxels.h"
#include "gpv_internal.h"
#include "gpv_store.h"

using namespace gpv;

namespace {

thread_local char g_last_err[256] = "";

int cuda_fail(cudaError_t e)
{
    strncpy(g_last_err, cudaGetErrorString(e), sizeof(g_last_err) - 1);
    g_last_err[sizeof(g_last_err) - 1] = 0;
    return GPV_ECUDA;
}
#define CK(x)                                  \
    do {                                       \
        cudaError_t e_ = (x);                  \
        if (e_ != cudaSuccess) return cuda_fail(e_); \
    } while (0)

struct Bucket {
    int hi;        // largest n of the bucket
    int smem;      // dynamic shared memory of its launch
    int grid;      // persistent CTAs
    bool tri_smem; // factor in shared memory (else in the global workspace slice)
};

struct PrecPlan {
    int nb = 0;
    Bucket b[kNumBuckets];
    int* d_hi = nullptr;  // device copy of the bucket upper bounds
    int nmax_smem = 0;
};

}  // namespace

struct gp_voxels {
    gp_voxels_config cfg;
    int dev = 0, sms = 0, Gp = 0;
    PrecPlan plan[3];
    int32_t* d_bcount = nullptr;
    int32_t* d_bbase = nullptr;
    int32_t* d_bcursor = nullptr;
    int32_t* d_next = nullptr;      // kNumBuckets + 2 dequeue counters
    int32_t* d_work = nullptr;      // max_voxels
    int32_t* d_esc_list = nullptr;  // 2 * max_voxels
    int32_t* d_esc_count = nullptr; // 2
    int32_t* d_one = nullptr;       // constant 1 (one-per-launch baseline)
    int32_t* d_ident = nullptr;     // 0..max_voxels-1
    int32_t* d_pl_next = nullptr;   // max_voxels counters (one-per-launch baseline)
    void* d_gws = nullptr;
    int64_t gws_stride = 0;         // elements (8-byte) per slice
    int gws_grid = 0;
    int esc_grid_small = 0, esc_smem_small = 0, esc_grid_big = 0, esc_smem_big = 0;
    cudaStream_t side[kNumBuckets] = {};
    cudaEvent_t ev_fork = nullptr;
    cudaEvent_t ev_join[kNumBuckets] = {};
    size_t bytes = 0;
    gpv_store* store = nullptr;
};

static int prec_kind(int precision)
{
    return precision == GPV_PREC_FP32 ? PREC_F32 : (precision == GPV_PREC_FP64 ? PREC_F64 : PREC_FF);
}

static int tsize(int kind) { return kind == PREC_F32 ? 4 : 8; }

static int validate(const gp_voxels_config* c)
{
    if (!c) return GPV_EINVAL;
    if (!(c->voxel_size > 0.f)) return GPV_EINVAL;
    if (c->grid_side < 1 || c->grid_side > kMaxG) return GPV_EINVAL;
    if (c->n_s < 1 || c->n_r < 1 || c->n_s * c->n_r != c->grid_side) return GPV_EINVAL;
    if (c->tau < 1 || c->max_points < c->tau || c->max_points > 2048) return GPV_EINVAL;
    if (c->max_voxels < 1) return GPV_EINVAL;
    if (c->mean_mode < 0 || c->mean_mode > 1) return GPV_EINVAL;
    if (c->precision < 0 || c->precision > 2) return GPV_EINVAL;
    if (c->init_mode < 0 || c->init_mode > 1) return GPV_EINVAL;
    if (!(c->esc_cond > 1.f)) return GPV_EINVAL;
    if (c->hash_capacity & (c->hash_capacity - 1)) return GPV_EINVAL;
    return GPV_OK;
}

// Bucket bounds: fixed ladder below max_points, plus the largest n whose factor fits
// shared memory, capped at kNumBuckets buckets.
static std::vector<int> bucket_bounds(int maxp, int nmax_smem)
{
    const int ladder[] = {16, 32, 48, 64, 96, 128, 160, 192, 256, 384, 512, 768, 1024, 2048};
    std::vector<int> b;
    for (int x : ladder)
        if (x < maxp) b.push_back(x);
    if (nmax_smem < maxp) b.push_back(nmax_smem);
    b.push_back(maxp);
    std::sort(b.begin(), b.end());
    b.erase(std::unique(b.begin(), b.end()), b.end());
    while ((int)b.size() > kNumBuckets) b.erase(b.begin());  // merge the smallest
    return b;
}

static int make_plan(gp_voxels_t* h, int kind, PrecPlan& P)
{
    const gp_voxels_config& c = h->cfg;
    CK(solve_max_smem_n(kind, c.grid_side, h->Gp, &P.nmax_smem));
    std::vector<int> bounds = bucket_bounds(c.max_points, P.nmax_smem);
    P.nb = (int)bounds.size();
    int hi_host[kNumBuckets];
    for (int i = 0; i < P.nb; ++i) {
        Bucket& B = P.b[i];
        B.hi = bounds[i];
        hi_host[i] = B.hi;
        B.tri_smem = B.hi <= P.nmax_smem;
        // the workspace variant lays out its slice for max_points, whatever the bucket
        B.smem = smem_plan(B.tri_smem ? B.hi : c.max_points, c.grid_side, h->Gp, tsize(kind),
                           B.tri_smem).total;
        int occ = 0;
        CK(solve_occupancy(kind, B.tri_smem, B.smem, &occ));
        if (occ < 1) return GPV_EINVAL;
        B.grid = B.tri_smem ? h->sms * occ : h->gws_grid;
    }
    CK(cudaMalloc(&P.d_hi, sizeof(int) * kNumBuckets));
    CK(cudaMemcpy(P.d_hi, hi_host, sizeof(int) * P.nb, cudaMemcpyHostToDevice));
    h->bytes += sizeof(int) * kNumBuckets;
    return GPV_OK;
}

extern "C" int gp_voxels_config_default(gp_voxels_config* c)
{
    if (!c) return GPV_EINVAL;
    memset(c, 0, sizeof(*c));
    c->voxel_size = 0.2f;
    c->n_s = 3;
    c->n_r = 3;
    c->grid_side = 9;
    c->tau = 10;
    c->max_points = 256;
    c->max_voxels = 1 << 16;
    c->mean_mode = 1;
    c->precision = GPV_PREC_MIXED;
    c->init_mode = 0;
    c->esc_cond = 1e7f;
    c->hash_capacity = 0;
    c->mem_budget = 0;
    return GPV_OK;
}

static size_t solve_bytes(const gp_voxels_config* c, int sms, int Gp)
{
    const size_t mv = (size_t)c->max_voxels;
    size_t b = 0;
    b += 4 * sizeof(int32_t) * (kNumBuckets + 2);
    b += sizeof(int32_t) * mv * 5;  // work, esc (2x), ident, per-launch counters
    b += 8 * (size_t)gws_slice_elems(c->max_points, c->grid_side, Gp) * (size_t)(2 * sms);
    return b;
}

extern "C" int gp_voxels_query_sizes(const gp_voxels_config* c, size_t* bytes_out)
{
    if (validate(c) != GPV_OK || !bytes_out) return GPV_EINVAL;
    int dev = 0, sms = 148;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int Gp = (c->grid_side + kQryBlk - 1) / kQryBlk * kQryBlk;
    *bytes_out = solve_bytes(c, sms, Gp) + store_bytes(c);
    return GPV_OK;
}

static void release(gp_voxels_t* h)
{
    if (!h) return;
    for (auto& P : h->plan) cudaFree(P.d_hi);
    cudaFree(h->d_bcount); cudaFree(h->d_bbase); cudaFree(h->d_bcursor); cudaFree(h->d_next);
    cudaFree(h->d_work); cudaFree(h->d_esc_list); cudaFree(h->d_esc_count); cudaFree(h->d_one);
    cudaFree(h->d_ident); cudaFree(h->d_pl_next); cudaFree(h->d_gws);
    for (int i = 0; i < kNumBuckets; ++i) {
        if (h->side[i]) cudaStreamDestroy(h->side[i]);
        if (h->ev_join[i]) cudaEventDestroy(h->ev_join[i]);
    }
    if (h->ev_fork) cudaEventDestroy(h->ev_fork);
    store_destroy(h->store);
    delete h;
}

__global__ void k_iota(int32_t* p, int n)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = i;
}

static int create_impl(gp_voxels_t* h)
{
    const gp_voxels_config& c = h->cfg;
    CK(cudaGetDevice(&h->dev));
    CK(cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, h->dev));
    h->Gp = (c.grid_side + kQryBlk - 1) / kQryBlk * kQryBlk;
    h->gws_grid = 2 * h->sms;
    const size_t need = solve_bytes(&c, h->sms, h->Gp) + store_bytes(&c);
    if (c.mem_budget && need > c.mem_budget) return GPV_EBUDGET;
    const size_t mv = (size_t)c.max_voxels;
    auto alloc = [&](void** p, size_t bytes) -> int {
        cudaError_t e = cudaMalloc(p, bytes);
        if (e == cudaErrorMemoryAllocation) { cudaGetLastError(); return GPV_ENOMEM; }
        if (e != cudaSuccess) return cuda_fail(e);
        h->bytes += bytes;
        return GPV_OK;
    };
    int rc;
#define AL(p, b) if ((rc = alloc((void**)&(p), (b))) != GPV_OK) return rc
    AL(h->d_bcount, sizeof(int32_t) * (kNumBuckets + 2));
    AL(h->d_bbase, sizeof(int32_t) * (kNumBuckets + 2));
    AL(h->d_bcursor, sizeof(int32_t) * (kNumBuckets + 2));
    AL(h->d_next, sizeof(int32_t) * (kNumBuckets + 2));
    AL(h->d_work, sizeof(int32_t) * mv);
    AL(h->d_esc_list, sizeof(int32_t) * mv * 2);
    AL(h->d_esc_count, sizeof(int32_t) * 2);
    AL(h->d_one, sizeof(int32_t));
    AL(h->d_ident, sizeof(int32_t) * mv);
    AL(h->d_pl_next, sizeof(int32_t) * mv);
    h->gws_stride = gws_slice_elems(c.max_points, c.grid_side, h->Gp);
    AL(h->d_gws, 8 * (size_t)h->gws_stride * (size_t)h->gws_grid);
#undef AL
    const int one = 1;
    CK(cudaMemcpy(h->d_one, &one, sizeof(int), cudaMemcpyHostToDevice));
    CK(cudaMemset(h->d_esc_count, 0, sizeof(int32_t) * 2));
    k_iota<<<(c.max_voxels + 255) / 256, 256>>>(h->d_ident, c.max_voxels);
    CK(cudaGetLastError());
    for (int k = 0; k < 3; ++k)
        if ((rc = make_plan(h, k, h->plan[k])) != GPV_OK) return rc;
    // FP64 escalation passes: shared-memory variant up to its limit, workspace above
    {
        const PrecPlan& P = h->plan[PREC_F64];
        const int nsm = std::min(P.nmax_smem, c.max_points);
        h->esc_smem_small = smem_plan(nsm, c.grid_side, h->Gp, 8, true).total;
        int occ = 0;
        CK(solve_occupancy(PREC_F64, true, h->esc_smem_small, &occ));
        h->esc_grid_small = h->sms * std::max(occ, 1);
        h->esc_smem_big = smem_plan(c.max_points, c.grid_side, h->Gp, 8, false).total;
        CK(solve_occupancy(PREC_F64, false, h->esc_smem_big, &occ));
        h->esc_grid_big = h->gws_grid;
    }
    for (int i = 0; i < kNumBuckets; ++i) {
        CK(cudaStreamCreateWithFlags(&h->side[i], cudaStreamNonBlocking));
        CK(cudaEventCreateWithFlags(&h->ev_join[i], cudaEventDisableTiming));
    }
    CK(cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming));
    if (c.hash_capacity > 0) {
        rc = store_create(&c, &h->store, &h->bytes);
        if (rc != GPV_OK) return rc;
    }
    CK(cudaDeviceSynchronize());
    return GPV_OK;
}

extern "C" int gp_voxels_create(const gp_voxels_config* cfg, gp_voxels_t** out)
{
    if (!out) return GPV_EINVAL;
    *out = nullptr;
    int rc = validate(cfg);
    if (rc != GPV_OK) return rc;
    gp_voxels_t* h = new (std::nothrow) gp_voxels_t();
    if (!h) return GPV_ENOMEM;
    h->cfg = *cfg;
    rc = create_impl(h);
    if (rc != GPV_OK) {
        release(h);
        return rc;
    }
    *out = h;
    return GPV_OK;
}

extern "C" int gp_voxels_destroy(gp_voxels_t* h)
{
    if (!h) return GPV_OK;
    cudaError_t e = cudaDeviceSynchronize();
    release(h);
    return e == cudaSuccess ? GPV_OK : cuda_fail(e);
}

// Shared by the CSR entry and the serving solve: queue one batched solve.
int gpv_solve_queue(gp_voxels_t* h, const float* d_xyz, const int64_t* d_offsets, int32_t nvox,
                    const float* d_centres, const float* d_lambda, const float* d_sf2,
                    const float* d_sn2, uint8_t* d_axis, float* d_mean, float* d_var,
                    uint32_t* d_status, float* d_pos, float* d_scale, float* d_quat,
                    uint32_t flags, cudaStream_t s)
{
    const gp_voxels_config& c = h->cfg;
    const int kind = prec_kind(c.precision);
    const PrecPlan& P = h->plan[kind];
    SolveArgs a;
    memset(&a, 0, sizeof(a));
    a.xyz = d_xyz; a.offsets = d_offsets; a.centres = d_centres;
    a.lam = d_lambda; a.sf2 = d_sf2; a.sn2 = d_sn2; a.nvox = nvox;
    a.size = c.voxel_size; a.G = c.grid_side; a.Gp = h->Gp; a.n_s = c.n_s; a.n_r = c.n_r;
    a.tau = c.tau; a.mean_mode = c.mean_mode; a.init_mode = c.init_mode;
    a.esc_cond = c.esc_cond;
    a.escalate = kind == PREC_FF ? 1 : 0;
    a.axis = d_axis; a.mean = d_mean; a.var = d_var; a.status = d_status;
    a.pos = d_pos; a.scale = d_scale; a.quat = d_quat;
    a.esc_list = h->d_esc_list; a.esc_count = h->d_esc_count;
    a.gws = h->d_gws; a.gws_stride = h->gws_stride;
    a.max_points = c.max_points;
    a.nmax_small_f64 = std::min(h->plan[PREC_F64].nmax_smem, c.max_points);
    CK(launch_classify(a, P.d_hi, P.nb, h->d_bcount, h->d_bbase, h->d_bcursor, h->d_work,
                       h->d_next, h->d_esc_count, s));
    if (nvox == 0) return GPV_OK;

    if (flags & GPV_SOLVE_ONE_PER_LAUNCH) {
        // Baseline: one launch per voxel, sized for that voxel.
        std::vector<int64_t> off((size_t)nvox + 1);
        CK(cudaMemcpyAsync(off.data(), d_offsets, sizeof(int64_t) * (nvox + 1), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        CK(cudaMemsetAsync(h->d_pl_next, 0, sizeof(int32_t) * nvox, s));
        a.escalate = 0;
        a.work_count = h->d_one;
        a.work_base = nullptr;
        for (int32_t v = 0; v < nvox; ++v) {
            const int64_t n = off[v + 1] - off[v];
            if (n < c.tau || n <= 0 || n > c.max_points) continue;
            a.work = h->d_ident + v;
            a.work_next = h->d_pl_next + v;
            a.nmax = (int)((n + 7) / 8 * 8);
            const bool sm = a.nmax <= P.nmax_smem;
            if (!sm) a.nmax = c.max_points;
            const int smem = smem_plan(a.nmax, c.grid_side, h->Gp, tsize(kind), sm).total;
            CK(launch_solve(kind, sm, a, 1, smem, s));
        }
        return GPV_OK;
    }

    // Batched: one persistent launch per size bucket, buckets on forked streams.
    // Buckets whose factor lives in the global workspace share it, so they run
    // one after another on the first side stream.
    CK(cudaEventRecord(h->ev_fork, s));
    int used = 0;
    for (int b = P.nb - 1; b >= 0; --b) {
        const Bucket& B = P.b[b];
        const int si = B.tri_smem ? 1 + b : 0;
        cudaStream_t ss = h->side[si % kNumBuckets];
        CK(cudaStreamWaitEvent(ss, h->ev_fork, 0));
        a.work = h->d_work;
        a.work_base = h->d_bbase + b;
        a.work_count = h->d_bcount + b;
        a.work_next = h->d_next + b;
        a.nmax = B.tri_smem ? B.hi : c.max_points;
        CK(launch_solve(kind, B.tri_smem, a, B.grid, B.smem, ss));
        used |= 1 << (si % kNumBuckets);
    }
    for (int i = 0; i < kNumBuckets; ++i)
        if (used & (1 << i)) {
            CK(cudaEventRecord(h->ev_join[i], h->side[i]));
            CK(cudaStreamWaitEvent(s, h->ev_join[i], 0));
        }
    if (kind == PREC_FF) {
        // FP64 re-solve of the voxels that failed the conditioning check
        a.escalate = 0;
        a.escalation_pass = 1;
        a.work = h->d_esc_list;
        a.work_base = nullptr;
        a.work_count = h->d_esc_count;
        a.work_next = h->d_next + P.nb;
        a.nmax = a.nmax_small_f64;
        CK(launch_solve(PREC_F64, true, a, h->esc_grid_small, h->esc_smem_small, s));
        if (c.max_points > a.nmax_small_f64) {
            a.work = h->d_esc_list + nvox;
            a.work_count = h->d_esc_count + 1;
            a.work_next = h->d_next + P.nb + 1;
            a.nmax = c.max_points;
            CK(launch_solve(PREC_F64, false, a, h->esc_grid_big, h->esc_smem_big, s));
        }
    }
    return GPV_OK;
}

extern "C" int gp_voxels_solve_csr(gp_voxels_t* h, const float* d_xyz, const int64_t* d_offsets,
                                   int32_t nvox, const float* d_centres, const float* d_lambda,
                                   const float* d_sf2, const float* d_sn2, uint8_t* d_axis,
                                   float* d_mean, float* d_var, uint32_t* d_status, float* d_pos,
                                   float* d_scale, float* d_quat, uint32_t flags,
                                   gpv_stream_t stream)
{
    if (!h || nvox < 0 || nvox > h->cfg.max_voxels) return GPV_EINVAL;
    if (nvox == 0) return GPV_OK;  // nothing to read or write
    if (!d_offsets || !d_axis || !d_mean || !d_var || !d_status) return GPV_EINVAL;
    if (nvox > 0 && (!d_xyz || !d_centres || !d_lambda || !d_sf2 || !d_sn2)) return GPV_EINVAL;
    const bool any_init = d_pos || d_scale || d_quat;
    if (any_init && !(d_pos && d_scale && d_quat)) return GPV_EINVAL;
    if (flags & ~(uint32_t)GPV_SOLVE_ONE_PER_LAUNCH) return GPV_EINVAL;
    return gpv_solve_queue(h, d_xyz, d_offsets, nvox, d_centres, d_lambda, d_sf2, d_sn2, d_axis,
                           d_mean, d_var, d_status, d_pos, d_scale, d_quat, flags,
                           (cudaStream_t)stream);
}

extern "C" int gp_voxels_init_gaussians(gp_voxels_t* h, int32_t nvox, const uint8_t* d_axis,
                                        const float* d_centres, const float* d_sf2,
                                        const float* d_mean, const float* d_var,
                                        const uint32_t* d_status, float* d_pos, float* d_scale,
                                        float* d_quat, gpv_stream_t stream)
{
    if (!h || nvox < 0) return GPV_EINVAL;
    if (nvox == 0) return GPV_OK;
    if (!d_axis || !d_centres || !d_sf2 || !d_mean || !d_var || !d_pos || !d_scale || !d_quat)
        return GPV_EINVAL;
    const gp_voxels_config& c = h->cfg;
    CK(launch_init(d_mean, d_var, d_axis, d_centres, d_sf2, d_status, nvox, c.voxel_size,
                   c.grid_side, c.n_s, c.n_r, c.init_mode, d_pos, d_scale, d_quat,
                   (cudaStream_t)stream));
    return GPV_OK;
}

extern "C" const char* gp_voxels_strerror(int s)
{
    switch (s) {
    case GPV_OK: return "ok";
    case GPV_EINVAL: return "invalid argument";
    case GPV_ENOMEM: return "out of memory";
    case GPV_EBUDGET: return "memory budget exceeded";
    case GPV_ECUDA: return "CUDA error";
    case GPV_ETIMEOUT: return "timed out";
    case GPV_EFULL: return "capacity exhausted";
    default: return "unknown status";
    }
}

extern "C" const char* gp_voxels_last_error(void) { return g_last_err; }
