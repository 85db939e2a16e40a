// gpv_api.cu -- the C ABI of include/gp_voxels.h: handle life cycle, the batched
// solve (size buckets on forked streams, persistent CTAs, FP64 escalation pass) and
// the standalone Gaussian initialisation.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <climits>
#include <new>
#include <vector>

#include "../../include/gp_voxels.h"
#include "gpv_alg3.h"
#include "gpv_internal.h"
#include "gpv_lp.h"
#include "gpv_raster.h"
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

// Launch configuration of the solve variant that hands the variance to the tensor cores
struct VarCfg {
    int nthr = 0, smem = 0, grid = 0;
    bool percol = false;
    int panel = 16;
};

struct Bucket {
    int hi;        // largest n of the bucket
    int nthr;      // CTA size
    int smem;      // dynamic shared memory of its launch
    int grid;      // persistent CTAs
    bool tri_smem; // factor in shared memory (else in the global workspace slice)
    bool percol;   // per-column (not blocked) factor and inverse
    int panel;     // panel width of the blocked factor (4, 8, 16)
    bool tall;     // the bucket's voxels take the tall-matrix tensor-core factorisation
    bool tcv_ok;   // float-float bucket whose voxels all take the tensor-core variance
    VarCfg v;      // its launch configuration in that case
};

struct PrecPlan {
    int nb = 0;
    Bucket b[kNumBuckets];
    int* d_hi = nullptr;  // device copy of the bucket upper bounds
    int nmax_smem = 0;
    int tc_nmax = 0;      // largest n of the tensor-core variance (0: off)
    int tc_nmax_gl = 0;   // the same for the global-workspace buckets
    // regular re-solve of what the variant could not hand over: voxels up to nmax_smem in
    // shared memory, larger ones with the factor in the global workspace (or, where the
    // context has one, on the tall-matrix path)
    int fb_smem = 0, fb_grid = 0, fb_nthr = 512;
    int fbb_smem = 0, fbb_grid = 0;
};

// Work queues, workspace and streams of one solve in flight.  The CSR entry owns one;
// every serving scan slot owns another, so solves of different scans overlap safely.
struct SolveCtx {
    int cap = 0;                    // rows
    int32_t* d_bcount = nullptr;
    int32_t* d_bbase = nullptr;
    int32_t* d_bcursor = nullptr;
    int32_t* d_next = nullptr;      // kNumBuckets + 2 dequeue counters
    int32_t* d_work = nullptr;      // cap
    int32_t* d_esc_list = nullptr;  // 2 * cap
    int32_t* d_esc_count = nullptr; // 2
    void* d_gws = nullptr;
    // tensor-core variance (float-float): workspace, counters, queue (tc_cap 0 = off)
    unsigned char* d_tc_ws = nullptr;
    uint64_t tc_cap = 0;
    TcCounters* d_tc = nullptr;
    int32_t* d_tc_v = nullptr;
    int64_t* d_tc_off = nullptr;
    int32_t* d_tc_fb = nullptr;
    long long* d_tc_off_v = nullptr;  // per row
    int32_t* d_tc_next = nullptr;     // k_var_tc dequeue counter per size bucket
    unsigned char* d_tall = nullptr;  // slice stores of the tall-matrix factorisation (one per CTA)
    cudaStream_t side[kNumBuckets] = {};
    cudaEvent_t ev_fork = nullptr;
    cudaEvent_t ev_join[kNumBuckets] = {};
};

}  // namespace

struct gp_voxels {
    gp_voxels_config cfg;
    int dev = 0, sms = 0, Gp = 0;
    PrecPlan plan[3];
    SolveCtx main;
    SolveCtx* sctx = nullptr;       // one per scan slot
    int32_t* d_one = nullptr;       // constant 1 (one-per-launch baseline)
    int32_t* d_ident = nullptr;     // 0..max_voxels-1
    int32_t* d_pl_next = nullptr;   // max_voxels counters (one-per-launch baseline)
    int64_t gws_stride = 0;         // elements (8-byte) per slice
    int gws_grid = 0;
    int tall_min = INT_MAX;         // voxels with more points take the tall-matrix path
    int64_t tall_stride = 0;        // bytes of one CTA's slice store
    bool timing = false;            // record events around the tall-matrix launches
    bool timed_tall = false;        // the last batch solve recorded them
    cudaEvent_t ev_tall[2] = {nullptr, nullptr};
    int esc_grid_small = 0, esc_smem_small = 0, esc_grid_big = 0, esc_smem_big = 0;
    size_t bytes = 0;
    gpv_store* store = nullptr;
    int last_launches = 0;          // kernels queued by the last solve call
    // workspace of the Alg. 3 formulation (allocated by its first call)
    struct {
        int nmax = 0, nsm = 0, kp = 0, qp = 0, chunk = 0;
        float *pk = nullptr, *tf = nullptr, *fa = nullptr, *fb = nullptr, *A = nullptr;
        uint32_t* st = nullptr;
        int32_t* n = nullptr;
        int32_t* vidx = nullptr;    // processing order (max_voxels) and its two counters
        int32_t* counts = nullptr;
        cudaStream_t side = nullptr;  // the class beyond shared memory runs beside the rest
        cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    } a3;
    // workspace of the structure similarity loss (grown on demand)
    struct LpWork {
        int32_t mcap = 0, ncap = 0;
        uint32_t H = 0;
        uint64_t* keys = nullptr;
        int32_t *head = nullptr, *next = nullptr, *pending = nullptr, *counters = nullptr;
        int32_t* arg = nullptr;
        float* best = nullptr;
        uint32_t* smax = nullptr;
        double* partial = nullptr;
    } lp;
    // workspace of the rasteriser (grown on demand)
    struct RsWork {
        int32_t mcap = 0, tcap = 0;
        int64_t kcap = 0;
        float4* sp = nullptr;
        int4* rect = nullptr;
        int32_t *count = nullptr, *off = nullptr, *cursor = nullptr;
        uint64_t* keys = nullptr;
    } rs;
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
    if (c->tau < 1 || c->max_points < c->tau || c->max_points > 1024) return GPV_EINVAL;
    if (c->max_voxels < 1) return GPV_EINVAL;
    if (c->mean_mode < 0 || c->mean_mode > 1) return GPV_EINVAL;
    if (c->precision < 0 || c->precision > 2) return GPV_EINVAL;
    if (c->init_mode < 0 || c->init_mode > 1) return GPV_EINVAL;
    if (!(c->esc_cond > 1.f)) return GPV_EINVAL;
    if (c->tc_workspace_mb < 0 || c->tc_workspace_mb > (1 << 20)) return GPV_EINVAL;
    if (c->refine < 0 || c->refine > 1) return GPV_EINVAL;
    if (c->tall_min_points < -1 || c->tall_min_points > 1024) return GPV_EINVAL;
    if (c->factor_panel != 0 && c->factor_panel != 4 && c->factor_panel != 8 && c->factor_panel != 16)
        return GPV_EINVAL;
    if (c->hash_capacity & (c->hash_capacity - 1)) return GPV_EINVAL;
    if (c->hash_capacity > 0) {
        if (c->scan_slots < 1 || c->scan_slots > 64) return GPV_EINVAL;
        if (c->max_scan_points < 1 || c->max_scan_points > (1 << 20)) return GPV_EINVAL;
        if (c->max_scan_voxels < 1 || c->max_scan_voxels > c->max_voxels ||
            c->max_scan_voxels >= (1 << 20) - 1)
            return GPV_EINVAL;
        if (c->snap_points < 0) return GPV_EINVAL;
        if (!(c->lambda > 0.f) || !(c->sf2 > 0.f) || !(c->sn2 >= 0.f)) return GPV_EINVAL;
        if (c->eta > 0.f && !(c->noise_floor >= 0.f && c->eta < 3.0e38f)) return GPV_EINVAL;
    }
    return GPV_OK;
}

// Bucket bounds: fixed ladder below max_points, plus the largest n whose factor fits
// shared memory, capped at kNumBuckets buckets.  With the tall-matrix path on, its one
// launch drains the buckets above tall_min (largest first: three bounds are enough) and
// the ladder below it is fine, so that the smallest voxels run in CTAs sized for them.
static std::vector<int> bucket_bounds(int maxp, int nmax_smem, int extra = 0, int tall_min = INT_MAX)
{
    std::vector<int> b;
    if (tall_min < maxp) {
        const int small[] = {8, 16, 24, 32, 48, 64, 96, 128, 160, 192};
        for (int x : small)
            if (x < tall_min) b.push_back(x);
        b.push_back(tall_min);
        for (int x : {256, 512})
            if (x > tall_min && x < maxp) b.push_back(x);
        b.push_back(maxp);
        std::sort(b.begin(), b.end());
        b.erase(std::unique(b.begin(), b.end()), b.end());
        while ((int)b.size() > kNumBuckets) b.erase(b.begin());  // merge the smallest
        return b;
    }
    const int ladder[] = {16, 32, 48, 64, 96, 128, 160, 192, 256, 384, 512, 768, 1024, 2048};
    for (int x : ladder)
        if (x < maxp) b.push_back(x);
    if (nmax_smem < maxp) b.push_back(nmax_smem);
    if (extra > 0 && extra < maxp) b.push_back(extra);
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
    // tensor-core variance (float-float; the batch entry or the scan slots have a
    // workspace): the variant without the contraction fits larger voxels in shared memory,
    // so its largest n is a bucket bound of its own
    P.tc_nmax = 0;
    P.tc_nmax_gl = 0;
    const bool tc_on = kind == PREC_FF && (h->main.tc_cap > 0 || (h->sctx && h->sctx[0].tc_cap > 0));
    if (tc_on) {
        int nmax_tcv = 0;
        CK(solve_max_smem_n(kind, c.grid_side, h->Gp, &nmax_tcv, true));
        P.tc_nmax = std::min(std::min(kTcMaxN, c.max_points), std::max(nmax_tcv, P.nmax_smem));
        P.tc_nmax_gl = std::min(kTcMaxNGl, c.max_points);
    }
    const bool tall_on = kind == prec_kind(c.precision) && h->tall_min != INT_MAX;
    std::vector<int> bounds = bucket_bounds(c.max_points, P.nmax_smem, P.tc_nmax,
                                            tall_on ? h->tall_min : INT_MAX);
    if (tall_on && std::find(bounds.begin(), bounds.end(), h->tall_min) == bounds.end()) {
        bounds.push_back(h->tall_min);
        std::sort(bounds.begin(), bounds.end());
        while ((int)bounds.size() > kNumBuckets) bounds.erase(bounds.begin());
    }
    P.nb = (int)bounds.size();
    int hi_host[kNumBuckets];
    for (int i = 0; i < P.nb; ++i) {
        Bucket& B = P.b[i];
        B.hi = bounds[i];
        hi_host[i] = B.hi;
        B.tri_smem = B.hi <= P.nmax_smem;
        // the workspace variant lays out its slice for max_points, whatever the bucket
        B.nthr = solve_threads(B.hi, B.tri_smem);
        // an explicit panel width selects the blocked factor for every shared-memory bucket
        B.percol = c.factor_panel == 0 && B.tri_smem && B.hi <= default_percol_max(tsize(kind));
        B.panel = c.factor_panel > 0 ? c.factor_panel : 16;
        if (B.tri_smem) default_bucket_shape(kind, B.hi, c.grid_side, c.factor_panel, &B.nthr, &B.panel);
        const SmemPlan sp = smem_plan(B.tri_smem ? B.hi : c.max_points, c.grid_side, h->Gp,
                                      tsize(kind), B.tri_smem, B.nthr);
        if (!B.tri_smem && (sp.pb < 4 || sp.rb < 4)) return GPV_EINVAL;  // panels too thin
        B.smem = sp.total;
        int occ = 0;
        CK(solve_occupancy(kind, B.tri_smem, B.nthr, B.smem, &occ));
        if (occ < 1) return GPV_EINVAL;
        B.grid = B.tri_smem ? h->sms * occ : h->gws_grid;
        B.tcv_ok = false;
        B.tall = tall_on && B.hi > h->tall_min;
    }
    if (tc_on) {  // the variant for every bucket up to its largest n (shared memory)
        for (int i = 0; i < P.nb; ++i) {
            Bucket& B = P.b[i];
            if (B.hi > P.tc_nmax || B.tall) continue;
            B.tcv_ok = true;
            // defaults as the autotuner picks them: without the contraction, 256-thread CTAs
            // (three per SM) beat 512 for blocked factors, 128-thread per-column ones for
            // the small buckets, one warp or two per voxel for the smallest when the query
            // grid is small (at most 128 queries, whose means the CTA forms)
            const bool fewq = c.grid_side * c.grid_side <= 128;
            B.v.nthr = fewq && B.hi <= 16 ? 32 : (fewq && B.hi <= 32 ? 64 : (B.hi <= 64 ? 128 : 256));
            B.v.percol = c.factor_panel == 0 && B.hi <= 64;
            B.v.panel = c.factor_panel > 0 ? c.factor_panel : 4;
            B.v.smem = smem_plan(B.hi, c.grid_side, h->Gp, 8, true, B.v.nthr, true).total;
            int occ = 0;
            CK(solve_occupancy(kind, true, B.v.nthr, B.v.smem, &occ, true));
            if (occ < 1) return GPV_EINVAL;
            B.v.grid = h->sms * occ;
        }
        // the re-solve of what the variant cannot hand over
        P.fb_nthr = solve_threads(P.nmax_smem, true);
        P.fb_smem = smem_plan(P.nmax_smem, c.grid_side, h->Gp, 8, true, P.fb_nthr).total;
        int occ = 0;
        CK(solve_occupancy(kind, true, P.fb_nthr, P.fb_smem, &occ));
        if (occ < 1) return GPV_EINVAL;
        P.fb_grid = h->sms * occ;
        P.fbb_smem = smem_plan(c.max_points, c.grid_side, h->Gp, 8, false, 512).total;
        CK(solve_occupancy(kind, false, 512, P.fbb_smem, &occ));
        if (occ < 1) return GPV_EINVAL;
        P.fbb_grid = h->gws_grid;
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
    c->scan_slots = 4;
    c->max_scan_points = 1 << 17;
    c->max_scan_voxels = 1 << 16;
    c->snap_points = 0;
    c->lambda = 1.f;
    c->sf2 = 1.f;
    c->sn2 = 4e-4f;
    c->tc_workspace_mb = 4096;
    c->refine = 1;
    return GPV_OK;
}

// Smallest n that is not taken by the tall-matrix path: INT_MAX where the path is off
// (FP64, tall_min_points = -1, or no voxel can exceed the threshold).  By default the
// threshold is the largest n of the shared-memory kernels of the configured precision
// (for the mixed precision with the tensor-core variance, the largest n of its
// shared-memory variant), so the tall path replaces the global-workspace kernel.
static int tall_threshold(const gp_voxels_config* c, int Gp)
{
    if (c->precision == GPV_PREC_FP64 || c->tall_min_points < 0) return INT_MAX;
    int t = c->tall_min_points;
    if (t == 0) {
        // The tall-matrix kernel solves voxels of more than about 128 points faster than
        // the shared-memory kernels (measured on the 1M-voxel stress batch: 1.12 against
        // 1.24 s per step in float-float; on the quadric and escalation batches too); with
        // G > 16 its query rows lengthen every panel, so 160 there.  FP32 keeps its
        // shared-memory kernels (and their refinement step of alpha) up to 160 points.
        const int kind = c->precision == GPV_PREC_FP32 ? PREC_F32 : PREC_FF;
        int nsm = 0;
        if (solve_max_smem_n(kind, c->grid_side, Gp, &nsm) != cudaSuccess) return INT_MAX;
        t = kind == PREC_F32 ? 160 : (c->grid_side > 16 ? 160 : 128);
        t = std::min(t, nsm);
    }
    return t < c->max_points ? t : INT_MAX;
}

static size_t tall_bytes(const gp_voxels_config* c, int sms, int Gp)
{
    if (tall_threshold(c, Gp) == INT_MAX) return 0;
    const int kind = c->precision == GPV_PREC_FP32 ? PREC_F32 : PREC_FF;
    return (size_t)sms * (size_t)tall_ws_stride(kind, c->max_points, c->grid_side);
}

static size_t ctx_bytes(const gp_voxels_config* c, int cap, int sms, int Gp)
{
    size_t b = 4 * sizeof(int32_t) * (kNumBuckets + 2) + 2 * sizeof(int32_t);
    b += sizeof(int32_t) * (size_t)cap * 3;  // work, escalation lists
    b += 8 * (size_t)gws_slice_elems(c->max_points, c->grid_side, Gp) * (size_t)(2 * sms);
    return b;
}

// Queue lists of the tensor-core variance for a context of cap voxels.
static size_t tc_lists(int cap)
{
    return (size_t)cap * (3 * sizeof(int32_t) + 2 * sizeof(int64_t)) + sizeof(TcCounters) +
           sizeof(int32_t) * kNumBuckets;
}

// Workspaces of the tensor-core variance, per solve context: the batch entry's and, when
// the store is on without the voxel state machine, each serving scan slot's (slots may be
// in flight together, so each needs its own; with the state machine the scans solve few,
// mostly small voxels, whose variance the CUDA cores form sooner than the extra launches
// of the tensor-core path).  The configured size is split evenly between the contexts;
// each share is capped by what the context's voxels of the largest eligible n could use
// and, under a memory budget, by what the budget leaves.  A share below 16 MB is not worth
// keeping.  Returned sizes include the queue lists; 0 means off for that context.
struct TcSplit { size_t main = 0, slot = 0; };

static TcSplit tc_split(const gp_voxels_config* c, int Gp, size_t rest)
{
    TcSplit t;
    if (c->precision != GPV_PREC_MIXED || c->tc_workspace_mb <= 0) return t;
    const int nmax = std::min(std::max(kTcMaxN, kTcMaxNGl), c->max_points);
    const size_t per = tc_need_bytes(nmax, c->grid_side, Gp);
    const int slots = (c->hash_capacity > 0 && !(c->eta > 0.f)) ? c->scan_slots : 0;
    size_t share = ((size_t)c->tc_workspace_mb << 20) / (size_t)(1 + slots);
    if (c->mem_budget) {
        const size_t lists = tc_lists(c->max_voxels) + (size_t)slots * tc_lists(c->max_scan_voxels);
        const size_t left = c->mem_budget > rest + lists ? c->mem_budget - rest - lists : 0;
        share = std::min(share, left / (size_t)(1 + slots));
    }
    auto one = [&](int cap) -> size_t {
        const size_t ws = std::min(share, (size_t)cap * per);
        return ws < ((size_t)16 << 20) ? 0 : ws + tc_lists(cap);
    };
    t.main = one(c->max_voxels);
    if (slots > 0) t.slot = one(c->max_scan_voxels);
    return t;
}

static size_t solve_bytes(const gp_voxels_config* c, int sms, int Gp)
{
    size_t b = ctx_bytes(c, c->max_voxels, sms, Gp);
    // the batch entry and every scan slot have a slice store of the tall-matrix path
    b += tall_bytes(c, sms, Gp) * (size_t)(1 + (c->hash_capacity > 0 ? c->scan_slots : 0));
    b += sizeof(int32_t) * ((size_t)c->max_voxels * 2 + 1);  // ident, per-launch counters
    if (c->hash_capacity > 0)
        b += (size_t)c->scan_slots * ctx_bytes(c, c->max_scan_voxels, sms, Gp);
    return b;
}

static size_t solve_bytes_tc(const gp_voxels_config* c, int sms, int Gp)
{
    const size_t rest = solve_bytes(c, sms, Gp) + store_bytes(c);
    const TcSplit t = tc_split(c, Gp, rest);
    return rest + t.main + (c->hash_capacity > 0 ? (size_t)c->scan_slots * t.slot : 0);
}

extern "C" int gp_voxels_query_sizes(const gp_voxels_config* c, size_t* bytes_out)
{
    if (validate(c) != GPV_OK || !bytes_out) return GPV_EINVAL;
    int dev = 0, sms = 148;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int Gp = (c->grid_side + kQryBlk - 1) / kQryBlk * kQryBlk;
    *bytes_out = solve_bytes_tc(c, sms, Gp);
    return GPV_OK;
}

static void ctx_release(SolveCtx& x)
{
    cudaFree(x.d_bcount); cudaFree(x.d_bbase); cudaFree(x.d_bcursor); cudaFree(x.d_next);
    cudaFree(x.d_work); cudaFree(x.d_esc_list); cudaFree(x.d_esc_count); cudaFree(x.d_gws);
    cudaFree(x.d_tc_ws); cudaFree(x.d_tc); cudaFree(x.d_tc_v); cudaFree(x.d_tc_off); cudaFree(x.d_tc_fb);
    cudaFree(x.d_tc_off_v); cudaFree(x.d_tc_next); cudaFree(x.d_tall);
    for (int i = 0; i < kNumBuckets; ++i) {
        if (x.side[i]) cudaStreamDestroy(x.side[i]);
        if (x.ev_join[i]) cudaEventDestroy(x.ev_join[i]);
    }
    if (x.ev_fork) cudaEventDestroy(x.ev_fork);
    x = SolveCtx();
}

static void release(gp_voxels_t* h)
{
    if (!h) return;
    for (auto& P : h->plan) cudaFree(P.d_hi);
    ctx_release(h->main);
    if (h->sctx) {
        for (int i = 0; i < h->cfg.scan_slots; ++i) ctx_release(h->sctx[i]);
        delete[] h->sctx;
    }
    cudaFree(h->d_one); cudaFree(h->d_ident); cudaFree(h->d_pl_next);
    for (auto& e : h->ev_tall)
        if (e) cudaEventDestroy(e);
    cudaFree(h->a3.pk); cudaFree(h->a3.tf); cudaFree(h->a3.fa); cudaFree(h->a3.fb); cudaFree(h->a3.A);
    cudaFree(h->a3.st); cudaFree(h->a3.n); cudaFree(h->a3.vidx); cudaFree(h->a3.counts);
    if (h->a3.side) cudaStreamDestroy(h->a3.side);
    if (h->a3.ev_fork) cudaEventDestroy(h->a3.ev_fork);
    if (h->a3.ev_join) cudaEventDestroy(h->a3.ev_join);
    cudaFree(h->lp.keys); cudaFree(h->lp.head); cudaFree(h->lp.next); cudaFree(h->lp.pending);
    cudaFree(h->lp.counters); cudaFree(h->lp.arg); cudaFree(h->lp.best); cudaFree(h->lp.smax);
    cudaFree(h->lp.partial);
    cudaFree(h->rs.sp); cudaFree(h->rs.rect); cudaFree(h->rs.count); cudaFree(h->rs.off);
    cudaFree(h->rs.cursor); cudaFree(h->rs.keys);
    store_destroy(h->store);
    delete h;
}

static int ctx_create(gp_voxels_t* h, SolveCtx& x, int cap, size_t tc_total = 0)
{
    auto alloc = [&](void** p, size_t bytes) -> int {
        cudaError_t e = cudaMalloc(p, bytes);
        if (e == cudaErrorMemoryAllocation) { cudaGetLastError(); return GPV_ENOMEM; }
        if (e != cudaSuccess) return cuda_fail(e);
        h->bytes += bytes;
        return GPV_OK;
    };
    int rc;
#define AL(p, b) if ((rc = alloc((void**)&(p), (b))) != GPV_OK) return rc
    x.cap = cap;
    AL(x.d_bcount, sizeof(int32_t) * (kNumBuckets + 2));
    AL(x.d_bbase, sizeof(int32_t) * (kNumBuckets + 2));
    AL(x.d_bcursor, sizeof(int32_t) * (kNumBuckets + 2));
    AL(x.d_next, sizeof(int32_t) * (kNumBuckets + 2));
    AL(x.d_work, sizeof(int32_t) * (size_t)cap);
    AL(x.d_esc_list, sizeof(int32_t) * (size_t)cap * 2);
    AL(x.d_esc_count, sizeof(int32_t) * 2);
    AL(x.d_gws, 8 * (size_t)h->gws_stride * (size_t)h->gws_grid);
    if (tc_total > 0) {
        x.tc_cap = tc_total - tc_lists(cap);
        AL(x.d_tc_ws, x.tc_cap);
        AL(x.d_tc, sizeof(TcCounters));
        AL(x.d_tc_v, sizeof(int32_t) * (size_t)cap);
        AL(x.d_tc_off, sizeof(int64_t) * (size_t)cap);
        AL(x.d_tc_fb, sizeof(int32_t) * (size_t)cap * 2);
        AL(x.d_tc_off_v, sizeof(long long) * (size_t)cap);
        AL(x.d_tc_next, sizeof(int32_t) * kNumBuckets);
    }
#undef AL
    CK(cudaMemset(x.d_esc_count, 0, sizeof(int32_t) * 2));
    for (int i = 0; i < kNumBuckets; ++i) {
        CK(cudaStreamCreateWithFlags(&x.side[i], cudaStreamNonBlocking));
        CK(cudaEventCreateWithFlags(&x.ev_join[i], cudaEventDisableTiming));
    }
    CK(cudaEventCreateWithFlags(&x.ev_fork, cudaEventDisableTiming));
    return GPV_OK;
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
    const size_t need_rest = solve_bytes(&c, h->sms, h->Gp) + store_bytes(&c);
    if (c.mem_budget && need_rest > c.mem_budget) return GPV_EBUDGET;
    const TcSplit need_tc = tc_split(&c, h->Gp, need_rest);
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
    AL(h->d_one, sizeof(int32_t));
    AL(h->d_ident, sizeof(int32_t) * mv);
    AL(h->d_pl_next, sizeof(int32_t) * mv);
#undef AL
    h->gws_stride = gws_slice_elems(c.max_points, c.grid_side, h->Gp);
    if ((rc = ctx_create(h, h->main, c.max_voxels, need_tc.main)) != GPV_OK) return rc;
    h->tall_min = tall_threshold(&c, h->Gp);
    if (h->tall_min != INT_MAX) {
        const int kind = prec_kind(c.precision);
        const int np = (c.max_points + 31) / 32 * 32;
        int dev = 0, optin = 0;
        CK(cudaGetDevice(&dev));
        CK(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
        if (tall_smem(kind, np) + 8192 > optin) return GPV_EINVAL;  // max_points too large
        CK(tall_prepare(kind, np));
        h->tall_stride = tall_ws_stride(kind, c.max_points, c.grid_side);
        const size_t b = (size_t)h->sms * (size_t)h->tall_stride;
        cudaError_t e = cudaMalloc((void**)&h->main.d_tall, b);
        if (e == cudaErrorMemoryAllocation) { cudaGetLastError(); return GPV_ENOMEM; }
        if (e != cudaSuccess) return cuda_fail(e);
        h->bytes += b;
    }
    const size_t tall_slot = h->tall_min != INT_MAX ? (size_t)h->sms * (size_t)h->tall_stride : 0;
    if (need_tc.main > 0 || (c.hash_capacity > 0 && need_tc.slot > 0)) CK(var_tc_prepare());
    if (c.hash_capacity > 0) {
        h->sctx = new (std::nothrow) SolveCtx[c.scan_slots];
        if (!h->sctx) return GPV_ENOMEM;
        for (int i = 0; i < c.scan_slots; ++i) {
            if ((rc = ctx_create(h, h->sctx[i], c.max_scan_voxels, need_tc.slot)) != GPV_OK) return rc;
            if (tall_slot) {
                cudaError_t e = cudaMalloc((void**)&h->sctx[i].d_tall, tall_slot);
                if (e == cudaErrorMemoryAllocation) { cudaGetLastError(); return GPV_ENOMEM; }
                if (e != cudaSuccess) return cuda_fail(e);
                h->bytes += tall_slot;
            }
        }
    }
    const int one = 1;
    CK(cudaMemcpy(h->d_one, &one, sizeof(int), cudaMemcpyHostToDevice));
    k_iota<<<(c.max_voxels + 255) / 256, 256>>>(h->d_ident, c.max_voxels);
    CK(cudaGetLastError());
    for (int k = 0; k < 3; ++k)
        if ((rc = make_plan(h, k, h->plan[k])) != GPV_OK) return rc;
    // FP64 escalation passes: shared-memory variant up to its limit, workspace above
    {
        const PrecPlan& P = h->plan[PREC_F64];
        const int nsm = std::min(P.nmax_smem, c.max_points);
        h->esc_smem_small = smem_plan(nsm, c.grid_side, h->Gp, 8, true, solve_threads(nsm, true)).total;
        int occ = 0;
        CK(solve_occupancy(PREC_F64, true, solve_threads(nsm, true), h->esc_smem_small, &occ));
        h->esc_grid_small = h->sms * std::max(occ, 1);
        h->esc_smem_big = smem_plan(c.max_points, c.grid_side, h->Gp, 8, false, 512).total;
        CK(solve_occupancy(PREC_F64, false, 512, h->esc_smem_big, &occ));
        h->esc_grid_big = h->gws_grid;
    }
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
static SolveArgs make_args(gp_voxels_t* h, SolveCtx& x, const float* d_xyz,
                           const int64_t* d_offsets, int32_t nvox, const int32_t* d_nvox,
                           const float* d_centres, const float* d_lambda, const float* d_sf2,
                           const float* d_sn2, uint8_t* d_axis, float* d_mean, float* d_var,
                           uint32_t* d_status, float* d_pos, float* d_scale, float* d_quat,
                           const float* d_noise = nullptr, float* d_pvar = nullptr,
                           const uint8_t* d_skip = nullptr)
{
    const gp_voxels_config& c = h->cfg;
    const int kind = prec_kind(c.precision);
    SolveArgs a;
    memset(&a, 0, sizeof(a));
    a.xyz = d_xyz; a.offsets = d_offsets; a.centres = d_centres;
    a.lam = d_lambda; a.sf2 = d_sf2; a.sn2 = d_sn2; a.nvox = nvox; a.nvox_dev = d_nvox;
    a.size = c.voxel_size; a.G = c.grid_side; a.Gp = h->Gp; a.n_s = c.n_s; a.n_r = c.n_r;
    a.tau = c.tau; a.mean_mode = c.mean_mode; a.init_mode = c.init_mode;
    a.esc_cond = c.esc_cond;
    a.escalate = kind == PREC_FF ? 1 : 0;
    a.refine = kind == PREC_F32 ? c.refine : 0;
    a.axis = d_axis; a.mean = d_mean; a.var = d_var; a.status = d_status;
    a.pos = d_pos; a.scale = d_scale; a.quat = d_quat;
    a.noise = d_noise; a.pvar = d_pvar; a.skip = d_skip;
    a.esc_list = x.d_esc_list; a.esc_count = x.d_esc_count;
    a.gws = x.d_gws; a.gws_stride = h->gws_stride;
    a.max_points = c.max_points;
    a.nmax_small_f64 = std::min(h->plan[PREC_F64].nmax_smem, c.max_points);
    if (kind == PREC_FF && x.tc_cap > 0 && h->plan[PREC_FF].tc_nmax > 0) {
        a.tc_ws = x.d_tc_ws;
        a.tc_cap = x.tc_cap;
        a.tc = x.d_tc;
        a.tc_v = x.d_tc_v;
        a.tc_off = x.d_tc_off;
        a.tc_fb = x.d_tc_fb;
        a.fb_nsmall = h->plan[PREC_FF].nmax_smem;
        a.tc_off_v = x.d_tc_off_v;
        a.tc_nmax = h->plan[PREC_FF].tc_nmax;
        a.tc_nmax_gl = h->plan[PREC_FF].tc_nmax_gl;
        // voxels of the tall-matrix path form their variance themselves
        if (x.d_tall) a.tc_nmax_gl = std::min(a.tc_nmax_gl, h->tall_min);
    }
    return a;
}

// An event record that also works inside a stream capture (it then becomes a node of the
// graph, recorded at every replay).
static cudaError_t record_event(cudaEvent_t e, cudaStream_t s)
{
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaError_t r = cudaStreamIsCapturing(s, &cs);
    if (r != cudaSuccess) return r;
    return cudaEventRecordWithFlags(e, s, cs == cudaStreamCaptureStatusActive ? cudaEventRecordExternal
                                                                                : cudaEventRecordDefault);
}

static int gpv_solve_queue(gp_voxels_t* h, SolveCtx& x, const float* d_xyz,
                           const int64_t* d_offsets, int32_t nvox, const int32_t* d_nvox,
                           const float* d_centres, const float* d_lambda, const float* d_sf2,
                           const float* d_sn2, uint8_t* d_axis, float* d_mean, float* d_var,
                           uint32_t* d_status, float* d_pos, float* d_scale, float* d_quat,
                           uint32_t flags, cudaStream_t s, const float* d_noise = nullptr,
                           float* d_pvar = nullptr, const uint8_t* d_skip = nullptr)
{
    const gp_voxels_config& c = h->cfg;
    const int kind = prec_kind(c.precision);
    const PrecPlan& P = h->plan[kind];
    SolveArgs a = make_args(h, x, d_xyz, d_offsets, nvox, d_nvox, d_centres, d_lambda, d_sf2,
                            d_sn2, d_axis, d_mean, d_var, d_status, d_pos, d_scale, d_quat,
                            d_noise, d_pvar, d_skip);
    CK(launch_classify(a, P.d_hi, P.nb, x.d_bcount, x.d_bbase, x.d_bcursor, x.d_work,
                       x.d_next, x.d_esc_count, s));
    h->last_launches = 3;  // classify, bucket offsets, scatter
    if (nvox == 0) return GPV_OK;

    if (flags & GPV_SOLVE_ONE_PER_LAUNCH) {
        // Baseline: one launch per voxel, sized for that voxel.
        std::vector<int64_t> off((size_t)nvox + 1);
        CK(cudaMemcpyAsync(off.data(), d_offsets, sizeof(int64_t) * (nvox + 1), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        CK(cudaMemsetAsync(h->d_pl_next, 0, sizeof(int32_t) * nvox, s));
        a.escalate = 0;
        a.tc_ws = nullptr;  // each launch forms its own variance
        a.work_count = h->d_one;
        a.work_base = nullptr;
        for (int32_t v = 0; v < nvox; ++v) {
            const int64_t n = off[v + 1] - off[v];
            if (n < c.tau || n <= 0 || n > c.max_points) continue;
            a.work = h->d_ident + v;
            a.work_next = h->d_pl_next + v;
            // the launch configuration of the voxel's size bucket, one CTA
            int b = P.nb - 1;
            for (int k = 0; k < P.nb; ++k)
                if (n <= P.b[k].hi) { b = k; break; }
            const Bucket& B = P.b[b];
            a.nmax = B.tri_smem ? B.hi : c.max_points;
            a.percol_max = B.percol ? B.hi : 0;
            a.panel = B.panel;
            CK(launch_solve(kind, B.tri_smem, B.nthr, a, 1, B.smem, s));
            ++h->last_launches;
        }
        return GPV_OK;
    }

    if (a.tc_ws) {  // no row handed over yet; per-bucket dequeue counters of k_var_tc
        CK(cudaMemsetAsync(a.tc_off_v, 0xFF, sizeof(long long) * (size_t)nvox, s));
        CK(cudaMemsetAsync(x.d_tc_next, 0, sizeof(int32_t) * kNumBuckets, s));
    }
    // Batched: one persistent launch per size bucket, buckets on forked streams.
    // Buckets whose factor lives in the global workspace share it, so they run
    // one after another on the first side stream.
    CK(cudaEventRecord(x.ev_fork, s));
    int used = 0;
    bool timed = false;               // events around the tall-matrix launches recorded
    cudaStream_t tall_ss = nullptr;
    for (int b = P.nb - 1; b >= 0; --b) {
        const Bucket& B = P.b[b];
        const bool tcv = a.tc_ws && B.tcv_ok;  // the variant, factor in shared memory
        const int si = (B.tri_smem || tcv) ? 1 + b : 0;
        cudaStream_t ss = x.side[si % kNumBuckets];
        CK(cudaStreamWaitEvent(ss, x.ev_fork, 0));
        a.work = x.d_work;
        a.work_base = x.d_bbase + b;
        a.work_count = x.d_bcount + b;
        a.work_next = x.d_next + b;
        a.nmax = (B.tri_smem || tcv) ? B.hi : c.max_points;
        if (B.tall && x.d_tall && !a.pvar) {  // large voxels: the tall-matrix factorisation
            if (tall_ss) continue;  // drained by the launch of the largest tall bucket
            // one persistent launch drains every tall bucket, largest voxels first
            int blo = b;
            while (blo > 0 && P.b[blo - 1].tall) --blo;
            if (h->timing && &x == &h->main && !timed) {
                CK(record_event(h->ev_tall[0], ss));
                timed = true;
            }
            SolveArgs at = a;
            at.work_base = x.d_bbase + blo;
            at.work_count = x.d_bcount + blo;
            at.work_next = x.d_next + blo;
            at.nqueues = b - blo + 1;
            CK(launch_tall(kind, at, x.d_tall, h->tall_stride, (B.hi + 31) / 32 * 32, h->sms, ss));
            tall_ss = ss;
        } else if (tcv) {  // the variance goes to the tensor cores
            a.percol_max = B.v.percol ? B.hi : 0;
            a.panel = B.v.panel;
            CK(launch_solve(kind, true, B.v.nthr, a, B.v.grid, B.v.smem, ss, true));
            ++h->last_launches;
            SolveArgs av = a;  // then the bucket's variances, on the same stream
            av.work_next = x.d_tc_next + b;
            CK(launch_var_tc(av, h->sms, ss));
        } else {
            a.percol_max = B.percol ? B.hi : 0;
            a.panel = B.panel;
            CK(launch_solve(kind, B.tri_smem, B.nthr, a, B.grid, B.smem, ss));
            if (a.tc_ws && !B.tri_smem && P.tc_nmax_gl > P.nmax_smem) {
                // workspace voxels hand their variance over as well
                ++h->last_launches;
                SolveArgs av = a;
                av.work_next = x.d_tc_next + b;
                CK(launch_var_tc(av, h->sms, ss));
            }
        }
        ++h->last_launches;
        used |= 1 << (si % kNumBuckets);
    }
    if (timed) CK(record_event(h->ev_tall[1], tall_ss));
    if (&x == &h->main) h->timed_tall = timed;
    for (int i = 0; i < kNumBuckets; ++i)
        if (used & (1 << i)) {
            CK(cudaEventRecord(x.ev_join[i], x.side[i]));
            CK(cudaStreamWaitEvent(s, x.ev_join[i], 0));
        }
    if (a.tc_ws) {  // variance and Gaussians of the voxels the buckets queued
        {   // voxels the variant could not hand over (workspace full): regular re-solve
            SolveArgs f = a;
            f.tc_ws = nullptr;
            f.work = a.tc_fb;
            f.work_base = nullptr;
            f.work_count = &a.tc->fb_count;
            f.work_next = &a.tc->fb_next;
            f.nmax = P.nmax_smem;
            f.percol_max = default_percol_max(8);
            f.panel = 16;
            CK(launch_solve(kind, true, P.fb_nthr, f, P.fb_grid, P.fb_smem, s));
            ++h->last_launches;
            if (P.tc_nmax > P.nmax_smem) {  // and those beyond the shared-memory kernels
                f.work = a.tc_fb + nvox;
                f.work_count = &a.tc->fb2_count;
                f.work_next = &a.tc->fb2_next;
                if (x.d_tall && !a.pvar) {
                    CK(launch_tall(kind, f, x.d_tall, h->tall_stride, (P.tc_nmax + 31) / 32 * 32,
                                   h->sms, s));
                } else {
                    f.nmax = c.max_points;
                    CK(launch_solve(kind, false, 512, f, P.fbb_grid, P.fbb_smem, s));
                }
                ++h->last_launches;
            }
        }
        if (a.pos) {
            CK(launch_init_tc(a, h->sms, s));
            ++h->last_launches;
        }
    }
    if (kind == PREC_FF) {
        // FP64 re-solve of the voxels that failed the conditioning check
        a.escalate = 0;
        a.escalation_pass = 1;
        a.work = x.d_esc_list;
        a.work_base = nullptr;
        a.work_count = x.d_esc_count;
        a.work_next = x.d_next + P.nb;
        a.nmax = a.nmax_small_f64;
        a.percol_max = default_percol_max(8);
        a.panel = 16;
        CK(launch_solve(PREC_F64, true, solve_threads(a.nmax, true), a, h->esc_grid_small,
                        h->esc_smem_small, s));
        ++h->last_launches;
        if (c.max_points > a.nmax_small_f64) {
            a.work = x.d_esc_list + nvox;
            a.work_count = x.d_esc_count + 1;
            a.work_next = x.d_next + P.nb + 1;
            a.nmax = c.max_points;
            CK(launch_solve(PREC_F64, false, 512, a, h->esc_grid_big, h->esc_smem_big, s));
            ++h->last_launches;
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
    return gp_voxels_solve_csr_noise(h, d_xyz, d_offsets, nvox, d_centres, d_lambda, d_sf2,
                                     d_sn2, nullptr, d_axis, d_mean, d_var, d_status, d_pos,
                                     d_scale, d_quat, nullptr, flags, stream);
}

extern "C" int gp_voxels_solve_csr_noise(gp_voxels_t* h, const float* d_xyz,
                                         const int64_t* d_offsets, int32_t nvox,
                                         const float* d_centres, const float* d_lambda,
                                         const float* d_sf2, const float* d_sn2,
                                         const float* d_noise, uint8_t* d_axis, float* d_mean,
                                         float* d_var, uint32_t* d_status, float* d_pos,
                                         float* d_scale, float* d_quat, float* d_pvar,
                                         uint32_t flags, gpv_stream_t stream)
{
    if (!h || nvox < 0 || nvox > h->cfg.max_voxels) return GPV_EINVAL;
    if (nvox == 0) return GPV_OK;  // nothing to read or write
    if (!d_offsets || !d_axis || !d_mean || !d_var || !d_status) return GPV_EINVAL;
    if (nvox > 0 && (!d_xyz || !d_centres || !d_lambda || !d_sf2 || !d_sn2)) return GPV_EINVAL;
    const bool any_init = d_pos || d_scale || d_quat;
    if (any_init && !(d_pos && d_scale && d_quat)) return GPV_EINVAL;
    if (flags & ~(uint32_t)GPV_SOLVE_ONE_PER_LAUNCH) return GPV_EINVAL;
    return gpv_solve_queue(h, h->main, d_xyz, d_offsets, nvox, nullptr, d_centres, d_lambda,
                           d_sf2, d_sn2, d_axis, d_mean, d_var, d_status, d_pos, d_scale, d_quat,
                           flags, (cudaStream_t)stream, d_noise, d_pvar, nullptr);
}

// Workspace of the Alg. 3 path: k_k* (two TF32 halves, in tensor-core operand tiles) and
// the K* factors of `chunk` voxels; the chunk is sized to about 512 MB.
static int alg3_workspace(gp_voxels_t* h)
{
    if (h->a3.pk) return GPV_OK;
    const gp_voxels_config& c = h->cfg;
    const int G = c.grid_side, Q = G * G;
    // every voxel up to max_points: ky in shared memory up to nsm points, in a global slice
    // per CTA of the persistent class above
    const int nsm = std::min(c.max_points, alg3_max_n(G));
    const int nmax = c.max_points;
    if (nmax < c.tau) return GPV_EINVAL;
    const int kp = (nmax + 31) / 32 * 32;
    const int qp = (Q + 127) / 128 * 128;
    const size_t tfb = (size_t)(kp / 16) * 2 * G * 20 * 4;  // K* factors per 16-point chunk
    const size_t per = (size_t)2 * qp * kp * 4 + (size_t)2 * kp * G * 4 + tfb + 8;
    int chunk = (int)std::min<size_t>((size_t)c.max_voxels, std::max<size_t>(1, ((size_t)512 << 20) / per));
    const size_t bigA = nmax > nsm ? (size_t)alg3_big_ctas() * kp * kp * 4 : 0;
    const size_t need = per * (size_t)chunk + bigA;
    if (c.mem_budget && h->bytes + need > c.mem_budget) return GPV_EBUDGET;
    auto al = [&](void** p, size_t b) -> int {
        cudaError_t e = cudaMalloc(p, b);
        if (e == cudaErrorMemoryAllocation) { cudaGetLastError(); return GPV_ENOMEM; }
        if (e != cudaSuccess) return cuda_fail(e);
        h->bytes += b;
        return GPV_OK;
    };
    int rc;
    if ((rc = al((void**)&h->a3.pk, (size_t)chunk * 2 * qp * kp * 4)) != GPV_OK) return rc;
    if ((rc = al((void**)&h->a3.tf, (size_t)chunk * tfb)) != GPV_OK) return rc;
    if ((rc = al((void**)&h->a3.fa, (size_t)chunk * kp * G * 4)) != GPV_OK) return rc;
    if ((rc = al((void**)&h->a3.fb, (size_t)chunk * kp * G * 4)) != GPV_OK) return rc;
    if ((rc = al((void**)&h->a3.st, (size_t)chunk * 4)) != GPV_OK) return rc;
    if ((rc = al((void**)&h->a3.n, (size_t)chunk * 4)) != GPV_OK) return rc;
    if (bigA && (rc = al((void**)&h->a3.A, bigA)) != GPV_OK) return rc;
    if ((rc = al((void**)&h->a3.vidx, (size_t)c.max_voxels * 4)) != GPV_OK) return rc;
    if ((rc = al((void**)&h->a3.counts, 8)) != GPV_OK) return rc;
    cudaError_t e = cudaStreamCreateWithFlags(&h->a3.side, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->a3.ev_fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->a3.ev_join, cudaEventDisableTiming);
    if (e != cudaSuccess) return cuda_fail(e);
    h->a3.nmax = nmax;
    h->a3.nsm = nsm;
    h->a3.kp = kp;
    h->a3.qp = qp;
    h->a3.chunk = chunk;
    return GPV_OK;
}

extern "C" int gp_voxels_solve_alg3(gp_voxels_t* h, const float* d_xyz, const int64_t* d_offsets,
                                    int32_t nvox, const float* d_centres, const float* d_lambda,
                                    const float* d_sf2, const float* d_sn2, uint8_t* d_axis,
                                    float* d_mean, float* d_cov, uint32_t* d_status,
                                    gpv_stream_t stream, int32_t* h_nmax)
{
    if (!h || nvox < 0 || nvox > h->cfg.max_voxels) return GPV_EINVAL;
    int rc = alg3_workspace(h);
    if (rc != GPV_OK) return rc;
    if (h_nmax) *h_nmax = h->a3.nmax;
    if (nvox == 0) return GPV_OK;
    if (!d_xyz || !d_offsets || !d_centres || !d_lambda || !d_sf2 || !d_sn2 || !d_axis ||
        !d_mean || !d_cov || !d_status)
        return GPV_EINVAL;
    const gp_voxels_config& c = h->cfg;
    Alg3Args a;
    memset(&a, 0, sizeof(a));
    a.xyz = d_xyz; a.offsets = d_offsets; a.centres = d_centres;
    a.lam = d_lambda; a.sf2 = d_sf2; a.sn2 = d_sn2;
    a.size = c.voxel_size; a.G = c.grid_side; a.tau = c.tau; a.mean_mode = c.mean_mode;
    a.nmax = h->a3.nmax; a.nsm = h->a3.nsm; a.kp = h->a3.kp; a.ws_A = h->a3.A;
    a.axis = d_axis; a.mean = d_mean; a.cov = d_cov; a.status = d_status;
    a.qp = h->a3.qp;
    a.ws_pk = h->a3.pk; a.ws_tf = h->a3.tf; a.ws_fa = h->a3.fa; a.ws_fb = h->a3.fb;
    a.ws_status = h->a3.st; a.ws_n = h->a3.n;
    // voxels beyond shared memory first: they share the first chunks, where their
    // kernel runs beside the shared-memory classes
    cudaStream_t s = (cudaStream_t)stream;
    CK(cudaMemsetAsync(h->a3.counts, 0, 8, s));
    CK(alg3_order(d_offsets, nvox, h->a3.nsm, h->a3.nmax, c.tau, h->a3.vidx, h->a3.counts, s));
    a.vidx = h->a3.vidx;
    h->last_launches = 1;
    for (int32_t s0 = 0; s0 < nvox; s0 += h->a3.chunk) {
        a.s0 = s0;
        int nl = 0;
        CK(alg3_launch_chunk(a, std::min(h->a3.chunk, nvox - s0), s, h->a3.side, h->a3.ev_fork,
                             h->a3.ev_join, &nl));
        h->last_launches += nl;
    }
    return GPV_OK;
}

static constexpr int kLpPartial = 1024;

// (Re)allocate the loss workspace for m Gaussians and n points.
static int lp_workspace(gp_voxels_t* h, int32_t m, int32_t n)
{
    auto& w = h->lp;
    if (m <= w.mcap && n <= w.ncap && w.keys) return GPV_OK;
    const int32_t mc = std::max(m, w.mcap), nc = std::max(n, w.ncap);
    uint32_t H = 1024;
    while (H < 2u * (uint32_t)std::max(mc, 1)) H <<= 1;
    cudaDeviceSynchronize();
    cudaFree(w.keys); cudaFree(w.head); cudaFree(w.next); cudaFree(w.pending);
    cudaFree(w.counters); cudaFree(w.arg); cudaFree(w.best); cudaFree(w.smax); cudaFree(w.partial);
    w = gp_voxels::LpWork();
    const size_t need = (size_t)H * 12 + (size_t)mc * 4 + (size_t)nc * 12 + 64 + kLpPartial * 8;
    if (h->cfg.mem_budget && h->bytes + need > h->cfg.mem_budget) return GPV_EBUDGET;
    auto al = [&](void** p, size_t b) -> int {
        cudaError_t e = cudaMalloc(p, b);
        if (e == cudaErrorMemoryAllocation) { cudaGetLastError(); return GPV_ENOMEM; }
        if (e != cudaSuccess) return cuda_fail(e);
        h->bytes += b;
        return GPV_OK;
    };
    int rc;
    if ((rc = al((void**)&w.keys, (size_t)H * 8)) != GPV_OK) return rc;
    if ((rc = al((void**)&w.head, (size_t)H * 4)) != GPV_OK) return rc;
    if ((rc = al((void**)&w.next, (size_t)std::max(mc, 1) * 4)) != GPV_OK) return rc;
    if ((rc = al((void**)&w.pending, (size_t)std::max(nc, 1) * 4)) != GPV_OK) return rc;
    if ((rc = al((void**)&w.arg, (size_t)std::max(nc, 1) * 4)) != GPV_OK) return rc;
    if ((rc = al((void**)&w.best, (size_t)std::max(nc, 1) * 4)) != GPV_OK) return rc;
    if ((rc = al((void**)&w.counters, 16)) != GPV_OK) return rc;
    if ((rc = al((void**)&w.smax, 16)) != GPV_OK) return rc;
    if ((rc = al((void**)&w.partial, kLpPartial * 8)) != GPV_OK) return rc;
    w.mcap = mc;
    w.ncap = nc;
    w.H = H;
    return GPV_OK;
}

extern "C" int gp_voxels_structure_loss(gp_voxels_t* h, const float* d_gpos,
                                        const float* d_gscale, int32_t m, const float* d_points,
                                        int32_t n, float cell, float* d_best, int32_t* d_arg,
                                        double* d_loss, int32_t* d_info, gpv_stream_t stream)
{
    if (!h || m < 1 || n < 0 || !(cell > 0.f) || !d_gpos || !d_gscale || !d_loss) return GPV_EINVAL;
    if (n > 0 && !d_points) return GPV_EINVAL;
    int rc = lp_workspace(h, m, n);
    if (rc != GPV_OK) return rc;
    auto& w = h->lp;
    LpArgs a;
    memset(&a, 0, sizeof(a));
    a.pts = d_points; a.n = n; a.gpos = d_gpos; a.gscale = d_gscale; a.m = m; a.h = cell;
    a.H = w.H; a.keys = w.keys; a.head = w.head; a.next = w.next; a.pending = w.pending;
    a.counters = w.counters; a.smax = w.smax; a.partial = w.partial;
    a.nb_partial = std::max(1, std::min(kLpPartial, (n + 255) / 256));
    a.sms = h->sms;
    a.best = d_best ? d_best : w.best;
    a.arg = d_arg ? d_arg : w.arg;
    a.loss = d_loss;
    cudaStream_t s = (cudaStream_t)stream;
    int nl = 0;
    CK(lp_launch(a, s, &nl));
    if (d_info) CK(cudaMemcpyAsync(d_info, w.counters, 8, cudaMemcpyDeviceToDevice, s));
    h->last_launches = nl;
    return GPV_OK;
}

static int dev_alloc(gp_voxels_t* h, void** p, size_t b)
{
    cudaError_t e = cudaMalloc(p, b);
    if (e == cudaErrorMemoryAllocation) { cudaGetLastError(); return GPV_ENOMEM; }
    if (e != cudaSuccess) return cuda_fail(e);
    h->bytes += b;
    return GPV_OK;
}

extern "C" int gp_voxels_render(gp_voxels_t* h, const float* d_pos, const float* d_scale,
                                const float* d_quat, const float* d_opacity,
                                const float* d_color, int32_t m, const gp_raster_camera* cam,
                                float* d_image, float* d_depth, float* d_silhouette,
                                gpv_stream_t stream, int64_t* h_pairs)
{
    if (!h || !cam || m < 0 || !d_image || !d_depth || !d_silhouette) return GPV_EINVAL;
    if (m > 0 && (!d_pos || !d_scale || !d_quat || !d_opacity || !d_color)) return GPV_EINVAL;
    if (cam->width < 1 || cam->height < 1 || cam->width > 16384 || cam->height > 16384 ||
        !(cam->fx > 0.f) || !(cam->fy > 0.f) || !(cam->near > 0.f))
        return GPV_EINVAL;
    auto& w = h->rs;
    const int tx = (cam->width + 15) / 16, ty = (cam->height + 15) / 16, nt = tx * ty;
    int rc;
    if (m > w.mcap || nt > w.tcap || !w.count) {
        cudaDeviceSynchronize();
        const int32_t mc = std::max(m, w.mcap), tc = std::max(nt, w.tcap);
        cudaFree(w.sp); cudaFree(w.rect); cudaFree(w.count); cudaFree(w.off); cudaFree(w.cursor);
        w.sp = nullptr; w.rect = nullptr; w.count = w.off = w.cursor = nullptr;
        w.mcap = w.tcap = 0;
        if ((rc = dev_alloc(h, (void**)&w.sp, sizeof(float4) * 3 * (size_t)std::max(mc, 1))) != GPV_OK) return rc;
        if ((rc = dev_alloc(h, (void**)&w.rect, sizeof(int4) * (size_t)std::max(mc, 1))) != GPV_OK) return rc;
        if ((rc = dev_alloc(h, (void**)&w.count, sizeof(int32_t) * (size_t)tc)) != GPV_OK) return rc;
        if ((rc = dev_alloc(h, (void**)&w.off, sizeof(int32_t) * (size_t)(tc + 1))) != GPV_OK) return rc;
        if ((rc = dev_alloc(h, (void**)&w.cursor, sizeof(int32_t) * (size_t)tc)) != GPV_OK) return rc;
        w.mcap = mc;
        w.tcap = tc;
    }
    RasterArgs a;
    memset(&a, 0, sizeof(a));
    a.pos = d_pos; a.scale = d_scale; a.quat = d_quat; a.opacity = d_opacity; a.color = d_color;
    a.m = m;
    memcpy(a.cam.R, cam->R, sizeof(a.cam.R));
    memcpy(a.cam.t, cam->t, sizeof(a.cam.t));
    a.cam.fx = cam->fx; a.cam.fy = cam->fy; a.cam.cx = cam->cx; a.cam.cy = cam->cy;
    a.cam.width = cam->width; a.cam.height = cam->height; a.cam.near = cam->near;
    a.tiles_x = tx; a.tiles_y = ty; a.ntile = nt;
    a.sp = w.sp; a.rect = w.rect; a.tile_count = w.count; a.tile_off = w.off; a.tile_cursor = w.cursor;
    a.C = d_image; a.D = d_depth; a.S = d_silhouette;
    cudaStream_t s = (cudaStream_t)stream;
    CK(raster_prepare(a, s));
    int32_t total = 0;  // the list size decides the key buffer: one host read per image
    CK(cudaMemcpyAsync(&total, w.off + nt, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (total < 0) return GPV_EFULL;  // more than 2^31 - 1 (tile, Gaussian) pairs
    if (total > w.kcap) {
        cudaFree(w.keys);
        w.keys = nullptr;
        w.kcap = 0;
        const int64_t kc = std::max<int64_t>((int64_t)total + total / 4, 1 << 16);
        if ((rc = dev_alloc(h, (void**)&w.keys, sizeof(uint64_t) * (size_t)kc)) != GPV_OK) return rc;
        w.kcap = kc;
    }
    a.keys = w.keys;
    a.cap = (int32_t)std::min<int64_t>(w.kcap, INT32_MAX);
    CK(raster_finish(a, s));
    h->last_launches = (m > 0 ? 2 : 1) + 3 + (m > 0 ? 1 : 0);
    if (h_pairs) *h_pairs = total;
    return GPV_OK;
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

// ---- serving ----------------------------------------------------------------------
extern "C" int gp_voxels_insert_scan(gp_voxels_t* h, const float* d_xyz, int64_t npts,
                                     uint64_t scan_id, gpv_stream_t stream, int32_t* slot_out)
{
    (void)scan_id;  // inserts are ordered by call order; the id is the caller's label
    if (!h || !h->store || !slot_out) return GPV_EINVAL;
    if (npts < 0 || npts > h->cfg.max_scan_points || (npts > 0 && !d_xyz)) return GPV_EINVAL;
    gpv_store* st = h->store;
    int si = -1;
    for (int i = 0; i < st->nslots; ++i)
        if (!st->slots[i].busy) { si = i; break; }
    if (si < 0) return GPV_EFULL;
    if (st->feedback && st->unsolved >= 0) return GPV_EINVAL;  // solve the previous scan first
    cudaStream_t s = (cudaStream_t)stream;
    gpv_scan_slot& S = st->slots[si];
    CK(cudaStreamWaitEvent(s, S.free_ev, 0));      // the slot's previous scan is done
    CK(cudaStreamWaitEvent(s, st->ev_insert, 0));  // inserts follow call order
    if (st->feedback) CK(cudaStreamWaitEvent(s, st->ev_fb, 0));  // types and noises are current
    CK(store_insert(st, si, d_xyz, (int)npts, s, &h->cfg));
    CK(cudaEventRecord(st->ev_insert, s));
    CK(cudaEventRecord(S.ins_ev, s));
    S.busy = true;
    if (st->feedback) st->unsolved = si;
    *slot_out = si;
    return GPV_OK;
}

extern "C" int gp_voxels_solve(gp_voxels_t* h, int32_t slot, uint8_t* d_axis, float* d_mean,
                               float* d_var, uint32_t* d_status, float* d_pos, float* d_scale,
                               float* d_quat, int64_t* d_keys, float* d_centres,
                               gpv_stream_t stream)
{
    if (!h || !h->store || slot < 0 || slot >= h->store->nslots || !h->store->slots[slot].busy)
        return GPV_EINVAL;
    if (!d_axis || !d_mean || !d_var || !d_status) return GPV_EINVAL;
    const bool any_init = d_pos || d_scale || d_quat;
    if (any_init && !(d_pos && d_scale && d_quat)) return GPV_EINVAL;
    gpv_store* st = h->store;
    gpv_scan_slot& S = st->slots[slot];
    cudaStream_t s = (cudaStream_t)stream;
    // the slot's insert may have been queued on another stream
    CK(cudaStreamWaitEvent(s, S.ins_ev, 0));
    const bool fb = st->feedback;
    int rc = gpv_solve_queue(h, h->sctx[slot], S.snap, S.snapoff, st->max_vox, S.counters,
                             S.centres, S.lam, S.sf2, S.sn2, d_axis, d_mean, d_var, d_status,
                             d_pos, d_scale, d_quat, 0, s, fb ? S.snap_noise : nullptr,
                             fb ? S.snap_pvar : nullptr, fb ? S.rskip : nullptr);
    if (rc != GPV_OK) return rc;
    CK(store_or_flags(st, slot, d_status, s));
    CK(store_copy_rows(st, slot, d_keys, d_centres, s));
    h->last_launches += 1 + ((d_keys || d_centres) ? 1 : 0);
    if (fb) {  // Sec. 3.3: noise feedback and type transitions, before the next insert
        CK(store_feedback(st, slot, d_status, d_var, &h->cfg, s));
        CK(cudaEventRecord(st->ev_fb, s));
        if (st->unsolved == slot) st->unsolved = -1;
        h->last_launches += 1;
    }
    return GPV_OK;
}

extern "C" int gp_voxels_scan_info(gp_voxels_t* h, int32_t slot, gpv_stream_t stream,
                                   int32_t* h_rows, int64_t* h_points, uint32_t* h_flags)
{
    if (!h || !h->store || slot < 0 || slot >= h->store->nslots || !h->store->slots[slot].busy)
        return GPV_EINVAL;
    gpv_scan_slot& S = h->store->slots[slot];
    cudaStream_t s = (cudaStream_t)stream;
    int32_t c[4];
    int64_t np = 0;
    CK(cudaStreamWaitEvent(s, S.ins_ev, 0));
    CK(cudaMemcpyAsync(c, S.counters, sizeof(c), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(&np, S.npoints, sizeof(np), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (h_rows) *h_rows = c[0];
    if (h_points) *h_points = np < h->store->snap_cap ? np : h->store->snap_cap;
    if (h_flags) *h_flags = (uint32_t)c[1];
    return GPV_OK;
}

extern "C" int gp_voxels_release_scan(gp_voxels_t* h, int32_t slot, gpv_stream_t stream)
{
    if (!h || !h->store || slot < 0 || slot >= h->store->nslots || !h->store->slots[slot].busy)
        return GPV_EINVAL;
    gpv_scan_slot& S = h->store->slots[slot];
    CK(cudaEventRecord(S.free_ev, (cudaStream_t)stream));
    S.busy = false;
    if (h->store->unsolved == slot) h->store->unsolved = -1;  // released unsolved: no update
    return GPV_OK;
}

extern "C" int gp_voxels_scan_types(gp_voxels_t* h, int32_t slot, uint8_t* d_before,
                                    uint8_t* d_after, gpv_stream_t stream)
{
    if (!h || !h->store || !h->store->feedback || slot < 0 || slot >= h->store->nslots ||
        !h->store->slots[slot].busy)
        return GPV_EINVAL;
    if (!d_before && !d_after) return GPV_OK;
    CK(store_copy_types(h->store, slot, d_before, d_after, (cudaStream_t)stream));
    return GPV_OK;
}

extern "C" int gp_voxels_type_counts(gp_voxels_t* h, int64_t* h_counts)
{
    if (!h || !h->store || !h_counts) return GPV_EINVAL;
    unsigned long long* d = nullptr;
    CK(cudaDeviceSynchronize());
    CK(cudaMalloc(&d, 4 * sizeof(unsigned long long)));
    cudaError_t e = store_type_counts(h->store, h->cfg.tau, d, 0);
    unsigned long long c[4] = {0, 0, 0, 0};
    if (e == cudaSuccess) e = cudaMemcpy(c, d, sizeof(c), cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess) return cuda_fail(e);
    for (int i = 0; i < 4; ++i) h_counts[i] = (int64_t)c[i];
    return GPV_OK;
}

extern "C" int gp_voxels_store_voxels(gp_voxels_t* h, int64_t* h_voxels)
{
    if (!h || !h->store || !h_voxels) return GPV_EINVAL;
    int32_t n = 0;
    CK(cudaDeviceSynchronize());
    CK(cudaMemcpy(&n, h->store->nvox, sizeof(n), cudaMemcpyDeviceToHost));
    *h_voxels = n;
    return GPV_OK;
}

extern "C" int gp_voxels_autotune(gp_voxels_t* h, const float* d_xyz, const int64_t* d_offsets,
                                  int32_t nvox, const float* d_centres, const float* d_lambda,
                                  const float* d_sf2, const float* d_sn2, uint8_t* d_axis,
                                  float* d_mean, float* d_var, uint32_t* d_status, float* d_pos,
                                  float* d_scale, float* d_quat, gpv_stream_t stream,
                                  int32_t* h_changed)
{
    if (!h || nvox <= 0 || nvox > h->cfg.max_voxels || !h_changed) return GPV_EINVAL;
    if (!d_xyz || !d_offsets || !d_centres || !d_lambda || !d_sf2 || !d_sn2 || !d_axis ||
        !d_mean || !d_var || !d_status)
        return GPV_EINVAL;
    const bool any_init = d_pos || d_scale || d_quat;
    if (any_init && !(d_pos && d_scale && d_quat)) return GPV_EINVAL;
    const gp_voxels_config& c = h->cfg;
    const int kind = prec_kind(c.precision);
    PrecPlan& P = h->plan[kind];
    SolveCtx& x = h->main;
    cudaStream_t s = (cudaStream_t)stream;
    SolveArgs a = make_args(h, x, d_xyz, d_offsets, nvox, nullptr, d_centres, d_lambda, d_sf2,
                            d_sn2, d_axis, d_mean, d_var, d_status, d_pos, d_scale, d_quat);
    a.escalate = 0;  // time every voxel in this precision
    CK(launch_classify(a, P.d_hi, P.nb, x.d_bcount, x.d_bbase, x.d_bcursor, x.d_work, x.d_next,
                       x.d_esc_count, s));
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    int changed = 0;
    const int cand[5] = {32, 64, 128, 256, 512};
    // The shared-memory buckets of a solve run at once on their own streams, so a
    // candidate is timed with all of them: bucket bc in the candidate's configuration,
    // the others in their current one (each followed by its tensor-core variances).
    auto launch_group = [&](int bc, int nt_c, bool pc_c, int pw_c, int smem_c, int grid_c,
                            cudaEvent_t ev_start) -> int {
        CK(cudaMemsetAsync(x.d_next, 0, sizeof(int32_t) * kNumBuckets, s));
        if (a.tc) {  // every timed run starts from an empty workspace
            CK(cudaMemsetAsync(reinterpret_cast<unsigned char*>(a.tc) + 8, 0, sizeof(TcCounters) - 8, s));
            CK(cudaMemsetAsync(x.d_tc_next, 0, sizeof(int32_t) * kNumBuckets, s));
            CK(cudaMemsetAsync(a.tc_off_v, 0xFF, sizeof(long long) * (size_t)nvox, s));
        }
        CK(cudaEventRecord(ev_start, s));
        CK(cudaEventRecord(x.ev_fork, s));
        int used = 0;
        for (int b2 = P.nb - 1; b2 >= 0; --b2) {
            const Bucket& B2 = P.b[b2];
            if (B2.tall && h->main.d_tall) continue;
            const bool tcv2 = a.tc_ws && B2.tcv_ok;
            if (!(B2.tri_smem || tcv2)) continue;
            const int si = (1 + b2) % kNumBuckets;
            cudaStream_t ss = x.side[si];
            CK(cudaStreamWaitEvent(ss, x.ev_fork, 0));
            SolveArgs a2 = a;
            a2.work = x.d_work;
            a2.work_base = x.d_bbase + b2;
            a2.work_count = x.d_bcount + b2;
            a2.work_next = x.d_next + b2;
            a2.nmax = B2.hi;
            const bool mine = b2 == bc;
            const int nt2 = mine ? nt_c : (tcv2 ? B2.v.nthr : B2.nthr);
            const bool pc2 = mine ? pc_c : (tcv2 ? B2.v.percol : B2.percol);
            const int pw2 = mine ? pw_c : (tcv2 ? B2.v.panel : B2.panel);
            const int sm2 = mine ? smem_c : (tcv2 ? B2.v.smem : B2.smem);
            const int gr2 = mine ? grid_c : (tcv2 ? B2.v.grid : B2.grid);
            a2.percol_max = pc2 ? B2.hi : 0;
            a2.panel = pw2;
            CK(launch_solve(kind, true, nt2, a2, gr2, sm2, ss, tcv2));
            if (tcv2) {
                SolveArgs av = a2;
                av.work_next = x.d_tc_next + b2;
                CK(launch_var_tc(av, h->sms, ss));
            }
            used |= 1 << si;
        }
        for (int i = 0; i < kNumBuckets; ++i)
            if (used & (1 << i)) {
                CK(cudaEventRecord(x.ev_join[i], x.side[i]));
                CK(cudaStreamWaitEvent(s, x.ev_join[i], 0));
            }
        return GPV_OK;
    };
    for (int b = 0; b < P.nb; ++b) {
        Bucket& B = P.b[b];
        if (B.tall && h->main.d_tall) continue;  // one launch shape: one CTA of 384 threads per SM
        const bool tcv = a.tc_ws && B.tcv_ok;  // tune the variant the batch entry launches
        const bool tri = B.tri_smem || tcv;     // its factor is in shared memory
        float best_ms = 3.0e38f;
        int best = tcv ? B.v.nthr : B.nthr, best_smem = tcv ? B.v.smem : B.smem;
        int best_grid = tcv ? B.v.grid : B.grid;
        bool best_pc = tcv ? B.v.percol : B.percol;
        int best_pw = tcv ? B.v.panel : B.panel;
        const int cur = best;
        const bool cur_pc = best_pc;
        const int cur_pw = best_pw;
        float cur_ms = 3.0e38f;
        for (int ci = 0; ci < 20; ++ci) {
            const int nt = cand[ci % 5];
            const int var = ci / 5;  // blocked with 16-, 8- or 4-column panels, or per column
            const bool pc = var == 3;
            const int pw = var == 0 ? 16 : (var == 1 ? 8 : 4);
            if (var > 0 && !tri) continue;  // variants of the shared-memory factor
            if (tri && nt < B.hi) continue;  // the shared-memory variants need n <= CTA size
            if (!tri && nt < 256) continue;
            const SmemPlan sp = smem_plan(tri ? B.hi : c.max_points, c.grid_side, h->Gp,
                                          tsize(kind), tri, nt, tcv);
            if (!tri && (sp.pb < 4 || sp.rb < 4)) continue;
            int occ = 0;
            CK(solve_occupancy(kind, tri, nt, sp.total, &occ, tcv));
            if (occ < 1) continue;
            const int grid = tri ? h->sms * occ : h->gws_grid;
            a.work = x.d_work;
            a.work_base = x.d_bbase + b;
            a.work_count = x.d_bcount + b;
            a.work_next = x.d_next + b;
            a.nmax = tri ? B.hi : c.max_points;
            a.percol_max = pc ? B.hi : 0;
            a.panel = pw;
            float ms = 3.0e38f;
            for (int rep = 0; rep < 2; ++rep) {  // the first run also loads the kernel
                CK(cudaMemsetAsync(x.d_next + b, 0, sizeof(int32_t), s));
                if (a.tc) {  // each timed launch starts from an empty workspace
                    CK(cudaMemsetAsync(reinterpret_cast<unsigned char*>(a.tc) + 8, 0,
                                       sizeof(TcCounters) - 8, s));
                    CK(cudaMemsetAsync(x.d_tc_next + b, 0, sizeof(int32_t), s));
                    // no voxel handed over yet: k_var_tc skips the ones this run keeps
                    CK(cudaMemsetAsync(a.tc_off_v, 0xFF, sizeof(long long) * (size_t)nvox, s));
                }
                if (tri) {
                    const int rc = launch_group(b, nt, pc, pw, sp.total, grid, e0);
                    if (rc != GPV_OK) return rc;
                } else {
                    CK(cudaEventRecord(e0, s));
                    CK(launch_solve(kind, tri, nt, a, grid, sp.total, s, tcv));
                }
                CK(cudaEventRecord(e1, s));
                CK(cudaEventSynchronize(e1));
                float t = 0.f;
                CK(cudaEventElapsedTime(&t, e0, e1));
                ms = std::min(ms, t);
            }
            if (nt == cur && pc == cur_pc && pw == cur_pw) cur_ms = ms;
            if (ms < best_ms) {
                best_ms = ms; best = nt; best_smem = sp.total; best_grid = grid; best_pc = pc;
                best_pw = pw;
            }
        }
        // a change must beat the default by more than the timing noise of a lone bucket
        if (best_ms > 0.98f * cur_ms) {
            best = cur; best_pc = cur_pc; best_pw = cur_pw;
            best_smem = tcv ? B.v.smem : B.smem;
            best_grid = tcv ? B.v.grid : B.grid;
        }
        if (best != cur || best_pc != cur_pc || best_pw != cur_pw) ++changed;
        if (tcv) {
            B.v.percol = best_pc; B.v.panel = best_pw; B.v.nthr = best; B.v.smem = best_smem;
            B.v.grid = best_grid;
        } else {
            B.percol = best_pc; B.panel = best_pw; B.nthr = best; B.smem = best_smem;
            B.grid = best_grid;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *h_changed = changed;
    return GPV_OK;
}

extern "C" int gp_voxels_plan_info(const gp_voxels_t* h, int32_t* h_info)
{
    if (!h || !h_info) return GPV_EINVAL;
    const PrecPlan& P = h->plan[prec_kind(h->cfg.precision)];
    h_info[0] = h->tall_min == INT_MAX ? -1 : h->tall_min;
    h_info[1] = P.tc_nmax;
    h_info[2] = P.nmax_smem;
    h_info[3] = P.nb;
    return GPV_OK;
}

extern "C" int gp_voxels_bucket_info(const gp_voxels_t* h, int32_t* h_info, int32_t cap,
                                     int32_t* h_count)
{
    if (!h || !h_info || !h_count || cap < 0) return GPV_EINVAL;
    const PrecPlan& P = h->plan[prec_kind(h->cfg.precision)];
    const bool tc = h->main.tc_cap > 0;
    for (int b = 0; b < P.nb && b < cap; ++b) {
        const Bucket& B = P.b[b];
        const bool tall = B.tall && h->main.d_tall;
        const bool tcv = !tall && tc && B.tcv_ok;
        int32_t* o = h_info + 5 * b;
        o[0] = B.hi;
        o[1] = tall ? 2 : (tcv ? 3 : (B.tri_smem ? 0 : 1));
        o[2] = tall ? 384 : (tcv ? B.v.nthr : B.nthr);
        o[3] = tall ? 0 : (int)(tcv ? B.v.percol : B.percol);
        o[4] = tall ? 32 : (tcv ? B.v.panel : B.panel);
    }
    *h_count = P.nb;
    return GPV_OK;
}

extern "C" int gp_voxels_set_timing(gp_voxels_t* h, int32_t on)
{
    if (!h) return GPV_EINVAL;
    if (on && !h->ev_tall[0]) {
        CK(cudaEventCreate(&h->ev_tall[0]));
        CK(cudaEventCreate(&h->ev_tall[1]));
    }
    h->timing = on != 0;
    h->timed_tall = false;
    return GPV_OK;
}

extern "C" int gp_voxels_last_tall_ms(gp_voxels_t* h, float* h_ms)
{
    if (!h || !h_ms) return GPV_EINVAL;
    *h_ms = 0.f;
    if (!h->timed_tall || !h->ev_tall[0]) return GPV_OK;
    CK(cudaEventSynchronize(h->ev_tall[1]));
    CK(cudaEventElapsedTime(h_ms, h->ev_tall[0], h->ev_tall[1]));
    return GPV_OK;
}

extern "C" int gp_voxels_last_launches(const gp_voxels_t* h, int32_t* h_kernels)
{
    if (!h || !h_kernels) return GPV_EINVAL;
    *h_kernels = h->last_launches;
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

void gpv::gpv_record_cuda_error(cudaError_t e) { cuda_fail(e); }
