// gpv_noalloc.cu -- gp_voxels_solve_csr_noalloc: the batched Voxel-GPR solve for callers
// that cannot allocate device memory.
//
// Who needs it: code that runs where cudaMalloc is not available or not allowed, e.g. a
// plugin inside a host application that owns every device allocation (a real-time
// mapping pipeline with a fixed memory plan, a framework custom op that may only use the
// tensors it is handed), or a process that must not grow its device footprint after
// start-up.  Such a caller hands in inputs and outputs it already owns and gets the same
// solve as gp_voxels_solve_csr, without creating a handle (which allocates).
//
// The solve needs scratch memory for its work queues (size buckets, per-bucket
// counters, the voxel work list and the escalation lists).  Here that scratch is one
// file-scope __device__ array of fixed size: it exists on every GPU that loads the
// library, for the life of the process, and every call shares it.  Its device address is
// taken with cudaGetSymbolAddress once per device and context, by the first call on a
// device (which should therefore come before any stream capture) and again after that
// device's context has been replaced (host code cannot use the array's name as a
// pointer: on the host that name is only a stand-in).  The counters that must start
// at zero are cleared on the stream at the start of every call.
//
// Limits: at most kNoAllocMaxVoxels voxels per call; voxels whose factor does not fit
// shared memory (no global workspace exists here) are reported GPV_VOX_TOO_LARGE.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <mutex>

#include "../../include/gp_voxels.h"
#include "gpv_internal.h"

using namespace gpv;

namespace {

constexpr int kNoAllocMaxVoxels = GPV_NOALLOC_MAX_VOXELS;
constexpr int kMaxDevices = 64;

// layout of the scratch array (int32 entries)
constexpr int kOffHi = 0;                              // bucket upper bounds
constexpr int kOffCount = kOffHi + kNumBuckets + 2;     // per-bucket counts
constexpr int kOffBase = kOffCount + kNumBuckets + 2;   // per-bucket first entry
constexpr int kOffCursor = kOffBase + kNumBuckets + 2;  // per-bucket scatter cursor
constexpr int kOffNext = kOffCursor + kNumBuckets + 2;  // per-launch dequeue counters
constexpr int kOffEscCount = kOffNext + kNumBuckets + 2;
constexpr int kOffWork = 128;                           // voxel work list
constexpr int kOffEsc = kOffWork + kNoAllocMaxVoxels;   // two escalation lists
constexpr int kScratchInts = kOffEsc + 2 * kNoAllocMaxVoxels;
static_assert(kOffEscCount + 2 <= kOffWork, "scratch header overflows");

static __device__ __align__(256) int32_t g_noalloc_scratch[kScratchInts];

std::mutex g_mu;
// per device: the scratch array's address and the context it was taken in.  A context
// that is destroyed and created again (cudaDeviceReset, a primary context released by its
// last user) reloads the module, and the array may then sit elsewhere, so the address is
// looked up again whenever the device's current context is not the one it was taken in.
struct ScratchAddr {
    void* ctx = nullptr;
    int32_t* ptr = nullptr;
};
ScratchAddr g_scratch[kMaxDevices];

// cuCtxGetCurrent, fetched through the runtime so that the library does not link the
// driver library itself (it must load on machines without a GPU driver)
typedef int (*CtxGetCurrentFn)(void**);
CtxGetCurrentFn ctx_get_current()
{
    static CtxGetCurrentFn fn = [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) !=
                cudaSuccess || q != cudaDriverEntryPointSuccess)
            p = nullptr;
        return reinterpret_cast<CtxGetCurrentFn>(p);
    }();
    return fn;
}

struct Bounds {
    int hi[kNumBuckets];
};

__global__ void k_set_bounds(Bounds b, int nb, int32_t* dst)
{
    const int i = threadIdx.x;
    if (i < nb) dst[i] = b.hi[i];
}

int fail(cudaError_t e)
{
    gpv_record_cuda_error(e);  // shown by gp_voxels_last_error()
    return GPV_ECUDA;
}

// Device address of the scratch array on the current device: taken once per device and
// context (the set-up of the first call on a device, or after its context changed).
int scratch_on_current_device(int32_t** out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(e);
    if (dev < 0 || dev >= kMaxDevices) return GPV_EINVAL;
    CtxGetCurrentFn getc = ctx_get_current();
    if (!getc) {
        gpv_record_cuda_error(cudaErrorDeviceUninitialized);
        return GPV_ECUDA;
    }
    void* ctx = nullptr;
    if (getc(&ctx) != 0) ctx = nullptr;  // null: no context is current yet
    std::lock_guard<std::mutex> lock(g_mu);
    ScratchAddr& sa = g_scratch[dev];
    if (!sa.ptr || !ctx || sa.ctx != ctx) {
        // the lookup itself makes the device's primary context current where none was
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return fail(e);
        if (getc(&ctx) != 0 || !ctx) {
            gpv_record_cuda_error(cudaErrorDeviceUninitialized);
            return GPV_ECUDA;
        }
        sa.ptr = static_cast<int32_t*>(p);
        sa.ctx = ctx;
    }
    *out = sa.ptr;
    return GPV_OK;
}

int kind_of(int precision)
{
    return precision == GPV_PREC_FP32 ? PREC_F32 : (precision == GPV_PREC_FP64 ? PREC_F64 : PREC_FF);
}

}  // namespace

extern "C" int gp_voxels_solve_csr_noalloc(const gp_voxels_config* c, const float* d_xyz,
                                           const int64_t* d_offsets, int32_t nvox,
                                           const float* d_centres, const float* d_lambda,
                                           const float* d_sf2, const float* d_sn2,
                                           uint8_t* d_axis, float* d_mean, float* d_var,
                                           uint32_t* d_status, float* d_pos, float* d_scale,
                                           float* d_quat, gpv_stream_t stream)
{
    if (!c || nvox < 0) return GPV_EINVAL;
    if (nvox > kNoAllocMaxVoxels) return GPV_EINVAL;  // larger than the static scratch
    if (!(c->voxel_size > 0.f) || c->grid_side < 1 || c->grid_side > kMaxG || c->n_s < 1 ||
        c->n_r < 1 || c->n_s * c->n_r != c->grid_side || c->tau < 1 ||
        c->max_points < c->tau || c->mean_mode < 0 || c->mean_mode > 1 || c->precision < 0 ||
        c->precision > 2 || c->init_mode < 0 || c->init_mode > 1 || !(c->esc_cond > 1.f) ||
        c->refine < 0 || c->refine > 1)
        return GPV_EINVAL;
    if (c->factor_panel != 0 && c->factor_panel != 4 && c->factor_panel != 8 && c->factor_panel != 16)
        return GPV_EINVAL;
    if (nvox == 0) return GPV_OK;
    if (!d_xyz || !d_offsets || !d_centres || !d_lambda || !d_sf2 || !d_sn2 || !d_axis ||
        !d_mean || !d_var || !d_status)
        return GPV_EINVAL;
    const bool any_init = d_pos || d_scale || d_quat;
    if (any_init && !(d_pos && d_scale && d_quat)) return GPV_EINVAL;

    int32_t* scr = nullptr;
    int rc = scratch_on_current_device(&scr);
    if (rc != GPV_OK) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    const int kind = kind_of(c->precision);
    const int G = c->grid_side;
    const int Gp = (G + kQryBlk - 1) / kQryBlk * kQryBlk;
    int dev = 0, sms = 0;
    cudaError_t e;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return fail(e);
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return fail(e);

    // largest voxel whose factor fits shared memory, in this precision and in the FP64
    // escalation pass of the mixed precision
    int nsm = 0, nsm64 = 0;
    if ((e = solve_max_smem_n(kind, G, Gp, &nsm)) != cudaSuccess) return fail(e);
    if ((e = solve_max_smem_n(PREC_F64, G, Gp, &nsm64)) != cudaSuccess) return fail(e);
    int maxp = std::min(c->max_points, nsm);
    if (kind == PREC_FF) maxp = std::min(maxp, nsm64);
    if (maxp < c->tau) return GPV_EINVAL;

    // size buckets up to maxp
    const int ladder[] = {16, 32, 48, 64, 96, 128, 160, 192, 256, 384, 512, 768, 1024};
    Bounds bnd;
    int nb = 0;
    for (int x : ladder)
        if (x < maxp && nb < kNumBuckets - 1) bnd.hi[nb++] = x;
    bnd.hi[nb++] = maxp;

    SolveArgs a;
    memset(&a, 0, sizeof(a));
    a.xyz = d_xyz; a.offsets = d_offsets; a.centres = d_centres;
    a.lam = d_lambda; a.sf2 = d_sf2; a.sn2 = d_sn2; a.nvox = nvox; a.nvox_dev = nullptr;
    a.size = c->voxel_size; a.G = G; a.Gp = Gp; a.n_s = c->n_s; a.n_r = c->n_r;
    a.tau = c->tau; a.mean_mode = c->mean_mode; a.init_mode = c->init_mode;
    a.esc_cond = c->esc_cond;
    a.escalate = kind == PREC_FF ? 1 : 0;
    a.refine = kind == PREC_F32 ? c->refine : 0;
    a.axis = d_axis; a.mean = d_mean; a.var = d_var; a.status = d_status;
    a.pos = d_pos; a.scale = d_scale; a.quat = d_quat;
    a.esc_list = scr + kOffEsc; a.esc_count = scr + kOffEscCount;
    a.gws = nullptr; a.gws_stride = 0;
    a.max_points = maxp;
    a.panel = c->factor_panel > 0 ? c->factor_panel : 16;
    a.nmax_small_f64 = std::min(nsm64, maxp);

    k_set_bounds<<<1, 32, 0, s>>>(bnd, nb, scr + kOffHi);
    if ((e = cudaGetLastError()) != cudaSuccess) return fail(e);
    // clears the bucket counts, cursors, dequeue counters and escalation counts
    if ((e = launch_classify(a, scr + kOffHi, nb, scr + kOffCount, scr + kOffBase,
                             scr + kOffCursor, scr + kOffWork, scr + kOffNext,
                             scr + kOffEscCount, s)) != cudaSuccess)
        return fail(e);
    for (int b = nb - 1; b >= 0; --b) {
        int nt = 0, pw = 0;  // the handle path's default shape of the bucket
        default_bucket_shape(kind, bnd.hi[b], G, c->factor_panel, &nt, &pw);
        a.panel = pw;
        const int smem = smem_plan(bnd.hi[b], G, Gp, kind == PREC_F32 ? 4 : 8, true, nt).total;
        int occ = 0;
        if ((e = solve_occupancy(kind, true, nt, smem, &occ)) != cudaSuccess) return fail(e);
        if (occ < 1) return GPV_EINVAL;
        a.work = scr + kOffWork;
        a.work_base = scr + kOffBase + b;
        a.work_count = scr + kOffCount + b;
        a.work_next = scr + kOffNext + b;
        a.nmax = bnd.hi[b];
        // an explicit panel width selects the blocked factor for every bucket
        a.percol_max = c->factor_panel == 0 && bnd.hi[b] <= default_percol_max(kind == PREC_F32 ? 4 : 8)
                           ? bnd.hi[b] : 0;
        if ((e = launch_solve(kind, true, nt, a, sms * occ, smem, s)) != cudaSuccess) return fail(e);
    }
    if (kind == PREC_FF) {  // FP64 re-solve of the voxels that failed the conditioning check
        const int nt = solve_threads(a.nmax_small_f64, true);
        const int smem = smem_plan(a.nmax_small_f64, G, Gp, 8, true, nt).total;
        int occ = 0;
        if ((e = solve_occupancy(PREC_F64, true, nt, smem, &occ)) != cudaSuccess) return fail(e);
        if (occ < 1) return GPV_EINVAL;
        a.escalate = 0;
        a.escalation_pass = 1;
        a.work = scr + kOffEsc;
        a.work_base = nullptr;
        a.work_count = scr + kOffEscCount;
        a.work_next = scr + kOffNext + nb;
        a.nmax = a.nmax_small_f64;
        a.percol_max = default_percol_max(8);
        a.panel = 16;  // the escalation pass of the handle path uses 16-column panels
        if ((e = launch_solve(PREC_F64, true, nt, a, sms * occ, smem, s)) != cudaSuccess) return fail(e);
    }
    return GPV_OK;
}
