// gpv_store.cu -- device voxel store of ALG.STORE / ALG.HASH (supplementary Alg. 2).
//
// Insert of one scan (all on the caller's stream, no host round trip):
//   k_hash      key = floor(p / s) per coordinate (FP32, IEEE division), open-addressing
//               insert (CAS, linear probing bounded by the capacity), first point index
//               and point count of each visited voxel
//   k_flag/scan the first point of each voxel marks it; an exclusive scan of the marks
//               gives S_updated in order of first appearance (deterministic)
//   k_fill      point indices grouped per visited voxel
//   k_append    one warp per voxel: its new points ranked by index (deterministic order),
//               the last max_points of them appended to the voxel's ring bucket
//   k_snap      the bucket of every visited voxel copied, oldest point first, into the
//               slot's CSR snapshot that the serving solve reads
#include <cuda_runtime.h>
#include <limits.h>
#include <stdint.h>
#include <string.h>

#include <new>

#include "gpv_internal.h"
#include "gpv_store.h"

namespace {

constexpr uint64_t kEmpty = ~0ull;
constexpr int kOff21 = 1 << 20;
constexpr int kScanBlock = 1024;

__device__ __forceinline__ uint64_t pack_key(int kx, int ky, int kz)
{
    const uint64_t m = 0x1FFFFFull;
    return ((uint64_t)(uint32_t)(kx + kOff21) & m) | (((uint64_t)(uint32_t)(ky + kOff21) & m) << 21) |
           (((uint64_t)(uint32_t)(kz + kOff21) & m) << 42);
}

__device__ __forceinline__ int unpack_axis(uint64_t k, int a)
{
    return (int)((k >> (21 * a)) & 0x1FFFFFull) - kOff21;
}

__device__ __forceinline__ uint32_t hash_slot(uint64_t key, uint32_t mask)
{
    uint64_t h = key * 0x9E3779B97F4A7C15ull;  // Fibonacci hashing
    h ^= h >> 31;
    return (uint32_t)h & mask;
}

__global__ void k_hash(const float* xyz, int npts, float size, uint64_t* keys, uint32_t mask,
                       int32_t* slot_of, int32_t* first, int32_t* cnt, int32_t* nvox,
                       int32_t* counters)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= npts) return;
    const int kx = (int)floorf(__fdiv_rn(xyz[3 * i + 0], size));
    const int ky = (int)floorf(__fdiv_rn(xyz[3 * i + 1], size));
    const int kz = (int)floorf(__fdiv_rn(xyz[3 * i + 2], size));
    const uint64_t key = pack_key(kx, ky, kz);
    const uint32_t h = hash_slot(key, mask);
    int s = -1;
    for (uint32_t p = 0; p <= mask; ++p) {  // at most one probe per slot
        const uint32_t t = (h + p) & mask;
        const uint64_t k = keys[t];  // a key, once written, never changes
        if (k == key) { s = (int)t; break; }
        if (k == kEmpty) {
            const uint64_t old = atomicCAS((unsigned long long*)&keys[t], (unsigned long long)kEmpty,
                                           (unsigned long long)key);
            if (old == kEmpty) { s = (int)t; atomicAdd(nvox, 1); break; }
            if (old == key) { s = (int)t; break; }
        }
    }
    slot_of[i] = s;
    if (s < 0) {
        atomicOr(counters + 1, 1);  // hash full: the point is dropped
        return;
    }
    atomicMin(&first[s], i);
    atomicAdd(&cnt[s], 1);
}

__global__ void k_flag(const int32_t* slot_of, const int32_t* first, int npts, int32_t* flag)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= npts) return;
    const int s = slot_of[i];
    flag[i] = (s >= 0 && first[s] == i) ? 1 : 0;
}

// ---- exclusive scan with a device-side length ------------------------------------
template <class O>
__device__ __forceinline__ O block_excl_scan(O v, O* wsum, O& total)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    O x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        O y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[wid] = x;
    __syncthreads();
    if (wid == 0) {
        O w = wsum[lane];
        O wx = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            O y = __shfl_up_sync(0xffffffffu, wx, o);
            if (lane >= o) wx += y;
        }
        wsum[lane] = wx - w;  // exclusive prefix of the warp totals
        if (lane == 31) wsum[32] = wx;
    }
    __syncthreads();
    total = wsum[32];
    O r = x - v + wsum[wid];
    __syncthreads();
    return r;
}

template <class O>
__global__ void __launch_bounds__(kScanBlock) k_scan_blocks(const int32_t* in, int n,
                                                            const int32_t* n_dev, O* out, O* bsum)
{
    __shared__ O wsum[33];
    const int len = n_dev ? min(n, *n_dev) : n;
    const int i = blockIdx.x * kScanBlock + threadIdx.x;
    const O v = i < len ? (O)in[i] : (O)0;
    O tot;
    const O r = block_excl_scan<O>(v, wsum, tot);
    if (i < n) out[i] = r;
    if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

template <class O>
__global__ void __launch_bounds__(kScanBlock) k_scan_top(O* bsum, int nb, O* total_out)
{
    __shared__ O wsum[33];
    const O v = (int)threadIdx.x < nb ? bsum[threadIdx.x] : (O)0;
    O tot;
    const O r = block_excl_scan<O>(v, wsum, tot);
    if ((int)threadIdx.x < nb) bsum[threadIdx.x] = r;
    if (threadIdx.x == 0 && total_out) *total_out = tot;
}

template <class O>
__global__ void k_scan_add(O* out, int n, const O* bsum)
{
    const int i = blockIdx.x * kScanBlock + threadIdx.x;
    if (i < n) out[i] += bsum[blockIdx.x];
}

// out[i] = sum of in[0 .. i-1] for i < n, entries at or past the device length read as 0
template <class O>
cudaError_t excl_scan(const int32_t* in, int n, const int32_t* n_dev, O* out, O* bsum,
                      O* total_out, cudaStream_t s)
{
    const int nb = (n + kScanBlock - 1) / kScanBlock;
    if (nb < 1 || nb > kScanBlock) return cudaErrorInvalidValue;
    k_scan_blocks<O><<<nb, kScanBlock, 0, s>>>(in, n, n_dev, out, bsum);
    k_scan_top<O><<<1, kScanBlock, 0, s>>>(bsum, nb, total_out);
    k_scan_add<O><<<nb, kScanBlock, 0, s>>>(out, n, bsum);
    return cudaGetLastError();
}

// rows = min(visited, max_vox); flag 2 when more voxels were visited
__global__ void k_rows(int32_t* counters, int max_vox)
{
    const int t = counters[2];
    counters[0] = t < max_vox ? t : max_vox;
    if (t > max_vox) atomicOr(counters + 1, 2);
}

__global__ void k_touch(const int32_t* slot_of, const int32_t* flag, const int32_t* pos,
                        int npts, int max_vox, int32_t* touched, int32_t* tmap)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= npts || !flag[i]) return;
    const int s = slot_of[i];
    const int t = pos[i];
    if (t < max_vox) {
        touched[t] = s;
        tmap[s] = t;
    } else {
        tmap[s] = -1;
    }
}

__global__ void k_segsz(const int32_t* counters, const int32_t* touched, const int32_t* cnt,
                        int32_t* segsz)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= counters[0]) return;
    segsz[t] = cnt[touched[t]];
}

__global__ void k_fill(const int32_t* slot_of, const int32_t* tmap, const int32_t* segoff,
                       int npts, int32_t* fill, int32_t* seg, int32_t* first, int32_t* cnt)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= npts) return;
    const int s = slot_of[i];
    if (s < 0) return;
    const int t = tmap[s];
    if (t < 0) {  // voxel beyond max_scan_voxels: not stored this scan; clear its marks
        first[s] = INT_MAX;
        cnt[s] = 0;
        return;
    }
    const int p = segoff[t] + atomicAdd(&fill[s], 1);
    seg[p] = i;
}

// Ascending sort of a[0 .. c) by one warp (a in shared or global memory): Batcher's bitonic
// network on the next power of two N >= c in the form whose comparators are all ascending
// (the first stage of each merge of size k compares mirror images i and i ^ (k - 1), the
// later ones i and i + j), so the positions from c up act as +infinity and their
// comparators are skipped.  O(c log^2 c) work against O(c^2) for ranking every element.
__device__ void warp_sort_asc(int32_t* a, int c, int lane)
{
    int N = 1;
    while (N < c) N <<= 1;
    for (int k = 2; k <= N; k <<= 1) {
        for (int j = k >> 1; j >= 1; j >>= 1) {
            for (int q = lane; q < (N >> 1); q += 32) {
                const int i = ((q & ~(j - 1)) << 1) | (q & (j - 1));  // bit j of i clear
                const int p = j == (k >> 1) ? (i ^ (k - 1)) : (i | j);
                if (p < c) {
                    const int32_t x = a[i], y = a[p];
                    if (x > y) {
                        a[i] = y;
                        a[p] = x;
                    }
                }
            }
            __syncwarp();
        }
    }
}

constexpr int kAppendWarps = 8;   // warps per k_append block (256 threads)
constexpr int kSortCap = 1024;    // segments up to this length are sorted in shared memory

// one warp per visited voxel: deterministic order, ring append, marks cleared
__global__ void __launch_bounds__(32 * kAppendWarps)
k_append(const float* xyz, const int32_t* counters, const int32_t* touched,
         const int32_t* segsz, const int32_t* segoff, const int32_t* seg, int32_t* seg2,
         int nmax, float* ring, float* rnoise, float sn2, int32_t* total, int32_t* cnt,
         int32_t* fill, int32_t* first, int32_t* snapsz, uint32_t* vflags)
{
    __shared__ int32_t sbuf[kAppendWarps][kSortCap];
    const int lane = threadIdx.x & 31;
    const int t = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (t >= counters[0]) return;
    const int s = touched[t];
    const int c = segsz[t];
    const int base = segoff[t];
    // the new points of the voxel in the order of their indices in the scan (a dense voxel
    // takes a few thousand points of one scan, so ranking each point against all was the
    // slowest part of the insert)
    int32_t* srt = c <= kSortCap ? sbuf[threadIdx.x >> 5] : seg2 + base;
    for (int e = lane; e < c; e += 32) srt[e] = seg[base + e];
    __syncwarp();
    warp_sort_asc(srt, c, lane);
    const int tot = total[s];
    const int keep = c < nmax ? c : nmax;
    for (int k = c - keep + lane; k < c; k += 32) {
        const int slotpos = (int)(((int64_t)tot + k) % nmax);
        const int src = srt[k];
        float* dst = ring + ((int64_t)s * nmax + slotpos) * 3;
        dst[0] = xyz[3 * src + 0];
        dst[1] = xyz[3 * src + 1];
        dst[2] = xyz[3 * src + 2];
        if (rnoise) rnoise[(int64_t)s * nmax + slotpos] = sn2;  // the sensor's variance
    }
    __syncwarp();
    if (lane == 0) {
        const int nt = tot + c;
        total[s] = nt;
        snapsz[t] = nt < nmax ? nt : nmax;
        vflags[t] = nt > nmax ? gpv::VOX_TRUNCATED : 0u;
        cnt[s] = 0;
        fill[s] = 0;
        first[s] = INT_MAX;
    }
}

// one warp per visited voxel: bucket -> snapshot, oldest point first; offsets clamped
// to the snapshot capacity (a voxel past it keeps fewer points and is flagged)
__global__ void k_snap(int32_t* counters, const int32_t* touched, const uint64_t* keys,
                       const int32_t* total, const int32_t* snapsz, int64_t* snapoff,
                       const float* ring, int nmax, int64_t cap, float size, float lam,
                       float sf2, float sn2, float* snap, int64_t* okeys, float* centres,
                       float* olam, float* osf2, float* osn2, uint32_t* vflags,
                       const float* rnoise, const uint8_t* vstate, int tau, float* snoise,
                       int32_t* ssrc, uint8_t* rtype, uint8_t* rskip)
{
    const int lane = threadIdx.x & 31;
    const int t = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int rows = counters[0];
    if (t > rows) return;
    if (t == rows) {  // closing offset (the total)
        if (lane == 0) snapoff[t] = snapoff[t] < cap ? snapoff[t] : cap;
        return;
    }
    const int s = touched[t];
    const int64_t o_raw = snapoff[t];
    const int64_t o = o_raw < cap ? o_raw : cap;
    int64_t e = o_raw + snapsz[t];
    if (e > cap) e = cap;
    const int n = (int)(e - o);
    const int tot = total[s];
    const int start = tot > nmax ? tot % nmax : 0;
    for (int k = lane; k < n; k += 32) {
        const int src = (start + k) % nmax;
        const float* p = ring + ((int64_t)s * nmax + src) * 3;
        float* d = snap + (o + k) * 3;
        d[0] = p[0]; d[1] = p[1]; d[2] = p[2];
        if (rnoise) {
            const int64_t r = (int64_t)s * nmax + src;
            snoise[o + k] = rnoise[r];
            ssrc[o + k] = (int32_t)r;
        }
    }
    __syncwarp();
    if (lane == 0) {
        snapoff[t] = o;
        if (rnoise) {  // voxel type before this scan's solve (Sec. 3.3)
            const int st = vstate[s];
            const int ty = st == 3 ? 3 : (st == 2 ? 2 : (n >= tau ? 1 : 0));
            rtype[t] = (uint8_t)ty;
            rskip[t] = ty == 3 ? 1 : 0;
        }
        const uint64_t key = keys[s];
        okeys[t] = (int64_t)key;
        for (int a = 0; a < 3; ++a)
            centres[3 * t + a] = __fmul_rn((float)unpack_axis(key, a) + 0.5f, size);
        olam[t] = lam;
        osf2[t] = sf2;
        osn2[t] = sn2;
        if (n < snapsz[t]) {
            vflags[t] |= gpv::VOX_TRUNCATED;
            atomicOr(counters + 1, 4);
        }
    }
}

__global__ void k_fill_i32(int32_t* p, int n, int32_t v)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = v;
}
__global__ void k_fill_u64(uint64_t* p, int n, uint64_t v)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = v;
}

__global__ void k_or_flags(const int32_t* counters, const uint32_t* vflags, uint32_t* status)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < counters[0]) status[t] |= vflags[t];
}

__global__ void k_copy_rows(const int32_t* counters, const int64_t* keys, const float* centres,
                            int64_t* okeys, float* ocentres)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= counters[0]) return;
    if (okeys) okeys[t] = keys[t];
    if (ocentres)
        for (int a = 0; a < 3; ++a) ocentres[3 * t + a] = centres[3 * t + a];
}

// one warp per row: variance feedback and the type transition of Sec. 3.3
__global__ void k_feedback(const int32_t* counters, const int32_t* touched,
                           const int64_t* snapoff, const uint32_t* status, const float* var,
                           int GG, const float* spvar, const int32_t* ssrc, float floor_,
                           float eta_sf2, const uint8_t* rtype, float* rnoise, uint8_t* vstate,
                           uint8_t* rafter)
{
    const int lane = threadIdx.x & 31;
    const int t = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (t >= counters[0]) return;
    const uint32_t st = status[t];
    const int before = rtype[t];
    const bool solved = (st & (gpv::VOX_BELOW_TAU | gpv::VOX_NOT_SPD | gpv::VOX_TOO_LARGE |
                               gpv::VOX_CONVERGED)) == 0;
    if (!solved) {
        if (lane == 0)
            rafter[t] = (st & gpv::VOX_CONVERGED) ? 3 : ((st & gpv::VOX_BELOW_TAU) && before < 2 ? 0 : before);
        return;
    }
    const int64_t o = snapoff[t], e = snapoff[t + 1];
    for (int64_t k = o + lane; k < e; k += 32) rnoise[ssrc[k]] = fmaxf(spvar[k], floor_);
    float acc = 0.f;
    for (int q = lane; q < GG; q += 32) acc += var[(int64_t)t * GG + q];
#pragma unroll
    for (int w = 16; w > 0; w >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, w);
    if (lane == 0) {
        const int after = __fdiv_rn(acc, (float)GG) <= eta_sf2 ? 3 : 2;
        vstate[touched[t]] = (uint8_t)after;
        rafter[t] = (uint8_t)after;
    }
}

__global__ void k_copy_types(const int32_t* counters, const uint8_t* rtype, const uint8_t* rafter,
                             uint8_t* before, uint8_t* after)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= counters[0]) return;
    if (before) before[t] = rtype[t];
    if (after) after[t] = rafter[t];
}

__global__ void k_type_counts(const uint64_t* keys, const int32_t* total, const uint8_t* vstate,
                              uint32_t H, int nmax, int tau, unsigned long long* counts)
{
    __shared__ unsigned long long c[4];
    if (threadIdx.x < 4) c[threadIdx.x] = 0;
    __syncthreads();
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < H && keys[i] != kEmpty) {
        const int n = total[i] < nmax ? total[i] : nmax;
        const int st = vstate ? vstate[i] : 0;
        atomicAdd(&c[st == 3 ? 3 : (st == 2 ? 2 : (n >= tau ? 1 : 0))], 1ull);
    }
    __syncthreads();
    if (threadIdx.x < 4 && c[threadIdx.x]) atomicAdd(&counts[threadIdx.x], c[threadIdx.x]);
}

size_t slot_bytes(const gp_voxels_config* c, int64_t cap)
{
    const size_t P = (size_t)c->max_scan_points, V = (size_t)c->max_scan_voxels;
    size_t b = 0;
    b += P * 4 * 5;
    b += V * 4 * 4 + (V + 1) * 4 + (V + 2) * 8 + V * 8 + V * 12 + V * 12 + V * 4;
    b += (size_t)cap * 12;
    b += (kScanBlock + 1) * 12 + 64;
    if (c->eta > 0.f) b += (size_t)cap * 12 + V * 3;  // feedback: noise, source, pvar; types
    return b;
}

int64_t snap_cap_of(const gp_voxels_config* c)
{
    return c->snap_points > 0 ? c->snap_points : (int64_t)c->max_scan_voxels * c->max_points;
}

}  // namespace

size_t store_bytes(const gp_voxels_config* c)
{
    if (!c || c->hash_capacity == 0) return 0;
    const size_t H = c->hash_capacity;
    size_t b = H * (8 + 4 * 5) + H * (size_t)c->max_points * 12 + 64;
    if (c->eta > 0.f) b += H * (size_t)c->max_points * 4 + H;  // point noise, voxel state
    b += (size_t)(c->scan_slots > 0 ? c->scan_slots : 0) * slot_bytes(c, snap_cap_of(c));
    return b;
}

void store_destroy(gpv_store* s)
{
    if (!s) return;
    cudaFree(s->keys); cudaFree(s->total); cudaFree(s->cnt); cudaFree(s->fill);
    cudaFree(s->first); cudaFree(s->tmap); cudaFree(s->ring); cudaFree(s->nvox);
    cudaFree(s->rnoise); cudaFree(s->vstate);
    if (s->slots) {
        for (int i = 0; i < s->nslots; ++i) {
            gpv_scan_slot& S = s->slots[i];
            cudaFree(S.slot_of); cudaFree(S.flag); cudaFree(S.pos); cudaFree(S.seg); cudaFree(S.seg2);
            cudaFree(S.touched); cudaFree(S.segsz); cudaFree(S.segoff); cudaFree(S.snapsz);
            cudaFree(S.snapoff); cudaFree(S.keys); cudaFree(S.centres); cudaFree(S.lam);
            cudaFree(S.sf2); cudaFree(S.sn2); cudaFree(S.vflags); cudaFree(S.snap);
            cudaFree(S.scan_tmp); cudaFree(S.scan_tmp64); cudaFree(S.counters); cudaFree(S.npoints);
            cudaFree(S.snap_noise); cudaFree(S.snap_src); cudaFree(S.snap_pvar);
            cudaFree(S.rtype); cudaFree(S.rskip); cudaFree(S.rafter);
            if (S.free_ev) cudaEventDestroy(S.free_ev);
            if (S.ins_ev) cudaEventDestroy(S.ins_ev);
        }
        delete[] s->slots;
    }
    if (s->ev_insert) cudaEventDestroy(s->ev_insert);
    if (s->ev_fb) cudaEventDestroy(s->ev_fb);
    delete s;
}

int store_create(const gp_voxels_config* c, gpv_store** out, size_t* bytes_acc)
{
    *out = nullptr;
    if (c->scan_slots < 1 || c->scan_slots > 64 || c->max_scan_points < 1 ||
        c->max_scan_points > kScanBlock * kScanBlock || c->max_scan_voxels < 1 ||
        c->max_scan_voxels >= kScanBlock * kScanBlock - 1 || c->max_scan_voxels > c->max_voxels)
        return GPV_EINVAL;
    gpv_store* s = new (std::nothrow) gpv_store();
    if (!s) return GPV_ENOMEM;
    s->H = c->hash_capacity;
    s->nmax = c->max_points;
    s->size = c->voxel_size;
    s->nslots = c->scan_slots;
    s->max_pts = c->max_scan_points;
    s->max_vox = c->max_scan_voxels;
    s->snap_cap = snap_cap_of(c);
    size_t acc = 0;
    bool ok = true;
    auto al = [&](void** p, size_t b) {
        if (!ok) return;
        if (cudaMalloc(p, b) != cudaSuccess) { cudaGetLastError(); ok = false; return; }
        acc += b;
    };
    const size_t H = s->H;
    al((void**)&s->keys, H * 8);
    al((void**)&s->total, H * 4);
    al((void**)&s->cnt, H * 4);
    al((void**)&s->fill, H * 4);
    al((void**)&s->first, H * 4);
    al((void**)&s->tmap, H * 4);
    al((void**)&s->ring, H * (size_t)s->nmax * 12);
    al((void**)&s->nvox, 4);
    s->feedback = c->eta > 0.f;
    if (s->feedback) {
        al((void**)&s->rnoise, H * (size_t)s->nmax * 4);
        al((void**)&s->vstate, H);
    }
    s->slots = new (std::nothrow) gpv_scan_slot[s->nslots];
    if (!s->slots) ok = false;
    for (int i = 0; ok && i < s->nslots; ++i) {
        gpv_scan_slot& S = s->slots[i];
        const size_t P = (size_t)s->max_pts, V = (size_t)s->max_vox;
        al((void**)&S.slot_of, P * 4); al((void**)&S.flag, P * 4); al((void**)&S.pos, P * 4);
        al((void**)&S.seg, P * 4); al((void**)&S.seg2, P * 4);
        al((void**)&S.touched, V * 4); al((void**)&S.segsz, (V + 1) * 4); al((void**)&S.segoff, (V + 1) * 4);
        al((void**)&S.snapsz, (V + 1) * 4); al((void**)&S.snapoff, (V + 2) * 8); al((void**)&S.keys, V * 8);
        al((void**)&S.centres, V * 12); al((void**)&S.lam, V * 4); al((void**)&S.sf2, V * 4);
        al((void**)&S.sn2, V * 4); al((void**)&S.vflags, V * 4);
        al((void**)&S.snap, (size_t)(s->snap_cap > 0 ? s->snap_cap : 1) * 12);
        al((void**)&S.scan_tmp, (kScanBlock + 1) * 4);
        al((void**)&S.scan_tmp64, (kScanBlock + 1) * 8);
        al((void**)&S.counters, 4 * 4);
        al((void**)&S.npoints, 8);
        if (s->feedback) {
            const size_t sc = (size_t)(s->snap_cap > 0 ? s->snap_cap : 1);
            al((void**)&S.snap_noise, sc * 4); al((void**)&S.snap_src, sc * 4);
            al((void**)&S.snap_pvar, sc * 4);
            al((void**)&S.rtype, V); al((void**)&S.rskip, V); al((void**)&S.rafter, V);
        }
        if (ok && cudaEventCreateWithFlags(&S.free_ev, cudaEventDisableTiming) != cudaSuccess) ok = false;
        if (ok && cudaEventCreateWithFlags(&S.ins_ev, cudaEventDisableTiming) != cudaSuccess) ok = false;
    }
    if (ok && cudaEventCreateWithFlags(&s->ev_insert, cudaEventDisableTiming) != cudaSuccess) ok = false;
    if (ok && cudaEventCreateWithFlags(&s->ev_fb, cudaEventDisableTiming) != cudaSuccess) ok = false;
    if (ok && s->feedback && cudaMemset(s->vstate, 0, H) != cudaSuccess) ok = false;
    if (ok) {
        const int blk = 256;
        const int grd = (int)((H + blk - 1) / blk);
        k_fill_u64<<<grd, blk>>>(s->keys, (int)H, kEmpty);
        k_fill_i32<<<grd, blk>>>(s->first, (int)H, INT_MAX);
        k_fill_i32<<<grd, blk>>>(s->tmap, (int)H, -1);
        ok = cudaMemset(s->total, 0, H * 4) == cudaSuccess && cudaMemset(s->cnt, 0, H * 4) == cudaSuccess &&
             cudaMemset(s->fill, 0, H * 4) == cudaSuccess && cudaMemset(s->nvox, 0, 4) == cudaSuccess &&
             cudaGetLastError() == cudaSuccess && cudaDeviceSynchronize() == cudaSuccess;
    }
    if (!ok) {
        store_destroy(s);
        return GPV_ENOMEM;
    }
    *bytes_acc += acc;
    *out = s;
    return GPV_OK;
}

cudaError_t store_insert(gpv_store* st, int si, const float* d_xyz, int npts, cudaStream_t s,
                         const gp_voxels_config* c)
{
    gpv_scan_slot& S = st->slots[si];
    cudaError_t e;
    if ((e = cudaMemsetAsync(S.counters, 0, 4 * 4, s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(S.snapoff, 0, 8, s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(S.npoints, 0, 8, s)) != cudaSuccess) return e;
    if (npts == 0) return cudaSuccess;
    const int blk = 256, grdp = (npts + blk - 1) / blk;
    const uint32_t mask = st->H - 1;
    k_hash<<<grdp, blk, 0, s>>>(d_xyz, npts, st->size, st->keys, mask, S.slot_of, st->first,
                                st->cnt, st->nvox, S.counters);
    k_flag<<<grdp, blk, 0, s>>>(S.slot_of, st->first, npts, S.flag);
    // S_updated: exclusive scan of the first-point marks; counters[2] = visited voxels
    if ((e = excl_scan<int32_t>(S.flag, npts, nullptr, S.pos, S.scan_tmp, S.counters + 2, s)) != cudaSuccess)
        return e;
    k_rows<<<1, 1, 0, s>>>(S.counters, st->max_vox);
    k_touch<<<grdp, blk, 0, s>>>(S.slot_of, S.flag, S.pos, npts, st->max_vox, S.touched, st->tmap);
    const int V = st->max_vox, grdv = (V + blk - 1) / blk;
    k_segsz<<<grdv, blk, 0, s>>>(S.counters, S.touched, st->cnt, S.segsz);
    if ((e = excl_scan<int32_t>(S.segsz, V, S.counters, S.segoff, S.scan_tmp, nullptr, s)) != cudaSuccess)
        return e;
    k_fill<<<grdp, blk, 0, s>>>(S.slot_of, st->tmap, S.segoff, npts, st->fill, S.seg, st->first,
                                st->cnt);
    const int wblk = 32 * kAppendWarps, grdw = (V * 32 + wblk - 1) / wblk;
    k_append<<<grdw, wblk, 0, s>>>(d_xyz, S.counters, S.touched, S.segsz, S.segoff, S.seg, S.seg2,
                                   st->nmax, st->ring, st->rnoise, c->sn2, st->total, st->cnt,
                                   st->fill, st->first, S.snapsz, S.vflags);
    // V + 1 outputs: snapoff[rows] is the total (entries at or past rows scan as zero)
    if ((e = excl_scan<int64_t>(S.snapsz, V + 1, S.counters, S.snapoff, S.scan_tmp64, S.npoints, s)) != cudaSuccess)
        return e;
    const int grdw2 = ((V + 1) * 32 + wblk - 1) / wblk;
    k_snap<<<grdw2, wblk, 0, s>>>(S.counters, S.touched, st->keys, st->total, S.snapsz, S.snapoff,
                                  st->ring, st->nmax, st->snap_cap, st->size, c->lambda, c->sf2,
                                  c->sn2, S.snap, S.keys, S.centres, S.lam, S.sf2, S.sn2, S.vflags,
                                  st->rnoise, st->vstate, c->tau, S.snap_noise, S.snap_src,
                                  S.rtype, S.rskip);
    return cudaGetLastError();
}

cudaError_t store_feedback(gpv_store* st, int si, const uint32_t* status, const float* var,
                           const gp_voxels_config* c, cudaStream_t s)
{
    gpv_scan_slot& S = st->slots[si];
    const int wblk = 256, grdw = (st->max_vox * 32 + wblk - 1) / wblk;
    k_feedback<<<grdw, wblk, 0, s>>>(S.counters, S.touched, S.snapoff, status, var,
                                     c->grid_side * c->grid_side, S.snap_pvar, S.snap_src,
                                     c->noise_floor, c->eta * c->sf2, S.rtype, st->rnoise,
                                     st->vstate, S.rafter);
    return cudaGetLastError();
}

cudaError_t store_copy_types(gpv_store* st, int si, uint8_t* before, uint8_t* after,
                             cudaStream_t s)
{
    gpv_scan_slot& S = st->slots[si];
    const int blk = 256, grd = (st->max_vox + blk - 1) / blk;
    k_copy_types<<<grd, blk, 0, s>>>(S.counters, S.rtype, S.rafter, before, after);
    return cudaGetLastError();
}

cudaError_t store_type_counts(gpv_store* st, int tau, unsigned long long* d_counts, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(d_counts, 0, 4 * sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    const int blk = 256, grd = (int)((st->H + blk - 1) / blk);
    k_type_counts<<<grd, blk, 0, s>>>(st->keys, st->total, st->vstate, st->H, st->nmax, tau, d_counts);
    return cudaGetLastError();
}

cudaError_t store_or_flags(gpv_store* st, int si, uint32_t* status, cudaStream_t s)
{
    gpv_scan_slot& S = st->slots[si];
    const int blk = 256, grd = (st->max_vox + blk - 1) / blk;
    k_or_flags<<<grd, blk, 0, s>>>(S.counters, S.vflags, status);
    return cudaGetLastError();
}

cudaError_t store_copy_rows(gpv_store* st, int si, int64_t* keys, float* centres, cudaStream_t s)
{
    if (!keys && !centres) return cudaSuccess;
    gpv_scan_slot& S = st->slots[si];
    const int blk = 256, grd = (st->max_vox + blk - 1) / blk;
    k_copy_rows<<<grd, blk, 0, s>>>(S.counters, S.keys, S.centres, keys, centres);
    return cudaGetLastError();
}
