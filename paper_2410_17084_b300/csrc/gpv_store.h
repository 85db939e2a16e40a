// gpv_store.h -- device voxel store of ALG.STORE / ALG.HASH (supplementary Alg. 2):
// an open-addressing hash from voxel key to slot, a capped point bucket per slot, and
// per-scan slots holding S_updated (visited voxels) with a CSR snapshot of their buckets.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "../../include/gp_voxels.h"

struct gpv_scan_slot {
    // per point
    int32_t* slot_of = nullptr;
    int32_t* flag = nullptr;
    int32_t* pos = nullptr;
    int32_t* seg = nullptr;
    int32_t* seg2 = nullptr;
    // per visited voxel
    int32_t* touched = nullptr;
    int32_t* segsz = nullptr;
    int32_t* segoff = nullptr;
    int32_t* snapsz = nullptr;
    int64_t* snapoff = nullptr;
    int64_t* keys = nullptr;
    float* centres = nullptr;
    float* lam = nullptr;
    float* sf2 = nullptr;
    float* sn2 = nullptr;
    uint32_t* vflags = nullptr;
    float* snap = nullptr;        // snapshot points [snap_cap, 3]
    // variance feedback (Sec. 3.3), allocated when the state machine is on
    float* snap_noise = nullptr;  // noise variance of every snapshot point [snap_cap]
    int32_t* snap_src = nullptr;  // ring entry each snapshot point came from [snap_cap]
    float* snap_pvar = nullptr;   // posterior variance at each snapshot point [snap_cap]
    uint8_t* rtype = nullptr;     // voxel type (a)-(d) of every row before the solve [V]
    uint8_t* rskip = nullptr;     // 1: converged, not solved [V]
    uint8_t* rafter = nullptr;    // voxel type after the solve [V]
    int32_t* scan_tmp = nullptr;  // block sums of the device scans
    int64_t* scan_tmp64 = nullptr;
    int32_t* counters = nullptr;  // [0] rows, [1] flags, [2] visited voxels
    int64_t* npoints = nullptr;
    cudaEvent_t free_ev = nullptr;  // the slot's last user is done
    cudaEvent_t ins_ev = nullptr;   // the slot's insert is done
    bool busy = false;
};

struct gpv_store {
    uint32_t H = 0;
    int nmax = 0;
    float size = 0.f;
    uint64_t* keys = nullptr;
    int32_t* total = nullptr;
    int32_t* cnt = nullptr;
    int32_t* fill = nullptr;
    int32_t* first = nullptr;
    int32_t* tmap = nullptr;
    float* ring = nullptr;
    float* rnoise = nullptr;   // noise variance of every ring entry (state machine on)
    uint8_t* vstate = nullptr; // per hash slot: 0 not in the map, 2 active, 3 converged
    int32_t* nvox = nullptr;
    bool feedback = false;     // the voxel state machine with variance feedback is on
    int unsolved = -1;         // feedback: slot inserted and not yet solved (or -1)
    cudaEvent_t ev_fb = nullptr;  // feedback: the last solve's state update is done
    int nslots = 0;
    int max_pts = 0, max_vox = 0;
    int64_t snap_cap = 0;
    gpv_scan_slot* slots = nullptr;
    cudaEvent_t ev_insert = nullptr;
};

size_t store_bytes(const gp_voxels_config* c);
int store_create(const gp_voxels_config* c, gpv_store** out, size_t* bytes_acc);
void store_destroy(gpv_store* s);
// queue ALG.STORE of one scan into slot `si` on stream s
cudaError_t store_insert(gpv_store* st, int si, const float* d_xyz, int npts, cudaStream_t s,
                         const gp_voxels_config* c);
// OR the per-voxel flags of a slot into a status array (row count on the device)
cudaError_t store_or_flags(gpv_store* st, int si, uint32_t* status, cudaStream_t s);
cudaError_t store_copy_rows(gpv_store* st, int si, int64_t* keys, float* centres, cudaStream_t s);
// feedback: write the posterior variance of solved voxels back to their points, and
// move every row's voxel to its new type (reads the solve's status and variance)
cudaError_t store_feedback(gpv_store* st, int si, const uint32_t* status, const float* var,
                           const gp_voxels_config* c, cudaStream_t s);
cudaError_t store_copy_types(gpv_store* st, int si, uint8_t* before, uint8_t* after,
                             cudaStream_t s);
// counts of stored voxels by type (a)-(d) into a device array of 4 int64 (zeroed first)
cudaError_t store_type_counts(gpv_store* st, int tau, unsigned long long* d_counts,
                              cudaStream_t s);
