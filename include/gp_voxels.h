/*
 * gp_voxels.h -- C ABI of the B300 Voxel-GPR library: per-voxel Gaussian Process
 * Regression of LiDAR points and covariance-centred initialisation of 3D Gaussians,
 * as defined in GS-LIVM (arXiv 2410.17084), Sec. 3.1-3.3 and the supplementary
 * Alg. 2 (ALG.STORE / ALG.HASH) and Alg. 3 (ALG.SOLVE).
 *
 * Conventions shared by every call:
 *  - Every call returns a gpv_status (0 = success, negative = error).  Calls never
 *    abort and never print.  CUDA errors map to GPV_ECUDA; the CUDA error text of the
 *    last failure is available from gp_voxels_last_error().
 *  - Pointers named d_* are DEVICE pointers, h_* are HOST pointers.  Buffers are owned
 *    by the caller unless stated otherwise; inputs are read-only and must stay valid
 *    until the work queued on the given stream has completed.
 *  - All GPU work is queued asynchronously on the caller's stream (NULL = legacy
 *    default stream).  A call that returns a host value (h_* output) synchronises.
 *  - Problems of single voxels do not fail a call: they are reported per voxel in the
 *    d_status word (GPV_VOX_* bits).
 *  - Layouts: points are FP32 [n, 3] row-major world coordinates.  A query grid has
 *    G x G nodes; query q = i * G + j, i along the first and j along the second
 *    parameter axis of the voxel's value axis (Alg. 1: X -> (y, z), Y -> (z, x),
 *    Z -> (x, y)).  Node i sits at -s/2 + (i + 1/2) s / G in voxel-local coordinates
 *    (s = voxel side).  Predicted means are value coordinates relative to the voxel
 *    centre.
 */
#ifndef GP_VOXELS_H
#define GP_VOXELS_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define GPV_API __attribute__((visibility("default")))
#else
#define GPV_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

struct CUstream_st;
typedef struct CUstream_st* gpv_stream_t; /* a cudaStream_t */

typedef struct gp_voxels gp_voxels_t; /* opaque; owns all device state it allocates */

typedef enum {
    GPV_OK = 0,
    GPV_EINVAL = -1,   /* bad argument (NULL where required, size out of range) */
    GPV_ENOMEM = -2,   /* a device or host allocation failed */
    GPV_EBUDGET = -3,  /* the request does not fit the configured memory budget */
    GPV_ECUDA = -4,    /* a CUDA runtime call failed */
    GPV_ETIMEOUT = -5, /* a bounded wait gave up */
    GPV_EFULL = -6     /* a fixed-capacity structure (hash, scan slots) is full */
} gpv_status;

/* Per-voxel status bits written to d_status. */
enum {
    GPV_VOX_OK = 0,
    GPV_VOX_BELOW_TAU = 1,  /* n < tau: not processed (Sec. 3.1); prior written */
    GPV_VOX_ESCALATED = 2,  /* re-solved in FP64 after the conditioning check */
    GPV_VOX_NOT_SPD = 4,    /* Gram not positive definite in the final precision */
    GPV_VOX_TRUNCATED = 8,  /* bucket overflowed; oldest points were dropped */
    GPV_VOX_TOO_LARGE = 16  /* n > max_points: not processed; prior written */
};

/* Arithmetic of the solve. */
enum {
    GPV_PREC_FP32 = 0,  /* every step in FP32 (the paper's cuBLAS S-routines) */
    GPV_PREC_MIXED = 1, /* float-float (FP32-pair) arithmetic, per-voxel FP64
                           escalation when (max L_ii / min L_ii)^2 > esc_cond */
    GPV_PREC_FP64 = 2   /* every step in FP64 */
};

/* Flags of gp_voxels_solve_csr. */
enum {
    GPV_SOLVE_ONE_PER_LAUNCH = 1 /* baseline: one kernel launch per voxel */
};

typedef struct {
    float voxel_size;    /* s, metres; paper: 0.2 (hyperparameter table) */
    int grid_side;       /* G = n_s * n_r query nodes per side (Sec. 3.2); 1..32 */
    int n_s, n_r;        /* Gaussians per voxel side, nodes per Gaussian side */
    int tau;             /* minimum points per voxel (Sec. 3.1, tau = 10) */
    int max_points;      /* largest n per voxel accepted by the solve; also the
                            bucket capacity of the voxel store */
    int max_voxels;      /* largest batch (voxels) per solve call */
    int mean_mode;       /* 0: zero prior mean (Eq. 2); 1: data mean of f */
    int precision;       /* GPV_PREC_* */
    int init_mode;       /* 0: scale = sqrt(eig Phi), rotation = eigenvectors;
                            1: Eq. 8 as printed, S = diag(Phi), R = identity */
    float esc_cond;      /* escalation threshold on (max L_ii / min L_ii)^2 */
    uint32_t hash_capacity; /* voxel slots of the device hash (power of two) */
    size_t mem_budget;   /* bytes the handle may allocate (0 = no limit) */
} gp_voxels_config;

/* Fill *cfg with the paper's defaults (size 0.2, n_s = n_r = 3, tau = 10, lambda 1
 * is a per-call input) and the library's limits.  Never fails for non-NULL cfg. */
GPV_API int gp_voxels_config_default(gp_voxels_config* cfg);

/* Create a handle on the current CUDA device.  Allocates the solve workspaces (work
 * queues, a global-memory factor workspace for voxels whose factor does not fit
 * shared memory) and, if hash_capacity > 0, the voxel store of Alg. 2.
 * Errors: GPV_EINVAL (bad config), GPV_EBUDGET (footprint > mem_budget),
 * GPV_ENOMEM, GPV_ECUDA.  On error *out is NULL and nothing is leaked. */
GPV_API int gp_voxels_create(const gp_voxels_config* cfg, gp_voxels_t** out);

/* Free all device state of the handle after synchronising the device work it
 * queued.  NULL-safe. */
GPV_API int gp_voxels_destroy(gp_voxels_t* h);

/* Voxel-GPR of a CSR batch of voxels (Alg. 1 lines 2-22, Eq. 2-3 of Sec. 3.1).
 * Inputs (device, FP32 unless stated):
 *   d_xyz [N, 3]        points of all voxels, voxel by voxel
 *   d_offsets [nvox+1]  int64; voxel v owns points offsets[v] .. offsets[v+1]-1
 *   d_centres [nvox, 3] voxel centres (local frame origin)
 *   d_lambda, d_sf2, d_sn2 [nvox]  kernel k(a,b) = sf2 exp(-lambda |a-b|^2) and noise
 *                       variance sigma^2 of Eq. 2, per voxel
 * Outputs (device, caller-owned):
 *   d_axis [nvox]       uint8 value axis 0/1/2 (255 when below tau)
 *   d_mean, d_var [nvox, G*G]  posterior mean mu* and diag(Sigma*) (Eq. 3)
 *   d_status [nvox]     GPV_VOX_* bits
 *   d_pos [nvox*n_s^2, 3], d_scale [.., 3], d_quat [.., 4] (w, x, y, z): optional
 *                       Gaussian initialisation fused into the solve (Sec. 3.2,
 *                       Eq. 6-8); pass all three NULL to skip it.
 * flags: 0 or GPV_SOLVE_ONE_PER_LAUNCH.
 * Voxels with n < tau or n > max_points are not solved: they get the prior
 * (mean 0, var sf2), axis 255 and GPV_VOX_BELOW_TAU / GPV_VOX_TOO_LARGE.
 * Errors: GPV_EINVAL (NULL input, nvox < 0 or > max_voxels), GPV_ECUDA. */
GPV_API int gp_voxels_solve_csr(gp_voxels_t* h, const float* d_xyz, const int64_t* d_offsets,
                        int32_t nvox, const float* d_centres, const float* d_lambda,
                        const float* d_sf2, const float* d_sn2, uint8_t* d_axis,
                        float* d_mean, float* d_var, uint32_t* d_status, float* d_pos,
                        float* d_scale, float* d_quat, uint32_t flags, gpv_stream_t stream);

/* Gaussian initialisation from given predictions (Sec. 3.2, Eq. 6-8): for each of the
 * n_s x n_s subgrids of each voxel, weights w = 1 / max(var, 1e-6 sf2), position
 * p = sum w P / sum w, Phi = sum w (P - p)(P - p)^T / sum w, then scale/rotation per
 * init_mode (see gp_voxels_config).  Inputs are the outputs of a solve (d_status may
 * be NULL); voxels flagged below tau or not SPD get scale 0 and identity rotation.
 * Outputs d_pos [nvox*n_s^2, 3] (world), d_scale [.., 3], d_quat [.., 4].
 * Errors: GPV_EINVAL, GPV_ECUDA. */
GPV_API int gp_voxels_init_gaussians(gp_voxels_t* h, int32_t nvox, const uint8_t* d_axis,
                             const float* d_centres, const float* d_sf2, const float* d_mean,
                             const float* d_var, const uint32_t* d_status, float* d_pos,
                             float* d_scale, float* d_quat, gpv_stream_t stream);

/* Device bytes a handle with this config allocates at create (solve workspaces and
 * the voxel store).  Errors: GPV_EINVAL. */
GPV_API int gp_voxels_query_sizes(const gp_voxels_config* cfg, size_t* bytes_out);

/* Static text of a gpv_status code. */
GPV_API const char* gp_voxels_strerror(int status);

/* Text of the last CUDA error seen by a call on this thread ("" if none). */
GPV_API const char* gp_voxels_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* GP_VOXELS_H */
