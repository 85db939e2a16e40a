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
    GPV_VOX_NOT_SPD = 4,    /* Gram not positive definite in the final precision (in
                               FP32 also a pivot ratio (max L_ii / min L_ii)^2 above
                               esc_cond, which leaves no significant digit); prior written */
    GPV_VOX_TRUNCATED = 8,  /* bucket overflowed; oldest points were dropped */
    GPV_VOX_TOO_LARGE = 16, /* n > max_points: not processed; prior written */
    GPV_VOX_CONVERGED = 32, /* serving with the state machine on: the voxel had
                               converged (type d, Sec. 3.3), not solved; prior written */
    GPV_VOX_FAILED = 64     /* a bounded wait of the tensor-core pipeline gave up; the
                               voxel's outputs are not valid */
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
    int max_points;      /* largest n per voxel accepted by the solve (<= 1024); also the
                            bucket capacity of the voxel store */
    int max_voxels;      /* largest batch (voxels) per solve call */
    int mean_mode;       /* 0: zero prior mean (Eq. 2); 1: data mean of f */
    int precision;       /* GPV_PREC_* */
    int init_mode;       /* 0: scale = sqrt(eig Phi), rotation = eigenvectors;
                            1: Eq. 8 as printed, S = diag(Phi), R = identity */
    float esc_cond;      /* escalation threshold on (max L_ii / min L_ii)^2 (FP32:
                            voxels above it are reported GPV_VOX_NOT_SPD) */
    uint32_t hash_capacity; /* voxel slots of the device hash (power of two);
                            0 = no voxel store (batch solves only) */
    size_t mem_budget;   /* bytes the handle may allocate at create (0 = no limit) */
    /* serving (used only when hash_capacity > 0) */
    int scan_slots;      /* scans that may be in flight at once (1..64) */
    int max_scan_points; /* points per scan (<= 2^20) */
    int max_scan_voxels; /* visited voxels per scan = rows of a serving solve */
    int64_t snap_points; /* points of one scan's solve snapshot
                            (0 = max_scan_voxels * max_points) */
    float lambda, sf2, sn2; /* kernel and noise of the serving solve (Sec. 3.1 uses
                            lambda = 1 and no signal variance, sf2 = 1) */
    /* voxel state machine of Sec. 3.3 (serving only; eta <= 0 turns it off) */
    float eta;           /* convergence threshold: a solved voxel whose mean predicted
                            variance over its G x G nodes is <= eta * sf2 is converged
                            (type d) and no longer solved; paper: 0.3 (hyperparameter
                            table) */
    float noise_floor;   /* lower bound of a point's fed-back noise variance (keeps the
                            Gram matrix conditioned); the paper gives none */
    int factor_panel;    /* 0: default factor (per column for 8-byte voxels up to 96
                            points, else blocked with 16-column panels); 4, 8 or 16: the
                            blocked shared-memory Cholesky with that panel width for every
                            voxel; gp_voxels_autotune may choose otherwise per size bucket */
    int tc_workspace_mb; /* GPV_PREC_MIXED solves: MiB of device workspace, in total, for the
                            posterior variance on the tensor cores (Eq. 3, diag(Sigma*) by
                            exact BF16 slice products; well-conditioned voxels of up to 255
                            points).  Split evenly between the batch entry and, with the
                            voxel store on and the state machine off (eta <= 0), each
                            scan slot; each share is capped by what
                            its voxels (max_voxels, max_scan_voxels) could use and, under
                            mem_budget, by what the budget leaves; a share below 16 MiB is
                            dropped.  A call whose eligible voxels need more than its share
                            forms every variance on the CUDA cores instead, so the choice
                            never depends on scheduling.  0 turns it off; default 4096. */
    int refine;          /* GPV_PREC_FP32 solves: 1 (default) adds one step of iterative
                            refinement of alpha = (K + sigma^2 I)^-1 (f - m): the residual
                            r = (f - m) - (K + sigma^2 I) alpha is accumulated in float-float,
                            the FP32 factor solves for the correction, and the mean of Eq. 3
                            is accumulated in float-float; 0: plain FP32 throughout */
    int tall_min_points; /* GPV_PREC_MIXED and GPV_PREC_FP32 batch solves: voxels with more
                            points than this take the tensor-core factorisation of the tall
                            matrix [K + sigma^2 I; K*^T] (left-looking Cholesky whose
                            updates are exact BF16 slice products; no L^-1); 0 (default):
                            every voxel too large for the shared-memory kernels; -1: off
                            (those voxels keep the global-workspace kernel) */
} gp_voxels_config;

/* Voxel types of Sec. 3.3 (gp_voxels_scan_types, gp_voxels_type_counts). */
enum {
    GPV_TYPE_A = 0, /* fewer than tau points: not processed */
    GPV_TYPE_B = 1, /* at least tau points, not yet solved into the map */
    GPV_TYPE_C = 2, /* solved, mean variance above eta * sf2: active, re-solved when
                       new points arrive, with the fed-back noise of its old points */
    GPV_TYPE_D = 3  /* converged: not processed any more */
};

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

/* Voxel-GPR with a noise variance per point (Sec. 3.3: the points of an active voxel
 * carry the variance estimated by its previous solve, new points the sensor's).  As
 * gp_voxels_solve_csr, with the Gram diagonal sf2 + d_noise[p] instead of sf2 + sn2:
 *   d_noise [N]   FP32 noise variance of every point (NULL: d_sn2 of its voxel)
 *   d_pvar  [N]   optional output: posterior variance of the latent surface at every
 *                 input, sf2 - k_p^T (K + D)^-1 k_p with k_p the kernel column of point
 *                 p (no noise); computed as d_p (1 - d_p [(K + D)^-1]_pp).  Left
 *                 unwritten for voxels not solved (status BELOW_TAU, TOO_LARGE, NOT_SPD).
 * In GPV_PREC_FP32 the subtraction in d_pvar loses about log10(n) digits of FP32;
 * use GPV_PREC_MIXED or FP64 where d_pvar feeds the next solve.
 * Errors: GPV_EINVAL, GPV_ECUDA. */
GPV_API int gp_voxels_solve_csr_noise(gp_voxels_t* h, const float* d_xyz,
                              const int64_t* d_offsets, int32_t nvox, const float* d_centres,
                              const float* d_lambda, const float* d_sf2, const float* d_sn2,
                              const float* d_noise, uint8_t* d_axis, float* d_mean,
                              float* d_var, uint32_t* d_status, float* d_pos, float* d_scale,
                              float* d_quat, float* d_pvar, uint32_t flags,
                              gpv_stream_t stream);

/* The paper's own formulation of the solve (supplementary Alg. 3), for comparison and
 * for the full posterior covariance: ky = K + sigma^2 I, LU with partial pivoting, the
 * explicit inverse ky^-1, k_k* = K*^T ky^-1, mu* = k_k* f and the FULL
 * Sigma* = K** - k_k* K* over the G^2 query nodes, all in FP32 as the paper's
 * single-precision library routines (the last product on the tensor cores as three TF32
 * products, which keeps FP32-level accuracy).  Value axis, local frame, grid, prior mean
 * (mean_mode) and kernel as gp_voxels_solve_csr; config precision is ignored.
 * Inputs as gp_voxels_solve_csr.  Outputs (device, caller-owned):
 *   d_axis [nvox] u8, d_mean [nvox, G*G], d_status [nvox] (GPV_VOX_* bits),
 *   d_cov [nvox, G*G, G*G] FP32 row-major: Sigma*(q, q') at d_cov[(v G^2 + q) G^2 + q'].
 * Every voxel up to max_points is solved: ky lives in one CTA's shared memory up to about
 * 200 points at G = 16, in a global-memory slice per CTA above (one persistent launch per
 * chunk for those).  Voxels below tau, above max_points (GPV_VOX_TOO_LARGE) or whose FP32 LU
 * meets a zero pivot (GPV_VOX_NOT_SPD) get mean 0 and the prior K**.  FP32 LU and inverse
 * lose about log10(cond(ky)) digits: on dense voxels the variances are far less accurate
 * than gp_voxels_solve_csr's.  The first call allocates a workspace of about 512 MB plus,
 * when max_points exceeds the shared-memory size, one kp x kp FP32 matrix per SM
 * (kp = max_points rounded up to 32; 600 MB at 1024 points), counted against mem_budget;
 * later calls allocate nothing.  h_nmax (may be NULL) receives the largest n solved
 * (max_points).  Errors: GPV_EINVAL, GPV_EBUDGET, GPV_ENOMEM, GPV_ECUDA. */
GPV_API int gp_voxels_solve_alg3(gp_voxels_t* h, const float* d_xyz, const int64_t* d_offsets,
                                 int32_t nvox, const float* d_centres, const float* d_lambda,
                                 const float* d_sf2, const float* d_sn2, uint8_t* d_axis,
                                 float* d_mean, float* d_cov, uint32_t* d_status,
                                 gpv_stream_t stream, int32_t* h_nmax);

/* Structure similarity loss of Eq. 11 (Sec. 3.3) between a set of 3D Gaussians and a
 * scan: for every scan point P_j, best_j = min over the Gaussians k of
 * |P_j - p_k| - mean(S_k) (the minimum of the expression as printed, which can pick a
 * farther Gaussian with a larger scale than the nearest one), and L_p = mean_j best_j.
 *   d_gpos [m, 3], d_gscale [m, 3]: Gaussian centres and scales (FP32, e.g. the d_pos
 *       and d_scale outputs of a solve), m >= 1
 *   d_points [n, 3]: the scan (FP32 world coordinates)
 *   cell: side of the hash-grid cells the Gaussians are binned in (about their spacing,
 *       e.g. voxel_size / n_s); any positive value gives the same result, only faster
 *       or slower
 * Outputs (device): d_best [n] FP32 and d_arg [n] int32 (the minimising k; ties: the
 * smallest k), either may be NULL; d_loss [1] FP64 (mean over the points, fixed-order
 * summation); d_info [2] int32 (optional): points settled by the exhaustive pass (no
 * Gaussian within 16 cells), and 1 if the hash table overflowed (never with its sizing).
 * The search is exact: cells are visited in growing rings until no farther Gaussian can
 * beat the best value.  A call with more Gaussians or points than any earlier call of
 * the handle grows its workspace (allocates, synchronises the device).
 * Errors: GPV_EINVAL, GPV_EBUDGET, GPV_ENOMEM, GPV_ECUDA. */
GPV_API int gp_voxels_structure_loss(gp_voxels_t* h, const float* d_gpos, const float* d_gscale,
                                     int32_t m, const float* d_points, int32_t n, float cell,
                                     float* d_best, int32_t* d_arg, double* d_loss,
                                     int32_t* d_info, gpv_stream_t stream);

/* A pinhole camera for gp_voxels_render: camera coordinates t = R p + t_wc of a world
 * point p (R row-major), image coordinates u = fx t_x / t_z + cx, v = fy t_y / t_z + cy in
 * pixels (pixel (x, y) spans [x, x + 1) x [y, y + 1), its centre at x + 1/2, y + 1/2). */
typedef struct {
    float R[9];
    float t[3];
    float fx, fy, cx, cy;
    int width, height;
    float near;  /* Gaussians with t_z <= near are not drawn */
} gp_raster_camera;

/* Rasterisation of 3D Gaussians into colour, depth and silhouette images (Sec. 3.3, Eq. 9,
 * with depth and silhouette blended alike): every Gaussian with t_z > near is projected
 * (covariance R diag(scale^2) R^T from the unit quaternion, Sigma' = J R_c Sigma R_c^T J^T
 * + 0.3 I with the perspective Jacobian J, its t_x / t_z and t_y / t_z clamped to 1.3 times
 * the half field of view) and reaches the pixels whose centres lie within
 * r = ceil(3 sqrt(lambda_max(Sigma'))) of its projected centre along both image axes;
 * there alpha = min(0.99, opacity exp(-d^T Sigma'^-1 d / 2)), ignored below 1/255.  In
 * order of depth t_z (ties: lower index), front to back: C += color alpha T, D += t_z alpha
 * T, S += alpha T, T *= 1 - alpha, stopping before a Gaussian that would take T below 1e-4.
 *   d_pos, d_scale [m, 3], d_quat [m, 4] (w, x, y, z), d_opacity [m], d_color [m, 3]: FP32
 *   outputs: d_image [H, W, 3], d_depth [H, W], d_silhouette [H, W] FP32 (every pixel written)
 * Synchronises `stream` once (the size of the per-tile lists decides their buffer, which
 * is grown when needed).  *h_pairs (may be NULL): (tile, Gaussian) pairs.
 * Errors: GPV_EINVAL, GPV_ENOMEM, GPV_EFULL (more than 2^31 - 1 pairs), GPV_ECUDA. */
GPV_API int gp_voxels_render(gp_voxels_t* h, const float* d_pos, const float* d_scale,
                             const float* d_quat, const float* d_opacity, const float* d_color,
                             int32_t m, const gp_raster_camera* cam, float* d_image,
                             float* d_depth, float* d_silhouette, gpv_stream_t stream,
                             int64_t* h_pairs);

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

/* ---- serving: the voxel store of Alg. 2 and re-solves of visited voxels ---------
 * A handle created with hash_capacity > 0 keeps, on the device, an open-addressing
 * hash from voxel key floor(p / s) (FP32, IEEE division) to a bucket of at most
 * max_points points per voxel.  A full bucket drops its oldest points; the points of a
 * bucket are kept in (scan, index-in-scan) order, so results do not depend on how
 * concurrent work interleaves.  scan_slots slots hold the state of the scans in
 * flight; their memory is reserved at create (and counted against mem_budget), so
 * admitting a scan is admitting it by memory.  Each slot has its own solve workspace:
 * solves of different slots may run concurrently on different streams.
 */

/* ALG.STORE (supplementary Alg. 2) for one LiDAR scan: every point is pushed into the
 * bucket of its voxel and the visited voxels form S_updated (each listed once, in the
 * order of their first point in the scan).  The call then copies the buckets of the
 * visited voxels (points after this scan) into the scan's slot, so a later
 * gp_voxels_solve of the slot sees exactly this state, whatever later scans insert.
 * Inserts are ordered by call order across all streams.
 * d_xyz: device FP32 [npts, 3] world points, caller-owned, read on `stream`.
 * *slot_out: the slot holding this scan until gp_voxels_release_scan.
 * Errors: GPV_EINVAL (no store, NULL, npts < 0 or > max_scan_points), GPV_EFULL (every
 * slot is in use: release one and retry), GPV_ECUDA.  A full hash, a scan visiting
 * more than max_scan_voxels voxels or a full snapshot are reported by
 * gp_voxels_scan_info, not as errors. */
GPV_API int gp_voxels_insert_scan(gp_voxels_t* h, const float* d_xyz, int64_t npts,
                                  uint64_t scan_id, gpv_stream_t stream, int32_t* slot_out);

/* Voxel-GPR of the visited voxels of a slot (Alg. 1 body over S_updated), rows in
 * S_updated order: the same outputs as gp_voxels_solve_csr, with buffers of
 * max_scan_voxels rows (the row count stays on the device; gp_voxels_scan_info returns
 * it), plus optional d_keys [rows] (packed voxel keys, 21 bits per axis, offset 2^20)
 * and d_centres [rows, 3].  Kernel and noise are the config's lambda, sf2, sn2.
 * Voxels whose bucket dropped points carry GPV_VOX_TRUNCATED.  No host sync.
 * Errors: GPV_EINVAL (bad slot, NULL output), GPV_ECUDA. */
GPV_API int gp_voxels_solve(gp_voxels_t* h, int32_t slot, uint8_t* d_axis, float* d_mean,
                            float* d_var, uint32_t* d_status, float* d_pos, float* d_scale,
                            float* d_quat, int64_t* d_keys, float* d_centres,
                            gpv_stream_t stream);

/* With the state machine on (eta > 0), the serving path follows Sec. 3.3:
 *  - every stored point carries a noise variance: the config's sn2 when inserted,
 *    then the posterior variance at that point from the last solve of its voxel
 *    (at least noise_floor);
 *  - gp_voxels_insert_scan records the type of every visited voxel: (a) fewer than tau
 *    points, (b) enough points but never solved, (c) active, (d) converged;
 *  - gp_voxels_solve solves the rows of types (b) and (c) with those per-point noises,
 *    writes the posterior variance back to the points, and moves each solved voxel to
 *    (d) when its mean predicted variance is <= eta * sf2, else to (c).  Rows of type
 *    (d) get GPV_VOX_CONVERGED and the prior.
 * Types depend on the previous scans' solves, so in this mode each scan must be solved
 * before the next one is inserted: gp_voxels_insert_scan returns GPV_EINVAL while an
 * inserted scan awaits its gp_voxels_solve, and it waits on the device for that
 * solve's state update. */

/* Voxel type (GPV_TYPE_*) of every row of a solved slot, before (d_before) and after
 * (d_after) the solve, uint8 [max_scan_voxels] each, either may be NULL.  After the
 * solve a voxel that could not be solved (NOT_SPD, TOO_LARGE) keeps type (b) or (c).
 * Errors: GPV_EINVAL (no store, state machine off, bad slot), GPV_ECUDA. */
GPV_API int gp_voxels_scan_types(gp_voxels_t* h, int32_t slot, uint8_t* d_before,
                                 uint8_t* d_after, gpv_stream_t stream);

/* Number of stored voxels of each type (a)-(d) after the work queued so far
 * (synchronises the device): h_counts[4].  Errors: GPV_EINVAL, GPV_ECUDA. */
GPV_API int gp_voxels_type_counts(gp_voxels_t* h, int64_t* h_counts);

/* Counts of a slot's scan: rows (visited voxels, at most max_scan_voxels), snapshot
 * points, flags (bit 0: hash full, points dropped; bit 1: more than max_scan_voxels
 * visited; bit 2: snapshot full).  Synchronises `stream`.  Errors: GPV_EINVAL, GPV_ECUDA. */
GPV_API int gp_voxels_scan_info(gp_voxels_t* h, int32_t slot, gpv_stream_t stream,
                                int32_t* h_rows, int64_t* h_points, uint32_t* h_flags);

/* Give a slot back.  It is reused only after the work queued on `stream` so far has
 * completed (no host wait), so pass the stream that read the slot's outputs.
 * Errors: GPV_EINVAL, GPV_ECUDA. */
GPV_API int gp_voxels_release_scan(gp_voxels_t* h, int32_t slot, gpv_stream_t stream);

/* Voxels currently held by the store (synchronises the device).  Errors: GPV_EINVAL,
 * GPV_ECUDA. */
GPV_API int gp_voxels_store_voxels(gp_voxels_t* h, int64_t* h_voxels);

/* ---- allocation-free batched solve -------------------------------------------------
 * No counterpart in the paper: an entry point for callers that may not allocate device
 * memory themselves or through this library -- for example code running inside a host
 * application that owns every device allocation under a fixed memory plan, or an op of
 * another framework that may only use the tensors it is handed.  It solves a CSR batch
 * like gp_voxels_solve_csr (same inputs, outputs, layouts and per-voxel status), without
 * a handle, using a static scratch area that the library holds on every GPU it is loaded
 * on (about 0.8 MB, kept until the process exits).
 *  - cfg: the configuration a handle would take (fields of the voxel store and of
 *    serving are ignored); precision FP32, MIXED or FP64.
 *  - At most GPV_NOALLOC_MAX_VOXELS voxels per call; larger batches get GPV_EINVAL.
 *  - Voxels whose factor does not fit shared memory (in FP32 about 256 points at
 *    G <= 16; in the 8-byte precisions about 176) are not solved and get
 *    GPV_VOX_TOO_LARGE; gp_voxels_solve_csr handles them.
 *  - The first call on a device looks up the scratch area's device address (again after
 *    the device's context has been replaced, e.g. by cudaDeviceReset); make that first
 *    call before capturing a stream.
 *  - cfg->factor_panel must be 0, 4, 8 or 16, as for gp_voxels_create.
 *  - All calls share the scratch area: calls whose GPU work overlaps (on different
 *    streams, or from several threads) race and give wrong results.  Serialise them.
 *  - No cudaMalloc, cudaFree or other allocating call is made.
 * Errors: GPV_EINVAL (bad config, NULL, nvox out of range), GPV_ECUDA. */
#define GPV_NOALLOC_MAX_VOXELS 65536
GPV_API int gp_voxels_solve_csr_noalloc(const gp_voxels_config* cfg, const float* d_xyz,
                                        const int64_t* d_offsets, int32_t nvox,
                                        const float* d_centres, const float* d_lambda,
                                        const float* d_sf2, const float* d_sn2,
                                        uint8_t* d_axis, float* d_mean, float* d_var,
                                        uint32_t* d_status, float* d_pos, float* d_scale,
                                        float* d_quat, gpv_stream_t stream);

/* Device bytes a handle with this config allocates at create (solve workspaces and
 * the voxel store).  Errors: GPV_EINVAL. */
GPV_API int gp_voxels_query_sizes(const gp_voxels_config* cfg, size_t* bytes_out);

/* Autotuner of the batched solve (the paper has no counterpart; its batch is a library
 * call): runs every size bucket of this batch with each candidate CTA size (128, 256 and
 * 512 threads, at least the bucket's largest n for shared-memory factors) and factor
 * variant (blocked with 16-, 8- or 4-column panels, or per column; shared-memory buckets),
 * persistent grids sized by occupancy, and keeps the fastest per bucket in the
 * handle for later solves of any batch.  Inputs and outputs as gp_voxels_solve_csr (the
 * outputs are overwritten with scratch results; the FP64 escalation is not run).
 * Synchronises `stream`.  *h_changed = buckets whose choice changed.
 * Errors: GPV_EINVAL, GPV_ECUDA. */
GPV_API int gp_voxels_autotune(gp_voxels_t* h, const float* d_xyz, const int64_t* d_offsets,
                               int32_t nvox, const float* d_centres, const float* d_lambda,
                               const float* d_sf2, const float* d_sn2, uint8_t* d_axis,
                               float* d_mean, float* d_var, uint32_t* d_status, float* d_pos,
                               float* d_scale, float* d_quat, gpv_stream_t stream,
                               int32_t* h_changed);

/* Number of CUDA kernels the last gp_voxels_solve_csr / gp_voxels_solve call of this
 * handle queued (a diagnostic; the paper has no counterpart).  Errors: GPV_EINVAL. */
GPV_API int gp_voxels_last_launches(const gp_voxels_t* h, int32_t* h_kernels);

/* Launch plan of this handle (a diagnostic; the paper has no counterpart):
 * h_info[0] = tall_min (voxels with more points take the tall-matrix tensor-core path; -1:
 * the path is off), [1] = largest n of the tensor-core variance with the factor in shared
 * memory (0: off), [2] = largest n of the shared-memory solve kernels, [3] = size buckets.
 * Errors: GPV_EINVAL. */
GPV_API int gp_voxels_plan_info(const gp_voxels_t* h, int32_t* h_info);

/* Size buckets of this handle's launch plan, as the defaults or gp_voxels_autotune left
 * them (a diagnostic; the paper has no counterpart).  Writes min(cap, buckets) records of
 * five int32 each to h_info: largest n of the bucket, path (0 = shared-memory solve,
 * 1 = global-workspace solve, 2 = tall-matrix path, 3 = shared-memory solve handing its
 * variance to the tensor cores), CTA threads, per-column factor (0/1), panel width of the
 * blocked factor; *h_count = number of buckets.  Host memory, owned by the caller.
 * Errors: GPV_EINVAL (null pointers, cap < 0). */
GPV_API int gp_voxels_bucket_info(const gp_voxels_t* h, int32_t* h_info, int32_t cap,
                                  int32_t* h_count);

/* Device time of the tall-matrix launches of this handle's batch solves (a diagnostic for
 * roofline measurement; the paper has no counterpart).  gp_voxels_set_timing(h, 1) makes
 * every later gp_voxels_solve_csr record CUDA events on the stream of those launches
 * around them (also inside a stream capture: the records become part of the graph);
 * gp_voxels_last_tall_ms waits for the last recorded end event and returns the elapsed
 * milliseconds (0 when the last solve had no tall-matrix voxels).  Errors: GPV_EINVAL,
 * GPV_ECUDA. */
GPV_API int gp_voxels_set_timing(gp_voxels_t* h, int32_t on);
GPV_API int gp_voxels_last_tall_ms(gp_voxels_t* h, float* h_ms);

/* Arithmetic peak of this GPU measured with the solve's own arithmetic (the paper has no
 * counterpart; a reference for roofline fractions): kind 0 = FP32 fused multiply-add, kind 1
 * = the float-float accumulate-form multiply-add of the variance contraction; 2 flops per
 * multiply-add, eight independent chains per thread on every SM, best of three launches.
 * Synchronises `stream`.  Errors: GPV_EINVAL, GPV_ECUDA. */
GPV_API int gp_voxels_measure_peak(int kind, gpv_stream_t stream, double* h_tflops);

/* Self-test of the bounded waits (no counterpart in the paper): every wait of this
 * library's kernels on an mbarrier polls at most a fixed number of times, then reports
 * (GPV_VOX_FAILED) and returns instead of hanging.  This call runs one such wait on an
 * mbarrier that nothing arrives at, with `polls` tries (1 .. 2^24), and sets
 * *h_timed_out = 1 when the wait gave up as it must.  Synchronises `stream`.
 * Errors: GPV_EINVAL, GPV_ECUDA. */
GPV_API int gp_voxels_selftest_bounded_wait(uint32_t polls, gpv_stream_t stream,
                                            int32_t* h_timed_out);

/* Static text of a gpv_status code. */
GPV_API const char* gp_voxels_strerror(int status);

/* Text of the last CUDA error seen by a call on this thread ("" if none). */
GPV_API const char* gp_voxels_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* GP_VOXELS_H */
