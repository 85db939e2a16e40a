"""Parity metrics between the CUDA path and the FP64 oracle.

TEST INFRASTRUCTURE ONLY (used by tests/, __graft_entry__.smoke() and bench.py's
reference leg).  Error metrics follow the stated tolerances:
  mean      max |mu - mu_ref|                                   (metres)
  variance  max |var - var_ref| / max(var_ref, 1e-3 sigma^2)     (relative, floored)
  scale     max |s - s_ref| / s_ref on pinned axes               (relative)
  rotation  angle between pinned eigen-directions, 2 acos |<q, q_ref>| when all pinned
An eigen-direction is pinned when its eigenvalue is separated from its neighbours by
at least 1e-3 of the largest eigenvalue; near-degenerate axes are reported, not compared.
A voxel is axis-ambiguous when its normal's two largest |components| differ by less
than 1e-3 or its smallest eigen-gap is below 1e-6 of the trace; for those the oracle is
re-run with the GPU's axis and the count is reported.
"""
from __future__ import annotations

import numpy as np

from . import oracle as O


def axis_ambiguous(pts: np.ndarray) -> bool:
    ax, nrm, ev = O.pca_axis(pts)
    a = np.sort(np.abs(nrm))
    gap = min(ev[1] - ev[0], ev[2] - ev[1])
    return bool(a[2] - a[1] < 1e-3 or gap < 1e-6 * max(ev.sum(), 1e-300))


def oracle_for_batch(b, gpu_axis: np.ndarray | None = None, mean_mode: int = 1, tau=None,
                     nthreads=None):
    """Oracle outputs for a synthetic batch; where the GPU chose another value axis on an
    axis-ambiguous voxel, that voxel is re-solved with the GPU's axis."""
    tau = b.tau if tau is None else tau
    ref = O.solve_batch(b.xyz, b.offsets, b.centres, b.lam, b.sf2, b.sn2, b.size, b.G, tau,
                        mean_mode=mean_mode, nthreads=nthreads)
    ref["ambiguous_rerun"] = 0
    if gpu_axis is None:
        return ref
    g = gpu_axis.astype(np.int32)
    solved = ref["axis"] >= 0
    diff = np.nonzero(solved & (g != ref["axis"]) & (g <= 2))[0]
    if diff.size:
        bad = [int(v) for v in diff
               if not axis_ambiguous(b.xyz[b.offsets[v]:b.offsets[v + 1]])]
        if bad:
            raise AssertionError(f"value axis differs on unambiguous voxels {bad[:10]}")
        ov = ref["axis"].copy()
        ov[diff] = g[diff]
        sub = b.subset(diff)
        r2 = O.solve_batch(sub.xyz, sub.offsets, sub.centres, sub.lam, sub.sf2, sub.sn2,
                           b.size, b.G, tau, mean_mode=mean_mode, axis_override=ov[diff],
                           nthreads=nthreads)
        for k in ("axis", "mean", "var", "status"):
            ref[k][diff] = r2[k]
        ref["ambiguous_rerun"] = int(diff.size)
    return ref


def gpr_errors(mean, var, ref, sn2, solved_mask=None) -> dict:
    """Error distribution of GPU mean/var against the oracle (FP64)."""
    mean = np.asarray(mean, dtype=np.float64)
    var = np.asarray(var, dtype=np.float64)
    m = ref["status"] == 0 if solved_mask is None else solved_mask
    if not np.any(m):
        return {"n": 0, "mean_max": 0.0, "mean_p99": 0.0, "var_max": 0.0, "var_p99": 0.0}
    em = np.abs(mean[m] - ref["mean"][m])
    floor = 1e-3 * np.asarray(sn2, dtype=np.float64)[m][:, None]
    ev = np.abs(var[m] - ref["var"][m]) / np.maximum(ref["var"][m], floor)
    per_vox_m = em.max(axis=1)
    per_vox_v = ev.max(axis=1)
    return {
        "n": int(m.sum()),
        "mean_max": float(em.max()),
        "mean_p99": float(np.quantile(per_vox_m, 0.99)),
        "var_max": float(ev.max()),
        "var_p99": float(np.quantile(per_vox_v, 0.99)),
        "worst_mean_voxel": int(np.nonzero(m)[0][np.argmax(per_vox_m)]),
        "worst_var_voxel": int(np.nonzero(m)[0][np.argmax(per_vox_v)]),
    }


def quat_to_rot(q: np.ndarray) -> np.ndarray:
    q = np.asarray(q, dtype=np.float64)
    q = q / np.linalg.norm(q, axis=-1, keepdims=True)
    w, x, y, z = q[..., 0], q[..., 1], q[..., 2], q[..., 3]
    R = np.empty(q.shape[:-1] + (3, 3))
    R[..., 0, 0] = 1 - 2 * (y * y + z * z); R[..., 0, 1] = 2 * (x * y - w * z); R[..., 0, 2] = 2 * (x * z + w * y)
    R[..., 1, 0] = 2 * (x * y + w * z); R[..., 1, 1] = 1 - 2 * (x * x + z * z); R[..., 1, 2] = 2 * (y * z - w * x)
    R[..., 2, 0] = 2 * (x * z - w * y); R[..., 2, 1] = 2 * (y * z + w * x); R[..., 2, 2] = 1 - 2 * (x * x + y * y)
    return R


def init_errors(pos, scale, quat, ref, valid=None, s_floor=None) -> dict:
    """Errors of Gaussian initialisation outputs against the oracle's, with the rule for
    pinned axes.  ``ref`` is oracle.init_batch output (arrays [V, ng, k])."""
    rp = ref["pos"].reshape(-1, 3)
    rs = ref["scale"].reshape(-1, 3)
    rq = ref["quat"].reshape(-1, 4)
    pos = np.asarray(pos, np.float64).reshape(-1, 3)
    scale = np.asarray(scale, np.float64).reshape(-1, 3)
    quat = np.asarray(quat, np.float64).reshape(-1, 4)
    if valid is None:
        valid = rs[:, 0] > 0
    pos_err = np.abs(pos[valid] - rp[valid]).max() if valid.any() else 0.0
    lam = rs[valid] ** 2
    l1 = np.maximum(lam[:, 0], 1e-300)
    gap01 = (lam[:, 0] - lam[:, 1]) / l1
    gap12 = (lam[:, 1] - lam[:, 2]) / l1
    pinned = np.stack([gap01 >= 1e-3, (gap01 >= 1e-3) & (gap12 >= 1e-3), gap12 >= 1e-3], 1)
    srel = np.abs(scale[valid] - rs[valid]) / rs[valid]
    R = quat_to_rot(quat[valid])
    Rr = quat_to_rot(rq[valid])
    cosang = np.abs(np.einsum("nik,nik->nk", R, Rr))  # per column
    ang = np.arccos(np.clip(cosang, -1.0, 1.0))
    ang_pinned = np.where(pinned, ang, 0.0)
    return {
        "n": int(valid.sum()),
        "pos_max": float(pos_err),
        "scale_rel_max": float(srel.max()) if srel.size else 0.0,
        "rot_max": float(ang_pinned.max()) if ang_pinned.size else 0.0,
        "unpinned_axes": int((~pinned).sum()),
    }
