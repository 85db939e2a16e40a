"""ctypes front end of the FP64 CPU oracle (``gp_oracle.c``) plus the voxel store of
Alg. 2, for tests and the CPU legs of the benchmark.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this module.
The CUDA product path (``paper_2410_17084_b300``) never imports it.

Functions follow GS-LIVM (arXiv 2410.17084): Voxel-GPR of Sec. 3.1 (Alg. 1, Eq. 2-3),
the Gaussian initialisation of Sec. 3.2 (Eq. 6-8) and ALG.STORE / ALG.HASH of the
supplementary Alg. 2, and the voxel state machine with variance feedback of Sec. 3.3.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gp_oracle.c")
_LIB = os.path.join(_HERE, "libgp_oracle.so")

BELOW_TAU = 1
NOT_SPD = 4
CONVERGED = 32  # map update of Sec. 3.3: a converged voxel is not solved


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (IEEE FP64, no fast-math, no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        subprocess.check_call([
            "gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
            "-fno-fast-math", "-o", _LIB, _SRC, "-lm", "-lpthread",
        ])
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        _lib.gpo_eig3.argtypes = [P, P, P]
        _lib.gpo_voxel_key.argtypes = [P, ctypes.c_int64, ctypes.c_float, P]
        _lib.gpo_voxel_centre.argtypes = [P, ctypes.c_int64, ctypes.c_float, P]
        _lib.gpo_pca_axis.argtypes = [P, ctypes.c_int64, P, P]
        _lib.gpo_pca_axis.restype = ctypes.c_int
        _lib.gpo_solve_voxel.argtypes = [P, ctypes.c_int64, P, ctypes.c_double, ctypes.c_int,
                                         ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                         ctypes.c_int, ctypes.c_int, P, P, P]
        _lib.gpo_solve_voxel_hetero.argtypes = [P, ctypes.c_int64, P, ctypes.c_double, ctypes.c_int,
                                                ctypes.c_double, ctypes.c_double, P, ctypes.c_int,
                                                ctypes.c_int, P, P, P, P]
        _lib.gpo_solve_voxel_fullcov.argtypes = [P, ctypes.c_int64, P, ctypes.c_double, ctypes.c_int,
                                                 ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                                 ctypes.c_int, ctypes.c_int, P, P, P]
        _lib.gpo_structure_loss.argtypes = [P, ctypes.c_int64, P, P, ctypes.c_int64, P, P]
        _lib.gpo_structure_loss.restype = ctypes.c_double
        _lib.gpo_rasterize.argtypes = [P, P, P, P, P, ctypes.c_int64, P, P, ctypes.c_double,
                                       ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                       ctypes.c_int, ctypes.c_int, ctypes.c_double, P, P, P, P]
        _lib.gpo_init_voxel.argtypes = [P, P, ctypes.c_int, P, ctypes.c_double, ctypes.c_int,
                                        ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                        ctypes.c_int, P, P, P, P]
        _lib.gpo_solve_batch.argtypes = [P, P, ctypes.c_int64, P, P, P, P, ctypes.c_double,
                                         ctypes.c_int, ctypes.c_int, ctypes.c_int, P,
                                         ctypes.c_int, P, P, P, P]
        _lib.gpo_init_batch.argtypes = [P, P, P, P, P, ctypes.c_int64, ctypes.c_double,
                                        ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                        P, P, P]
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def eig3(A) -> tuple[np.ndarray, np.ndarray]:
    """Jacobi eigen decomposition of a symmetric 3x3 matrix: (evals, V columns)."""
    A = np.ascontiguousarray(A, dtype=np.float64).reshape(3, 3)
    ev = np.zeros(3)
    V = np.zeros((3, 3))
    lib().gpo_eig3(_p(A), _p(ev), _p(V))
    return ev, V


def voxel_keys(xyz: np.ndarray, size: float) -> np.ndarray:
    """ALG.HASH: integer voxel index floor(p / size), decided in FP32."""
    xyz = np.ascontiguousarray(xyz, dtype=np.float32)
    out = np.zeros((xyz.shape[0], 3), dtype=np.int32)
    lib().gpo_voxel_key(_p(xyz), xyz.shape[0], float(size), _p(out))
    return out


def voxel_centres(keys3: np.ndarray, size: float) -> np.ndarray:
    keys3 = np.ascontiguousarray(keys3, dtype=np.int32)
    out = np.zeros((keys3.shape[0], 3), dtype=np.float32)
    lib().gpo_voxel_centre(_p(keys3), keys3.shape[0], float(size), _p(out))
    return out


def pca_axis(xyz: np.ndarray):
    """ALG.PCA + value-axis switch: (axis, normal, ascending eigenvalues)."""
    xyz = np.ascontiguousarray(xyz, dtype=np.float32)
    nrm = np.zeros(3)
    ev = np.zeros(3)
    ax = lib().gpo_pca_axis(_p(xyz), xyz.shape[0], _p(nrm), _p(ev))
    return ax, nrm, ev


def solve_voxel(xyz, centre, size, G, lam, sf2, sn2, mean_mode=1, axis_override=-1):
    """Voxel-GPR of one voxel: (status, axis, mean[G*G], var[G*G])."""
    xyz = np.ascontiguousarray(xyz, dtype=np.float32).reshape(-1, 3)
    centre = np.ascontiguousarray(centre, dtype=np.float32).reshape(3)
    mean = np.zeros(G * G)
    var = np.zeros(G * G)
    ax = ctypes.c_int(0)
    st = lib().gpo_solve_voxel(_p(xyz), xyz.shape[0], _p(centre), float(size), int(G),
                               float(lam), float(sf2), float(sn2), int(mean_mode),
                               int(axis_override), ctypes.byref(ax), _p(mean), _p(var))
    return st, ax.value, mean, var


def solve_voxel_hetero(xyz, centre, size, G, lam, sf2, noise, mean_mode=1, axis_override=-1):
    """Voxel-GPR with a noise variance per training point (Sec. 3.3): (status, axis,
    mean[G*G], var[G*G], pvar[n]) with pvar the posterior variance at the inputs."""
    xyz = np.ascontiguousarray(xyz, dtype=np.float32).reshape(-1, 3)
    centre = np.ascontiguousarray(centre, dtype=np.float32).reshape(3)
    noise = np.ascontiguousarray(noise, dtype=np.float64).reshape(-1)
    mean = np.zeros(G * G)
    var = np.zeros(G * G)
    pvar = np.zeros(xyz.shape[0])
    ax = ctypes.c_int(0)
    st = lib().gpo_solve_voxel_hetero(_p(xyz), xyz.shape[0], _p(centre), float(size), int(G),
                                      float(lam), float(sf2), _p(noise), int(mean_mode),
                                      int(axis_override), ctypes.byref(ax), _p(mean), _p(var),
                                      _p(pvar))
    return st, ax.value, mean, var, pvar


def solve_voxel_fullcov(xyz, centre, size, G, lam, sf2, sn2, mean_mode=1, axis_override=-1):
    """Posterior mean and full G^2 x G^2 covariance Sigma* of the query nodes (Eq. 3,
    the Sigma* of the supplementary Alg. 3): (status, axis, mean[G*G], cov[G*G, G*G])."""
    xyz = np.ascontiguousarray(xyz, dtype=np.float32).reshape(-1, 3)
    centre = np.ascontiguousarray(centre, dtype=np.float32).reshape(3)
    Q = G * G
    mean = np.zeros(Q)
    cov = np.zeros((Q, Q))
    ax = ctypes.c_int(0)
    st = lib().gpo_solve_voxel_fullcov(_p(xyz), xyz.shape[0], _p(centre), float(size), int(G),
                                       float(lam), float(sf2), float(sn2), int(mean_mode),
                                       int(axis_override), ctypes.byref(ax), _p(mean), _p(cov))
    return st, ax.value, mean, cov


def structure_loss(points, gpos, gscale):
    """Structure similarity loss of Eq. 11 by brute force: (L_p, best[n], arg[n]) with
    best[j] = min_k |P_j - p_k| - mean(S_k) and arg[j] its k (ties: smallest k)."""
    pts = np.ascontiguousarray(points, dtype=np.float32).reshape(-1, 3)
    gp = np.ascontiguousarray(gpos, dtype=np.float32).reshape(-1, 3)
    gs = np.ascontiguousarray(gscale, dtype=np.float32).reshape(-1, 3)
    best = np.zeros(pts.shape[0])
    arg = np.zeros(pts.shape[0], dtype=np.int64)
    loss = lib().gpo_structure_loss(_p(pts), pts.shape[0], _p(gp), _p(gs), gp.shape[0],
                                    _p(best), _p(arg))
    return loss, best, arg


def rasterize(pos, scale, quat, opacity, color, Rc, tc, fx, fy, cx, cy, W, H, near=0.2):
    """Colour, depth and silhouette images of Eq. 9 (front-to-back alpha blending of the
    projected Gaussians; see gpo_rasterize): (C [H, W, 3], D [H, W], S [H, W], amb [H, W])
    with amb marking pixels where a threshold decision is within rounding."""
    f32 = lambda a, k: np.ascontiguousarray(a, dtype=np.float32).reshape(-1, k)
    pos, scale, quat, color = f32(pos, 3), f32(scale, 3), f32(quat, 4), f32(color, 3)
    opacity = np.ascontiguousarray(opacity, dtype=np.float32).reshape(-1)
    Rc = np.ascontiguousarray(Rc, dtype=np.float64).reshape(3, 3)
    tc = np.ascontiguousarray(tc, dtype=np.float64).reshape(3)
    C = np.zeros((H, W, 3))
    D = np.zeros((H, W))
    S = np.zeros((H, W))
    amb = np.zeros((H, W), dtype=np.uint8)
    lib().gpo_rasterize(_p(pos), _p(scale), _p(quat), _p(opacity), _p(color), pos.shape[0],
                        _p(Rc), _p(tc), float(fx), float(fy), float(cx), float(cy), int(W),
                        int(H), float(near), _p(C), _p(D), _p(S), _p(amb))
    return C, D, S, amb


def init_voxel(mean, var, axis, centre, size, G, n_s, n_r, sf2, init_mode=0):
    """Gaussian initialisation of one voxel: (pos, scale, quat, Phi) per subgrid."""
    mean = np.ascontiguousarray(mean, dtype=np.float64)
    var = np.ascontiguousarray(var, dtype=np.float64)
    centre = np.ascontiguousarray(centre, dtype=np.float32).reshape(3)
    ng = n_s * n_s
    pos = np.zeros((ng, 3)); scale = np.zeros((ng, 3)); quat = np.zeros((ng, 4))
    phi = np.zeros((ng, 3, 3))
    rc = lib().gpo_init_voxel(_p(mean), _p(var), int(axis), _p(centre), float(size), int(G),
                              int(n_s), int(n_r), float(sf2), int(init_mode), _p(pos),
                              _p(scale), _p(quat), _p(phi))
    if rc != 0:
        raise ValueError("bad init arguments")
    return pos, scale, quat, phi


def solve_batch(xyz, offsets, centres, lam, sf2, sn2, size, G, tau, mean_mode=1,
                axis_override=None, nthreads=None):
    """Voxel-GPR over a CSR batch of voxels; returns dict of FP64 outputs."""
    xyz = np.ascontiguousarray(xyz, dtype=np.float32).reshape(-1, 3)
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    nvox = offsets.shape[0] - 1
    centres = np.ascontiguousarray(centres, dtype=np.float32).reshape(nvox, 3)
    lam = np.ascontiguousarray(np.broadcast_to(np.float32(lam) if np.isscalar(lam) else lam,
                                               (nvox,)), dtype=np.float32)
    sf2 = np.ascontiguousarray(np.broadcast_to(np.float32(sf2) if np.isscalar(sf2) else sf2,
                                               (nvox,)), dtype=np.float32)
    sn2 = np.ascontiguousarray(np.broadcast_to(np.float32(sn2) if np.isscalar(sn2) else sn2,
                                               (nvox,)), dtype=np.float32)
    ov = None
    if axis_override is not None:
        ov = np.ascontiguousarray(axis_override, dtype=np.int32)
    axis = np.zeros(nvox, dtype=np.int32)
    mean = np.zeros((nvox, G * G))
    var = np.zeros((nvox, G * G))
    status = np.zeros(nvox, dtype=np.int32)
    nthreads = nthreads or os.cpu_count() or 1
    lib().gpo_solve_batch(_p(xyz), _p(offsets), nvox, _p(centres), _p(lam), _p(sf2), _p(sn2),
                          float(size), int(G), int(tau), int(mean_mode),
                          _p(ov) if ov is not None else None, int(nthreads), _p(axis),
                          _p(mean), _p(var), _p(status))
    return {"axis": axis, "mean": mean, "var": var, "status": status, "nthreads": nthreads}


def init_batch(mean, var, axis, centres, sf2, size, G, n_s, n_r, init_mode=0):
    mean = np.ascontiguousarray(mean, dtype=np.float64)
    var = np.ascontiguousarray(var, dtype=np.float64)
    axis = np.ascontiguousarray(axis, dtype=np.int32)
    nvox = axis.shape[0]
    centres = np.ascontiguousarray(centres, dtype=np.float32).reshape(nvox, 3)
    sf2 = np.ascontiguousarray(np.broadcast_to(np.float32(sf2) if np.isscalar(sf2) else sf2,
                                               (nvox,)), dtype=np.float32)
    ng = n_s * n_s
    pos = np.zeros((nvox, ng, 3)); scale = np.zeros((nvox, ng, 3)); quat = np.zeros((nvox, ng, 4))
    lib().gpo_init_batch(_p(mean), _p(var), _p(axis), _p(centres), _p(sf2), nvox, float(size),
                         int(G), int(n_s), int(n_r), int(init_mode), _p(pos), _p(scale), _p(quat))
    return {"pos": pos, "scale": scale, "quat": quat}


class VoxelStore:
    """ALG.STORE of Alg. 2: every point is pushed into the bucket of its voxel, and the
    voxels visited by a frame form S_updated (each voxel listed once).

    Buckets keep at most ``max_points`` points: a full bucket drops its oldest points,
    oldest meaning smallest (scan_id, index-in-scan).  Points are held in that order.
    """

    # voxel types of Sec. 3.3
    BELOW, READY, ACTIVE, CONVERGED = 0, 1, 2, 3

    def __init__(self, size: float, max_points: int, sensor_var: float = 0.0):
        self.size = np.float32(size)
        self.max_points = int(max_points)
        self.sensor_var = float(np.float32(sensor_var))
        self.buckets: dict[tuple, list] = {}
        self.noise: dict[tuple, list] = {}   # noise variance of every stored point
        self.total: dict[tuple, int] = {}
        self.state: dict[tuple, int] = {}

    def insert_scan(self, xyz: np.ndarray) -> list:
        xyz = np.ascontiguousarray(xyz, dtype=np.float32).reshape(-1, 3)
        keys = voxel_keys(xyz, self.size)
        touched = []
        seen = set()
        for i in range(xyz.shape[0]):  # Alg. 2, one point at a time
            k = (int(keys[i, 0]), int(keys[i, 1]), int(keys[i, 2]))
            b = self.buckets.setdefault(k, [])
            nz = self.noise.setdefault(k, [])
            b.append(xyz[i].copy())
            nz.append(self.sensor_var)
            if len(b) > self.max_points:
                b.pop(0)
                nz.pop(0)
            self.total[k] = self.total.get(k, 0) + 1
            if k not in seen:
                seen.add(k)
                touched.append(k)
        return touched

    def voxel_type(self, key, tau: int) -> int:
        """Type of a stored voxel (Sec. 3.3): (d) converged and (c) active come from its
        solves; otherwise (b) once it holds tau points, else (a)."""
        st = self.state.get(key, self.BELOW)
        if st in (self.ACTIVE, self.CONVERGED):
            return st
        return self.READY if len(self.buckets.get(key, ())) >= tau else self.BELOW

    def process_scan(self, xyz, G: int, lam: float, sf2: float, tau: int, eta: float,
                     noise_floor: float, mean_mode: int = 1, axis_of=None, decide=None):
        """One scan through the map update of Sec. 3.3.

        The scan is stored (Alg. 2); each visited voxel is classified as (a)-(d) before
        any solve.  Types (b) and (c) are solved with the noise variance every stored
        point carries (the sensor's for new points, the last posterior variance at the
        point for old ones); the stored points then take the new posterior variance at
        them (at least noise_floor; kept as FP32 like the store), and the voxel becomes
        (d) when the mean predicted variance over its G x G nodes is at most
        eta * sf2, else (c).  Types (a) and (d) are not processed.

        axis_of(key, pts) may return a value axis to impose (for axis-ambiguous voxels)
        or -1; decide(key, mean_var, threshold) may return the converged flag where the
        comparison is within rounding of the threshold, or None.
        Returns one dict per visited voxel, in S_updated order."""
        touched = self.insert_scan(xyz)
        types = [self.voxel_type(k, tau) for k in touched]
        thr = float(np.float32(np.float32(eta) * np.float32(sf2)))
        out = []
        for k, ty in zip(touched, types):
            pts = self.points(k)
            r = {"key": k, "type_before": ty, "n": pts.shape[0]}
            if ty in (self.READY, self.ACTIVE):
                ax = axis_of(k, pts) if axis_of else -1
                nz = np.array(self.noise[k], dtype=np.float64)
                st, axis, mean, var, pvar = solve_voxel_hetero(
                    pts, self.centre(k), float(self.size), G, lam, sf2, nz, mean_mode, ax)
                r.update(status=st, axis=axis, mean=mean, var=var, pvar=pvar, noise=nz)
                if st == 0:
                    fl = np.float32(noise_floor)
                    self.noise[k] = [float(max(np.float32(v), fl)) for v in pvar]
                    mv = float(np.mean(var))
                    conv = decide(k, mv, thr) if decide else None
                    if conv is None:
                        conv = mv <= thr
                    self.state[k] = self.CONVERGED if conv else self.ACTIVE
                    r["mean_var"] = mv
                r["type_after"] = self.state.get(k, ty) if st == 0 else ty
            else:
                r.update(status=CONVERGED if ty == self.CONVERGED else 1, type_after=ty)
            out.append(r)
        return out

    def points(self, key) -> np.ndarray:
        return np.array(self.buckets[key], dtype=np.float32).reshape(-1, 3)

    def centre(self, key) -> np.ndarray:
        return voxel_centres(np.array([key], dtype=np.int32), self.size)[0]
