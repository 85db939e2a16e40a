"""Thin ctypes binding of ``include/gp_voxels.h`` (libgp_voxels.so, sm_103a).

Argument marshalling only: every step of the Voxel-GPR path runs in the CUDA
library.  PyTorch supplies device memory (``tensor.data_ptr()``) and streams
(``torch.cuda.current_stream().cuda_stream``).  If the library is missing, importing
the functions raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgp_voxels.so")

GPV_OK, GPV_EINVAL, GPV_ENOMEM, GPV_EBUDGET, GPV_ECUDA, GPV_ETIMEOUT, GPV_EFULL = 0, -1, -2, -3, -4, -5, -6
VOX_OK, VOX_BELOW_TAU, VOX_ESCALATED, VOX_NOT_SPD, VOX_TRUNCATED, VOX_TOO_LARGE = 0, 1, 2, 4, 8, 16
VOX_CONVERGED, VOX_FAILED = 32, 64
TYPE_A, TYPE_B, TYPE_C, TYPE_D = 0, 1, 2, 3  # voxel types of Sec. 3.3
PREC_FP32, PREC_MIXED, PREC_FP64 = 0, 1, 2
SOLVE_ONE_PER_LAUNCH = 1

EXPORTED = [
    "gp_voxels_config_default", "gp_voxels_create", "gp_voxels_destroy", "gp_voxels_solve_csr",
    "gp_voxels_init_gaussians", "gp_voxels_query_sizes", "gp_voxels_strerror",
    "gp_voxels_last_error", "gp_voxels_insert_scan", "gp_voxels_solve", "gp_voxels_scan_info",
    "gp_voxels_release_scan", "gp_voxels_store_voxels", "gp_voxels_solve_csr_noalloc",
    "gp_voxels_last_launches", "gp_voxels_autotune", "gp_voxels_solve_csr_noise",
    "gp_voxels_scan_types", "gp_voxels_type_counts", "gp_voxels_solve_alg3",
    "gp_voxels_structure_loss", "gp_voxels_render", "gp_voxels_measure_peak",
    "gp_voxels_selftest_bounded_wait", "gp_voxels_plan_info", "gp_voxels_bucket_info",
    "gp_voxels_set_timing",
    "gp_voxels_last_tall_ms",
]
NOALLOC_MAX_VOXELS = 65536


class gp_voxels_config(ctypes.Structure):
    _fields_ = [
        ("voxel_size", ctypes.c_float),
        ("grid_side", ctypes.c_int),
        ("n_s", ctypes.c_int),
        ("n_r", ctypes.c_int),
        ("tau", ctypes.c_int),
        ("max_points", ctypes.c_int),
        ("max_voxels", ctypes.c_int),
        ("mean_mode", ctypes.c_int),
        ("precision", ctypes.c_int),
        ("init_mode", ctypes.c_int),
        ("esc_cond", ctypes.c_float),
        ("hash_capacity", ctypes.c_uint32),
        ("mem_budget", ctypes.c_size_t),
        ("scan_slots", ctypes.c_int),
        ("max_scan_points", ctypes.c_int),
        ("max_scan_voxels", ctypes.c_int),
        ("snap_points", ctypes.c_int64),
        ("lambda_", ctypes.c_float),
        ("sf2", ctypes.c_float),
        ("sn2", ctypes.c_float),
        ("eta", ctypes.c_float),
        ("noise_floor", ctypes.c_float),
        ("factor_panel", ctypes.c_int),
        ("tc_workspace_mb", ctypes.c_int),
        ("refine", ctypes.c_int),
        ("tall_min_points", ctypes.c_int),
    ]


class gp_raster_camera(ctypes.Structure):
    _fields_ = [
        ("R", ctypes.c_float * 9),
        ("t", ctypes.c_float * 3),
        ("fx", ctypes.c_float), ("fy", ctypes.c_float), ("cx", ctypes.c_float), ("cy", ctypes.c_float),
        ("width", ctypes.c_int), ("height", ctypes.c_int),
        ("near", ctypes.c_float),
    ]


def make_camera(R, t, fx, fy, cx, cy, width, height, near=0.2) -> gp_raster_camera:
    c = gp_raster_camera()
    c.R[:] = [float(x) for x in np.asarray(R, dtype=np.float32).reshape(9)]
    c.t[:] = [float(x) for x in np.asarray(t, dtype=np.float32).reshape(3)]
    c.fx, c.fy, c.cx, c.cy = float(fx), float(fy), float(cx), float(cy)
    c.width, c.height, c.near = int(width), int(height), float(near)
    return c


class GpvError(RuntimeError):
    def __init__(self, fn, code):
        self.code = code
        super().__init__(f"{fn} failed: {strerror(code)} ({code}) {last_error()}")


_lib = None


def lib() -> ctypes.CDLL:
    """Load libgp_voxels.so; raises if it was not built (no fallback path exists)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "`python -m paper_2410_17084_b300.build` (needs nvcc)")
        L = ctypes.CDLL(LIB_PATH)
        P, I, U32 = ctypes.c_void_p, ctypes.c_int, ctypes.c_uint32
        L.gp_voxels_config_default.argtypes = [ctypes.POINTER(gp_voxels_config)]
        L.gp_voxels_create.argtypes = [ctypes.POINTER(gp_voxels_config), ctypes.POINTER(P)]
        L.gp_voxels_destroy.argtypes = [P]
        L.gp_voxels_solve_csr.argtypes = [P, P, P, ctypes.c_int32, P, P, P, P, P, P, P, P, P, P,
                                          P, U32, P]
        L.gp_voxels_init_gaussians.argtypes = [P, ctypes.c_int32, P, P, P, P, P, P, P, P, P, P]
        L.gp_voxels_query_sizes.argtypes = [ctypes.POINTER(gp_voxels_config),
                                            ctypes.POINTER(ctypes.c_size_t)]
        L.gp_voxels_strerror.argtypes = [I]
        L.gp_voxels_strerror.restype = ctypes.c_char_p
        L.gp_voxels_insert_scan.argtypes = [P, P, ctypes.c_int64, ctypes.c_uint64, P,
                                             ctypes.POINTER(ctypes.c_int32)]
        L.gp_voxels_solve.argtypes = [P, ctypes.c_int32, P, P, P, P, P, P, P, P, P, P]
        L.gp_voxels_scan_info.argtypes = [P, ctypes.c_int32, P, ctypes.POINTER(ctypes.c_int32),
                                          ctypes.POINTER(ctypes.c_int64),
                                          ctypes.POINTER(ctypes.c_uint32)]
        L.gp_voxels_release_scan.argtypes = [P, ctypes.c_int32, P]
        L.gp_voxels_store_voxels.argtypes = [P, ctypes.POINTER(ctypes.c_int64)]
        L.gp_voxels_solve_csr_noalloc.argtypes = [ctypes.POINTER(gp_voxels_config), P, P,
                                                  ctypes.c_int32, P, P, P, P, P, P, P, P, P,
                                                  P, P, P]
        L.gp_voxels_last_launches.argtypes = [P, ctypes.POINTER(ctypes.c_int32)]
        L.gp_voxels_plan_info.argtypes = [P, ctypes.POINTER(ctypes.c_int32)]
        L.gp_voxels_bucket_info.argtypes = [P, ctypes.POINTER(ctypes.c_int32), ctypes.c_int32,
                                            ctypes.POINTER(ctypes.c_int32)]
        L.gp_voxels_set_timing.argtypes = [P, ctypes.c_int32]
        L.gp_voxels_last_tall_ms.argtypes = [P, ctypes.POINTER(ctypes.c_float)]
        L.gp_voxels_autotune.argtypes = [P, P, P, ctypes.c_int32, P, P, P, P, P, P, P, P, P, P,
                                         P, P, ctypes.POINTER(ctypes.c_int32)]
        # h, xyz, offsets, nvox, centres, lam, sf2, sn2, noise, axis, mean, var, status,
        # pos, scale, quat, pvar, flags, stream
        L.gp_voxels_solve_csr_noise.argtypes = [P, P, P, ctypes.c_int32] + [P] * 13 + [U32, P]
        L.gp_voxels_scan_types.argtypes = [P, ctypes.c_int32, P, P, P]
        L.gp_voxels_type_counts.argtypes = [P, ctypes.POINTER(ctypes.c_int64)]
        L.gp_voxels_solve_alg3.argtypes = [P, P, P, ctypes.c_int32] + [P] * 9 + [
            ctypes.POINTER(ctypes.c_int32)]
        L.gp_voxels_structure_loss.argtypes = [P, P, P, ctypes.c_int32, P, ctypes.c_int32,
                                               ctypes.c_float, P, P, P, P, P]
        L.gp_voxels_measure_peak.argtypes = [I, P, ctypes.POINTER(ctypes.c_double)]
        L.gp_voxels_selftest_bounded_wait.argtypes = [U32, P, ctypes.POINTER(ctypes.c_int32)]
        L.gp_voxels_render.argtypes = [P, P, P, P, P, P, ctypes.c_int32,
                                       ctypes.POINTER(gp_raster_camera), P, P, P, P,
                                       ctypes.POINTER(ctypes.c_int64)]
        L.gp_voxels_last_error.argtypes = []
        L.gp_voxels_last_error.restype = ctypes.c_char_p
        for name in EXPORTED:
            if name not in ("gp_voxels_strerror", "gp_voxels_last_error"):
                getattr(L, name).restype = I
        _lib = L
    return _lib


def strerror(code: int) -> str:
    return lib().gp_voxels_strerror(int(code)).decode()


def last_error() -> str:
    return lib().gp_voxels_last_error().decode()


def _check(fn, rc):
    if rc != GPV_OK:
        raise GpvError(fn, rc)


def _ptr(t):
    if t is None:
        return None
    assert t.is_cuda and t.is_contiguous(), "device tensors must be contiguous CUDA tensors"
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


# ---- same names as the C ABI -----------------------------------------------------
def gp_voxels_config_default(**overrides) -> gp_voxels_config:
    cfg = gp_voxels_config()
    _check("gp_voxels_config_default", lib().gp_voxels_config_default(ctypes.byref(cfg)))
    for k, v in overrides.items():
        setattr(cfg, k, v)
    return cfg


def gp_voxels_create(cfg: gp_voxels_config) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    _check("gp_voxels_create", lib().gp_voxels_create(ctypes.byref(cfg), ctypes.byref(h)))
    return h


def gp_voxels_destroy(h) -> None:
    _check("gp_voxels_destroy", lib().gp_voxels_destroy(h))


def gp_voxels_query_sizes(cfg: gp_voxels_config) -> int:
    n = ctypes.c_size_t()
    _check("gp_voxels_query_sizes", lib().gp_voxels_query_sizes(ctypes.byref(cfg), ctypes.byref(n)))
    return n.value


def gp_voxels_solve_csr(h, xyz, offsets, nvox, centres, lam, sf2, sn2, axis, mean, var, status,
                        pos=None, scale=None, quat=None, flags=0, stream=None) -> None:
    rc = lib().gp_voxels_solve_csr(h, _ptr(xyz), _ptr(offsets), int(nvox), _ptr(centres),
                                   _ptr(lam), _ptr(sf2), _ptr(sn2), _ptr(axis), _ptr(mean),
                                   _ptr(var), _ptr(status), _ptr(pos), _ptr(scale), _ptr(quat),
                                   int(flags), _stream(stream))
    _check("gp_voxels_solve_csr", rc)


def gp_voxels_solve_csr_noise(h, xyz, offsets, nvox, centres, lam, sf2, sn2, noise, axis, mean,
                              var, status, pos=None, scale=None, quat=None, pvar=None, flags=0,
                              stream=None) -> None:
    """Voxel-GPR with a noise variance per point (None: sn2 of its voxel) and, optionally,
    the posterior variance at every input point (Sec. 3.3 variance feedback)."""
    rc = lib().gp_voxels_solve_csr_noise(h, _ptr(xyz), _ptr(offsets), int(nvox), _ptr(centres),
                                         _ptr(lam), _ptr(sf2), _ptr(sn2), _ptr(noise),
                                         _ptr(axis), _ptr(mean), _ptr(var), _ptr(status),
                                         _ptr(pos), _ptr(scale), _ptr(quat), _ptr(pvar),
                                         int(flags), _stream(stream))
    _check("gp_voxels_solve_csr_noise", rc)


def gp_voxels_solve_alg3(h, xyz, offsets, nvox, centres, lam, sf2, sn2, axis, mean, cov, status,
                         stream=None) -> int:
    """The paper's Alg. 3 formulation in FP32 with the full posterior covariance
    cov [nvox, G*G, G*G]; returns the largest voxel size it solves."""
    nmax = ctypes.c_int32()
    rc = lib().gp_voxels_solve_alg3(h, _ptr(xyz), _ptr(offsets), int(nvox), _ptr(centres),
                                    _ptr(lam), _ptr(sf2), _ptr(sn2), _ptr(axis), _ptr(mean),
                                    _ptr(cov), _ptr(status), _stream(stream), ctypes.byref(nmax))
    _check("gp_voxels_solve_alg3", rc)
    return nmax.value


def gp_voxels_structure_loss(h, gpos, gscale, m, points, n, cell, loss, best=None, arg=None,
                             info=None, stream=None) -> None:
    """Structure similarity loss of Eq. 11 into the device FP64 scalar ``loss``; per-point
    minima and arguments into ``best`` / ``arg`` when given."""
    rc = lib().gp_voxels_structure_loss(h, _ptr(gpos), _ptr(gscale), int(m), _ptr(points),
                                        int(n), float(cell), _ptr(best), _ptr(arg), _ptr(loss),
                                        _ptr(info), _stream(stream))
    _check("gp_voxels_structure_loss", rc)


def gp_voxels_render(h, pos, scale, quat, opacity, color, m, cam, image, depth, silhouette,
                     stream=None) -> int:
    """Colour, depth and silhouette images of m Gaussians (Eq. 9); returns the number of
    (tile, Gaussian) pairs."""
    pairs = ctypes.c_int64()
    rc = lib().gp_voxels_render(h, _ptr(pos), _ptr(scale), _ptr(quat), _ptr(opacity),
                                _ptr(color), int(m), ctypes.byref(cam), _ptr(image), _ptr(depth),
                                _ptr(silhouette), _stream(stream), ctypes.byref(pairs))
    _check("gp_voxels_render", rc)
    return pairs.value


def gp_voxels_measure_peak(kind: int, stream=None) -> float:
    """Measured TFLOP/s: kind 0 FP32 FMA, kind 1 float-float accumulate-form FMA."""
    t = ctypes.c_double()
    _check("gp_voxels_measure_peak", lib().gp_voxels_measure_peak(int(kind), _stream(stream),
                                                                  ctypes.byref(t)))
    return t.value


def gp_voxels_selftest_bounded_wait(polls: int, stream=None) -> bool:
    """True when a bounded mbarrier wait that nothing completes gave up after ``polls``."""
    t = ctypes.c_int32(-1)
    _check("gp_voxels_selftest_bounded_wait",
           lib().gp_voxels_selftest_bounded_wait(int(polls), _stream(stream), ctypes.byref(t)))
    return t.value == 1


def gp_voxels_scan_types(h, slot, before=None, after=None, stream=None) -> None:
    """Voxel types (TYPE_A..TYPE_D) of a solved slot's rows before and after its solve."""
    rc = lib().gp_voxels_scan_types(h, int(slot), _ptr(before), _ptr(after), _stream(stream))
    _check("gp_voxels_scan_types", rc)


def gp_voxels_type_counts(h) -> list[int]:
    """Stored voxels of each type (a)-(d); synchronises the device."""
    c = (ctypes.c_int64 * 4)()
    _check("gp_voxels_type_counts", lib().gp_voxels_type_counts(h, c))
    return [int(x) for x in c]


def gp_voxels_solve_csr_noalloc(cfg, xyz, offsets, nvox, centres, lam, sf2, sn2, axis, mean,
                                var, status, pos=None, scale=None, quat=None,
                                stream=None) -> None:
    """The batched solve without a handle and without any device allocation: the
    library's static scratch area holds its work queues (see include/gp_voxels.h)."""
    rc = lib().gp_voxels_solve_csr_noalloc(ctypes.byref(cfg), _ptr(xyz), _ptr(offsets),
                                           int(nvox), _ptr(centres), _ptr(lam), _ptr(sf2),
                                           _ptr(sn2), _ptr(axis), _ptr(mean), _ptr(var),
                                           _ptr(status), _ptr(pos), _ptr(scale), _ptr(quat),
                                           _stream(stream))
    _check("gp_voxels_solve_csr_noalloc", rc)


def gp_voxels_init_gaussians(h, nvox, axis, centres, sf2, mean, var, status, pos, scale, quat,
                             stream=None) -> None:
    rc = lib().gp_voxels_init_gaussians(h, int(nvox), _ptr(axis), _ptr(centres), _ptr(sf2),
                                        _ptr(mean), _ptr(var), _ptr(status), _ptr(pos),
                                        _ptr(scale), _ptr(quat), _stream(stream))
    _check("gp_voxels_init_gaussians", rc)


def gp_voxels_insert_scan(h, xyz, npts, scan_id=0, stream=None) -> int:
    """Queue ALG.STORE of one scan; returns the slot, or raises GpvError (EFULL: no free
    slot)."""
    slot = ctypes.c_int32(-1)
    rc = lib().gp_voxels_insert_scan(h, _ptr(xyz) if npts else None, int(npts), int(scan_id),
                                     _stream(stream), ctypes.byref(slot))
    _check("gp_voxels_insert_scan", rc)
    return slot.value


def gp_voxels_solve(h, slot, axis, mean, var, status, pos=None, scale=None, quat=None,
                    keys=None, centres=None, stream=None) -> None:
    rc = lib().gp_voxels_solve(h, int(slot), _ptr(axis), _ptr(mean), _ptr(var), _ptr(status),
                               _ptr(pos), _ptr(scale), _ptr(quat), _ptr(keys), _ptr(centres),
                               _stream(stream))
    _check("gp_voxels_solve", rc)


def gp_voxels_scan_info(h, slot, stream=None) -> tuple[int, int, int]:
    r, p, f = ctypes.c_int32(), ctypes.c_int64(), ctypes.c_uint32()
    rc = lib().gp_voxels_scan_info(h, int(slot), _stream(stream), ctypes.byref(r), ctypes.byref(p),
                                   ctypes.byref(f))
    _check("gp_voxels_scan_info", rc)
    return r.value, p.value, f.value


def gp_voxels_release_scan(h, slot, stream=None) -> None:
    _check("gp_voxels_release_scan", lib().gp_voxels_release_scan(h, int(slot), _stream(stream)))


def gp_voxels_autotune(h, xyz, offsets, nvox, centres, lam, sf2, sn2, axis, mean, var, status,
                       pos=None, scale=None, quat=None, stream=None) -> int:
    changed = ctypes.c_int32()
    rc = lib().gp_voxels_autotune(h, _ptr(xyz), _ptr(offsets), int(nvox), _ptr(centres),
                                  _ptr(lam), _ptr(sf2), _ptr(sn2), _ptr(axis), _ptr(mean),
                                  _ptr(var), _ptr(status), _ptr(pos), _ptr(scale), _ptr(quat),
                                  _stream(stream), ctypes.byref(changed))
    _check("gp_voxels_autotune", rc)
    return changed.value


def gp_voxels_last_launches(h) -> int:
    n = ctypes.c_int32()
    _check("gp_voxels_last_launches", lib().gp_voxels_last_launches(h, ctypes.byref(n)))
    return n.value


def gp_voxels_plan_info(h) -> dict:
    a = (ctypes.c_int32 * 4)()
    _check("gp_voxels_plan_info", lib().gp_voxels_plan_info(h, a))
    return {"tall_min": a[0], "tc_nmax": a[1], "nmax_smem": a[2], "buckets": a[3]}


def gp_voxels_bucket_info(h) -> list:
    """The launch plan's size buckets: dicts of hi, path, threads, percol, panel."""
    cap = 32
    a = (ctypes.c_int32 * (5 * cap))()
    n = ctypes.c_int32()
    _check("gp_voxels_bucket_info", lib().gp_voxels_bucket_info(h, a, cap, ctypes.byref(n)))
    paths = {0: "shared", 1: "workspace", 2: "tall", 3: "shared+tc"}
    return [{"hi": a[5 * b], "path": paths.get(a[5 * b + 1], a[5 * b + 1]), "threads": a[5 * b + 2],
             "percol": bool(a[5 * b + 3]), "panel": a[5 * b + 4]} for b in range(min(n.value, cap))]


def gp_voxels_set_timing(h, on: bool) -> None:
    _check("gp_voxels_set_timing", lib().gp_voxels_set_timing(h, 1 if on else 0))


def gp_voxels_last_tall_ms(h) -> float:
    ms = ctypes.c_float()
    _check("gp_voxels_last_tall_ms", lib().gp_voxels_last_tall_ms(h, ctypes.byref(ms)))
    return ms.value


def gp_voxels_store_voxels(h) -> int:
    n = ctypes.c_int64()
    _check("gp_voxels_store_voxels", lib().gp_voxels_store_voxels(h, ctypes.byref(n)))
    return n.value


def unpack_keys(keys):
    """Integer voxel indices (kx, ky, kz) of packed keys (21 bits per axis, offset 2^20)."""
    import numpy as np
    k = np.asarray(keys, dtype=np.int64)
    m = (1 << 21) - 1
    return np.stack([(k & m) - (1 << 20), ((k >> 21) & m) - (1 << 20),
                     ((k >> 42) & m) - (1 << 20)], axis=-1).astype(np.int32)


# ---- convenience wrapper ------------------------------------------------------------
class GpVoxels:
    """Owns one library handle; allocates output tensors with torch."""

    def __init__(self, cfg: gp_voxels_config | None = None, **overrides):
        self.cfg = cfg if cfg is not None else gp_voxels_config_default(**overrides)
        if cfg is not None:
            for k, v in overrides.items():
                setattr(self.cfg, k, v)
        self.h = gp_voxels_create(self.cfg)

    def close(self):
        if self.h is not None:
            gp_voxels_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def outputs(self, nvox: int, device="cuda", init: bool = False) -> dict:
        G = self.cfg.grid_side
        ng = self.cfg.n_s * self.cfg.n_s
        out = {
            "axis": torch.empty(nvox, dtype=torch.uint8, device=device),
            "mean": torch.empty(nvox, G * G, dtype=torch.float32, device=device),
            "var": torch.empty(nvox, G * G, dtype=torch.float32, device=device),
            "status": torch.empty(nvox, dtype=torch.int32, device=device),
        }
        if init:
            out["pos"] = torch.empty(nvox * ng, 3, dtype=torch.float32, device=device)
            out["scale"] = torch.empty(nvox * ng, 3, dtype=torch.float32, device=device)
            out["quat"] = torch.empty(nvox * ng, 4, dtype=torch.float32, device=device)
        return out

    def solve_csr(self, xyz, offsets, centres, lam, sf2, sn2, out=None, init=False,
                  one_per_launch=False, stream=None) -> dict:
        nvox = offsets.shape[0] - 1
        if out is None:
            out = self.outputs(nvox, xyz.device, init)
        gp_voxels_solve_csr(self.h, xyz, offsets, nvox, centres, lam, sf2, sn2, out["axis"],
                            out["mean"], out["var"], out["status"], out.get("pos"),
                            out.get("scale"), out.get("quat"),
                            SOLVE_ONE_PER_LAUNCH if one_per_launch else 0, stream)
        return out

    def autotune(self, xyz, offsets, centres, lam, sf2, sn2, init=True, stream=None) -> int:
        """Choose the CTA size of every size bucket by timing this batch."""
        nvox = offsets.shape[0] - 1
        out = self.outputs(nvox, xyz.device, init)
        return gp_voxels_autotune(self.h, xyz, offsets, nvox, centres, lam, sf2, sn2,
                                  out["axis"], out["mean"], out["var"], out["status"],
                                  out.get("pos"), out.get("scale"), out.get("quat"), stream)

    def init_gaussians(self, axis, centres, sf2, mean, var, status=None, stream=None) -> dict:
        nvox = axis.shape[0]
        ng = self.cfg.n_s * self.cfg.n_s
        dev = mean.device
        out = {
            "pos": torch.empty(nvox * ng, 3, dtype=torch.float32, device=dev),
            "scale": torch.empty(nvox * ng, 3, dtype=torch.float32, device=dev),
            "quat": torch.empty(nvox * ng, 4, dtype=torch.float32, device=dev),
        }
        gp_voxels_init_gaussians(self.h, nvox, axis, centres, sf2, mean, var, status, out["pos"],
                                 out["scale"], out["quat"], stream)
        return out


def capture_graph(fn, warmup: int = 1):
    """Capture the GPU work that ``fn()`` queues on the current stream (solve calls
    queue only capturable operations: kernels, memsets, event fork/join) into a CUDA
    graph; returns the graph (``graph.replay()`` re-runs it)."""
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        for _ in range(warmup):
            fn()
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        fn()
    torch.cuda.synchronize()
    return g


def batch_to_device(b, device="cuda") -> dict:
    """Copy a synthetic CSR batch (numpy arrays) to device tensors."""
    return {
        "xyz": torch.from_numpy(b.xyz).to(device),
        "offsets": torch.from_numpy(b.offsets).to(device),
        "centres": torch.from_numpy(b.centres).to(device),
        "lam": torch.from_numpy(b.lam).to(device),
        "sf2": torch.from_numpy(b.sf2).to(device),
        "sn2": torch.from_numpy(b.sn2).to(device),
    }
