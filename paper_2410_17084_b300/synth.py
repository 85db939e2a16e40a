"""Seeded synthetic inputs shaped like the workloads of GS-LIVM's Voxel-GPR.

The paper evaluates on recorded outdoor LiDAR datasets, which are not available here;
these generators stand in for them.  This module holds no arithmetic of the method
(no kernel, no regression, no hashing): it only draws points, per-voxel
hyperparameters and LiDAR scans from fixed seeds, so the GPU path and the CPU oracle
can be fed the very same arrays.

Batch workloads are CSR batches of voxels:
  xyz      float32 [N, 3]   world points, voxel by voxel
  offsets  int64   [V + 1]  points of voxel v are xyz[offsets[v]:offsets[v+1]]
  centres  float32 [V, 3]   voxel centres, ((key + 0.5) * size) in FP32
  lam, sf2, sn2 float32 [V] kernel inverse-length, signal and noise variance
"""
from __future__ import annotations

import dataclasses

import numpy as np


@dataclasses.dataclass
class VoxelBatch:
    name: str
    xyz: np.ndarray
    offsets: np.ndarray
    centres: np.ndarray
    lam: np.ndarray
    sf2: np.ndarray
    sn2: np.ndarray
    size: float
    G: int
    n_s: int
    n_r: int
    tau: int
    counts: np.ndarray
    degenerate: np.ndarray

    @property
    def nvox(self) -> int:
        return int(self.offsets.shape[0] - 1)

    def subset(self, idx: np.ndarray) -> "VoxelBatch":
        """The voxels ``idx`` (in that order) as a new CSR batch."""
        idx = np.asarray(idx, dtype=np.int64)
        cnt = self.counts[idx]
        off = np.zeros(idx.shape[0] + 1, dtype=np.int64)
        np.cumsum(cnt, out=off[1:])
        xyz = np.concatenate([self.xyz[self.offsets[v]:self.offsets[v + 1]] for v in idx]
                             or [np.zeros((0, 3), np.float32)]).astype(np.float32)
        return VoxelBatch(self.name + "[sub]", np.ascontiguousarray(xyz), off,
                          self.centres[idx].copy(), self.lam[idx].copy(), self.sf2[idx].copy(),
                          self.sn2[idx].copy(), self.size, self.G, self.n_s, self.n_r, self.tau,
                          cnt.copy(), self.degenerate[idx].copy())


def _lattice_keys(nvox: int) -> np.ndarray:
    """Disjoint voxel cells, one voxel per cell of a 3D lattice around the origin."""
    v = np.arange(nvox, dtype=np.int64)
    side = 128
    kx = v % side - side // 2
    ky = (v // side) % side - side // 2
    kz = v // (side * side) - 8
    return np.stack([kx, ky, kz], axis=1).astype(np.int32)


def _powerlaw_counts(rng, nvox: int, lo: int, hi: int) -> np.ndarray:
    """Counts with density proportional to n^-1.5 on [lo, hi], floored (inverse CDF)."""
    u = rng.random(nvox)
    a, b = lo ** -0.5, hi ** -0.5
    n = (a - u * (a - b)) ** -2.0
    return np.clip(np.floor(n), lo, hi).astype(np.int64)


def _assemble(name, rng, counts, size, G, n_s, n_r, tau, surface, degenerate=None,
              axes="z", ell=None, sd=None):
    nvox = counts.shape[0]
    keys = _lattice_keys(nvox)
    centres = ((keys.astype(np.float32) + np.float32(0.5)) * np.float32(size)).astype(np.float32)
    if degenerate is None:
        degenerate = np.zeros(nvox, dtype=bool)
    offsets = np.zeros(nvox + 1, dtype=np.int64)
    np.cumsum(counts, out=offsets[1:])
    N = int(offsets[-1])
    # local coordinates: parameter plane uniform over the voxel face
    xy = rng.uniform(-size / 2, size / 2, size=(N, 2))
    vox = np.repeat(np.arange(nvox), counts)
    f = surface(rng, vox, xy, nvox)
    noise_sd = sd[vox]
    f = f + noise_sd * rng.standard_normal(N)
    # near-degenerate voxels: points on a line (t, kappa t) with tiny jitter
    if degenerate.any():
        dv = degenerate[vox]
        kap = rng.uniform(-1.0, 1.0, size=nvox)[vox]
        t = xy[:, 0]
        jit = 1e-5 * size * rng.standard_normal(N)
        xy[dv, 1] = np.clip(kap[dv] * t[dv], -size / 2, size / 2) + jit[dv]
    local = np.stack([xy[:, 0], xy[:, 1], f], axis=1)
    if axes == "random":
        # value axis drawn per voxel: Z (ground-like), X or Y (wall-like); the local
        # (a, b, value) triple is laid out along the cyclic parameter order
        val = rng.integers(0, 3, size=nvox)[vox]
        out = np.empty_like(local)
        for a in range(3):
            m = val == a
            p1, p2 = (a + 1) % 3, (a + 2) % 3
            out[m, a] = local[m, 2]
            out[m, p1] = local[m, 0]
            out[m, p2] = local[m, 1]
        local = out
    xyz = (centres[vox].astype(np.float64) + local).astype(np.float32)
    lam = (1.0 / (2.0 * ell.astype(np.float64) ** 2)).astype(np.float32)
    sn2 = (sd.astype(np.float64) ** 2).astype(np.float32)
    sf2 = np.ones(nvox, dtype=np.float32)
    return VoxelBatch(name, np.ascontiguousarray(xyz), offsets, centres, lam, sf2, sn2,
                      float(size), G, n_s, n_r, tau, counts, degenerate)


def _plane(rng, vox, xy, nvox):
    a = rng.uniform(-0.5, 0.5, nvox)
    b = rng.uniform(-0.5, 0.5, nvox)
    c = rng.uniform(-0.1, 0.1, nvox)
    return a[vox] * xy[:, 0] + b[vox] * xy[:, 1] + c[vox]


def _quadric(rng, vox, xy, nvox):
    a, b, c = (rng.uniform(-2, 2, nvox) for _ in range(3))
    d, e = (rng.uniform(-0.5, 0.5, nvox) for _ in range(2))
    g = rng.uniform(-0.1, 0.1, nvox)
    x, y = xy[:, 0], xy[:, 1]
    return (a[vox] * x * x + b[vox] * x * y + c[vox] * y * y + d[vox] * x + e[vox] * y
            + g[vox])


def plane_batch(nvox: int = 1000, seed: int = 0) -> VoxelBatch:
    """Planes z = a x + b y + c + 0.02 N(0,1), n ~ U{8..64}, 0.5 m voxels, lengthscale
    0.2 (lambda 12.5), sf 1, sn 0.02, 10 x 10 query grid."""
    rng = np.random.default_rng(seed)
    counts = rng.integers(8, 65, size=nvox).astype(np.int64)
    ell = np.full(nvox, 0.2)
    sd = np.full(nvox, 0.02)
    return _assemble("plane1k", rng, counts, 0.5, 10, 2, 5, 8, _plane, ell=ell, sd=sd)


def quadric_batch(nvox: int = 50000, seed: int = 1, axes: str = "random") -> VoxelBatch:
    """Quadric surfaces (curvature U[-2,2]), lognormal counts (median 64, sigma 0.5)
    clipped to [16, 256], noise sd U[0.01, 0.05], lengthscale U[0.1, 0.4], 16 x 16 grid."""
    rng = np.random.default_rng(seed)
    counts = np.clip(np.round(np.exp(rng.normal(np.log(64.0), 0.5, nvox))), 16, 256)
    counts = counts.astype(np.int64)
    ell = rng.uniform(0.1, 0.4, nvox)
    sd = rng.uniform(0.01, 0.05, nvox)
    return _assemble("quadric50k", rng, counts, 0.5, 16, 4, 4, 16, _quadric, axes=axes,
                     ell=ell, sd=sd)


def mixed_batch(nvox: int = 200000, seed: int = 2, axes: str = "random") -> VoxelBatch:
    """Power-law counts on [32, 512], quadric surfaces, 10% near-degenerate voxels
    (collinear inputs, sn = 1e-4) whose Gram is conditioned beyond 1e8, 32 x 32 grid."""
    rng = np.random.default_rng(seed)
    counts = _powerlaw_counts(rng, nvox, 32, 512)
    ell = rng.uniform(0.1, 0.4, nvox)
    sd = rng.uniform(0.01, 0.05, nvox)
    deg = rng.random(nvox) < 0.10
    sd[deg] = 1e-4
    return _assemble("mixed200k", rng, counts, 0.5, 32, 8, 4, 32, _quadric, degenerate=deg,
                     axes=axes, ell=ell, sd=sd)


def stress_batch(nvox: int = 1000000, seed: int = 4, axes: str = "random") -> VoxelBatch:
    """Power-law counts on [4, 1024], quadric surfaces, 9 x 9 grid (n_s = n_r = 3)."""
    rng = np.random.default_rng(seed)
    counts = _powerlaw_counts(rng, nvox, 4, 1024)
    ell = rng.uniform(0.1, 0.4, nvox)
    sd = rng.uniform(0.01, 0.05, nvox)
    return _assemble("stress1m", rng, counts, 0.5, 9, 3, 3, 4, _quadric, axes=axes,
                     ell=ell, sd=sd)


def fixed_batch(nvox: int, n: int, G: int = 9, seed: int = 5) -> VoxelBatch:
    """nvox voxels of exactly n points each, otherwise as the stress workload (quadric
    surfaces, lengthscale U[0.1, 0.4], noise sd U[0.01, 0.05]); for per-size timing."""
    rng = np.random.default_rng(seed)
    counts = np.full(nvox, n, dtype=np.int64)
    ell = rng.uniform(0.1, 0.4, nvox)
    sd = rng.uniform(0.01, 0.05, nvox)
    ns = 3 if G % 3 == 0 else (4 if G % 4 == 0 else 1)
    return _assemble(f"fixed{n}", rng, counts, 0.5, G, ns, G // ns, 4, _quadric, axes="random",
                     ell=ell, sd=sd)


def point_noise(b: VoxelBatch, seed: int, lo: float = 0.1, hi: float = 10.0) -> np.ndarray:
    """Per-point noise variances for a batch: each point's voxel sn2 times a log-uniform
    factor on [lo, hi] (the spread of fed-back variances around the sensor's)."""
    rng = np.random.default_rng(seed)
    per_pt = np.repeat(b.sn2.astype(np.float64), b.counts)
    f = np.exp(rng.uniform(np.log(lo), np.log(hi), per_pt.shape[0]))
    return (per_pt * f).astype(np.float32)


# ---------------------------------------------------------------------------
# Spinning-LiDAR scans for the serving loop
# ---------------------------------------------------------------------------
@dataclasses.dataclass
class LidarScene:
    box_lo: np.ndarray   # [B, 3]
    box_hi: np.ndarray   # [B, 3]
    path: np.ndarray     # [S, 3] sensor positions
    arrivals: np.ndarray  # [S] arrival time in seconds (Poisson, 10 Hz)
    seed: int


def lidar_scene(nscans: int = 2000, nboxes: int = 200, seed: int = 3) -> LidarScene:
    """A 200 m random-walk sensor path 1.8 m above a ground plane, with ``nboxes``
    axis-aligned boxes (footprint U[1,5] m, height U[1,4] m) within 60 m of the path,
    and Poisson arrivals at 10 Hz."""
    rng = np.random.default_rng(seed)
    heading = np.cumsum(rng.normal(0.0, 0.05, nscans))
    step = 200.0 / max(nscans - 1, 1)
    xy = np.cumsum(np.stack([np.cos(heading), np.sin(heading)], 1) * step, axis=0)
    xy -= xy[0]
    path = np.concatenate([xy, np.full((nscans, 1), 1.8)], axis=1)
    anchor = path[rng.integers(0, nscans, nboxes), :2]
    ang = rng.uniform(0, 2 * np.pi, nboxes)
    rad = rng.uniform(4.0, 60.0, nboxes)
    cxy = anchor + np.stack([np.cos(ang), np.sin(ang)], 1) * rad[:, None]
    fp = rng.uniform(1.0, 5.0, (nboxes, 2))
    h = rng.uniform(1.0, 4.0, nboxes)
    lo = np.concatenate([cxy - fp / 2, np.zeros((nboxes, 1))], 1)
    hi = np.concatenate([cxy + fp / 2, h[:, None]], 1)
    gaps = rng.exponential(0.1, nscans)
    arrivals = np.cumsum(gaps) - gaps[0]
    return LidarScene(lo, hi, path, arrivals, seed)


def lidar_scan(scene: LidarScene, k: int, beams: int = 64, azimuths: int = 1024,
               range_sd: float = 0.02) -> np.ndarray:
    """World-frame points of scan ``k``: 64 beams evenly over [-25, +15] degrees of
    elevation x 1024 azimuths, ranges clipped to [1, 80] m, Gaussian range noise.
    Rays hit the ground plane z = 0 or the nearest box (slab test); each box is tested
    only against the azimuth columns its footprint covers as seen from the sensor."""
    rng = np.random.default_rng((scene.seed, k))
    o = scene.path[k]
    el = np.deg2rad(np.linspace(-25.0, 15.0, beams))
    step = 2 * np.pi / azimuths
    az0 = rng.uniform(0, step)
    az = np.arange(azimuths) * step + az0
    ce, se = np.cos(el)[:, None], np.sin(el)[:, None]
    d = np.stack([np.broadcast_to(ce * np.cos(az), (beams, azimuths)),
                  np.broadcast_to(ce * np.sin(az), (beams, azimuths)),
                  np.broadcast_to(se, (beams, azimuths))], -1)  # [beams, az, 3]
    t = np.full((beams, azimuths), np.inf)
    down = d[..., 2] < 0
    t[down] = -o[2] / d[..., 2][down]
    ctr = (scene.box_lo[:, :2] + scene.box_hi[:, :2]) / 2
    near = np.nonzero(np.linalg.norm(ctr - o[:2], axis=1) < 90.0)[0]
    with np.errstate(divide="ignore", invalid="ignore"):
        for b in near:
            lo, hi = scene.box_lo[b], scene.box_hi[b]
            cx = np.array([lo[0], hi[0], hi[0], lo[0]]) - o[0]
            cy = np.array([lo[1], lo[1], hi[1], hi[1]]) - o[1]
            if lo[0] <= o[0] <= hi[0] and lo[1] <= o[1] <= hi[1]:
                cols = np.arange(azimuths)
            else:
                ang = np.arctan2(cy, cx)
                mid = np.arctan2(ctr[b, 1] - o[1], ctr[b, 0] - o[0])
                rel = np.angle(np.exp(1j * (ang - mid)))  # corner angles around the centre
                a_lo, a_hi = mid + rel.min() - step, mid + rel.max() + step
                i0 = int(np.floor((a_lo - az0) / step))
                i1 = int(np.ceil((a_hi - az0) / step))
                cols = np.arange(i0, i1 + 1) % azimuths
            dd = d[:, cols, :]
            inv = 1.0 / dd
            t1 = (lo - o) * inv
            t2 = (hi - o) * inv
            tmin = np.nanmax(np.minimum(t1, t2), axis=-1)
            tmax = np.nanmin(np.maximum(t1, t2), axis=-1)
            hit = (tmax >= np.maximum(tmin, 0.0)) & (tmin > 0)
            tc = t[:, cols]
            t[:, cols] = np.where(hit & (tmin < tc), tmin, tc)
    t = t.reshape(-1)
    d = d.reshape(-1, 3)
    ok = (t >= 1.0) & (t <= 80.0)
    r = t[ok] + range_sd * rng.standard_normal(int(ok.sum()))
    pts = o + d[ok] * r[:, None]
    return np.ascontiguousarray(pts.astype(np.float32))
