"""Serving loop for streamed LiDAR scans over the C ABI (continuous batching).

Scans arrive at given times (Poisson, 10 Hz in the synthetic workload).  A scan is
admitted as soon as it has arrived and one of the handle's scan slots is free; the slots
are the memory reserved under the configured budget, so admission is by memory.  Each
admitted scan runs on its own CUDA stream: host-to-device copy of its points, ALG.STORE
into the resident voxel hash (the library orders inserts by call order), the Voxel-GPR
re-solve of the visited voxels and the fused Gaussian initialisation.  With the voxel
state machine of Sec. 3.3 on (eta > 0) the library orders each insert after the previous
scan's solve, since a voxel's type and its points' noise come from that solve.  Work of scans in
flight overlaps on the device.  The latency of a scan is the time from its arrival to the
completion of its last queued GPU operation.
"""
from __future__ import annotations

import time

import numpy as np
import torch

from . import gp_voxels as gv


class Lane:
    """Per-slot stream and buffers (device inputs and outputs, pinned staging)."""

    def __init__(self, cfg, device):
        V, P = cfg.max_scan_voxels, cfg.max_scan_points
        G, ng = cfg.grid_side, cfg.n_s * cfg.n_s
        self.stream = torch.cuda.Stream(device)
        self.pin = torch.empty(P, 3, dtype=torch.float32).pin_memory()
        self.xyz = torch.empty(P, 3, dtype=torch.float32, device=device)
        self.out = {
            "axis": torch.empty(V, dtype=torch.uint8, device=device),
            "mean": torch.empty(V, G * G, dtype=torch.float32, device=device),
            "var": torch.empty(V, G * G, dtype=torch.float32, device=device),
            "status": torch.empty(V, dtype=torch.int32, device=device),
            "pos": torch.empty(V * ng, 3, dtype=torch.float32, device=device),
            "scale": torch.empty(V * ng, 3, dtype=torch.float32, device=device),
            "quat": torch.empty(V * ng, 4, dtype=torch.float32, device=device),
            "keys": torch.empty(V, dtype=torch.int64, device=device),
            "centres": torch.empty(V, 3, dtype=torch.float32, device=device),
        }
        if cfg.eta > 0:  # voxel types of Sec. 3.3 before and after each solve
            self.out["type_before"] = torch.empty(V, dtype=torch.uint8, device=device)
            self.out["type_after"] = torch.empty(V, dtype=torch.uint8, device=device)
        self.done = torch.cuda.Event()
        self.busy = False
        self.scan = -1
        self.slot = -1


class Server:
    def __init__(self, cfg: gv.gp_voxels_config, device="cuda"):
        assert cfg.hash_capacity > 0, "serving needs the voxel store (hash_capacity > 0)"
        self.cfg = cfg
        self.g = gv.GpVoxels(cfg)
        self.lanes = [Lane(cfg, device) for _ in range(cfg.scan_slots)]

    def close(self):
        torch.cuda.synchronize()
        self.g.close()

    def _submit(self, lane: Lane, k: int, pts: np.ndarray, keep_slot: bool):
        n = pts.shape[0]
        if n > self.cfg.max_scan_points:
            raise ValueError(f"scan {k} has {n} points > max_scan_points")
        lane.pin[:n].copy_(torch.from_numpy(pts))
        with torch.cuda.stream(lane.stream):
            lane.xyz[:n].copy_(lane.pin[:n], non_blocking=True)
            slot = gv.gp_voxels_insert_scan(self.g.h, lane.xyz, n, k, lane.stream)
            o = lane.out
            gv.gp_voxels_solve(self.g.h, slot, o["axis"], o["mean"], o["var"], o["status"],
                               o["pos"], o["scale"], o["quat"], o["keys"], o["centres"],
                               lane.stream)
            if "type_before" in o:
                gv.gp_voxels_scan_types(self.g.h, slot, o["type_before"], o["type_after"],
                                        lane.stream)
            if not keep_slot:
                gv.gp_voxels_release_scan(self.g.h, slot, lane.stream)
            lane.done.record(lane.stream)
        lane.busy, lane.scan, lane.slot = True, k, (slot if keep_slot else -1)

    def _collect(self, lane: Lane) -> dict:
        rows, npts, flags = gv.gp_voxels_scan_info(self.g.h, lane.slot, lane.stream)
        ng = self.cfg.n_s * self.cfg.n_s
        o = lane.out
        res = {k: o[k][:rows].cpu().numpy() for k in ("axis", "mean", "var", "status", "keys",
                                                       "centres", "type_before", "type_after")
               if k in o}
        for k in ("pos", "scale", "quat"):
            res[k] = o[k][:rows * ng].cpu().numpy()
        res.update(rows=rows, points=npts, flags=flags)
        gv.gp_voxels_release_scan(self.g.h, lane.slot, lane.stream)
        lane.slot = -1
        return res

    def run(self, scans, arrivals=None, realtime=True, collect=False, max_inflight=None):
        """Serve ``scans`` (list of float32 [n, 3] arrays) arriving at ``arrivals``
        (seconds from the start; None = all at once).  Returns latencies (s) per scan,
        the wall time, and with ``collect`` the per-scan results on the host."""
        nscan = len(scans)
        arr = np.zeros(nscan) if arrivals is None else np.asarray(arrivals, dtype=np.float64)
        lanes = self.lanes[: max_inflight or len(self.lanes)]
        lat = np.full(nscan, np.nan)
        results = [None] * nscan
        nxt = 0
        finished = 0
        t0 = time.perf_counter()
        while finished < nscan:
            now = time.perf_counter() - t0
            progressed = False
            for ln in lanes:  # completions
                if ln.busy and ln.done.query():
                    lat[ln.scan] = (time.perf_counter() - t0) - arr[ln.scan]
                    if collect:
                        results[ln.scan] = self._collect(ln)
                    ln.busy = False
                    finished += 1
                    progressed = True
            # admissions, in arrival order, while slots are free
            while nxt < nscan and (not realtime or arr[nxt] <= now):
                free = next((ln for ln in lanes if not ln.busy), None)
                if free is None:
                    break
                self._submit(free, nxt, scans[nxt], keep_slot=collect)
                nxt += 1
                progressed = True
            if not progressed:
                time.sleep(2e-4)
        wall = time.perf_counter() - t0
        return lat, wall, results


def serving_config(**overrides) -> gv.gp_voxels_config:
    """The LiDAR serving workload: 0.5 m voxels, 9 x 9 query grid (n_s = n_r = 3),
    tau = 10, 256 points per bucket (voxels beyond the shared-memory kernels take the
    tall-matrix tensor-core path, which every scan slot has a slice store for),
    lengthscale 0.2 m (lambda 12.5), sn 0.02 m, a 4 GB memory budget."""
    d = dict(voxel_size=0.5, grid_side=9, n_s=3, n_r=3, tau=10, max_points=256,
             max_voxels=1 << 16, precision=gv.PREC_MIXED, hash_capacity=1 << 19,
             mem_budget=4 << 30, scan_slots=4, max_scan_points=1 << 17,
             max_scan_voxels=1 << 15, snap_points=1 << 21, lambda_=12.5, sf2=1.0, sn2=4e-4)
    d.update(overrides)
    return gv.gp_voxels_config_default(**d)
