"""Run one batched solve on a prefix of a synthetic workload, for profilers (ncu).

    python -m paper_2410_17084_b300.profile_solve --nvox 10000 --precision 1

prints the CUDA-event time of each repetition.  Workloads: quadric (the bench workload),
mixed (escalation workload), stress (1M-voxel workload), plane.
"""
from __future__ import annotations

import argparse

import torch

from . import build, gp_voxels as gv, synth


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--nvox", type=int, default=10000)
    ap.add_argument("--precision", type=int, default=gv.PREC_MIXED)
    ap.add_argument("--reps", type=int, default=1)
    ap.add_argument("--init", type=int, default=1)
    ap.add_argument("--workload", default="quadric",
                    choices=["quadric", "mixed", "stress", "plane", "serving"])
    ap.add_argument("--scans", type=int, default=12)
    a = ap.parse_args()
    build.build()
    if a.workload == "serving":  # scans one after another through the serving path
        from . import serve
        scene = synth.lidar_scene()
        scans = [synth.lidar_scan(scene, k) for k in range(a.scans)]
        srv = serve.Server(serve.serving_config())
        lat, wall, _ = srv.run(scans, realtime=False, max_inflight=1)
        srv.close()
        print("per-scan ms", [round(x * 1e3, 1) for x in lat.tolist()])
        return
    gen = {"quadric": synth.quadric_batch, "mixed": synth.mixed_batch,
           "stress": synth.stress_batch, "plane": synth.plane_batch}[a.workload]
    b = gen(a.nvox)
    d = gv.batch_to_device(b)
    g = gv.GpVoxels(gv.gp_voxels_config_default(
        voxel_size=b.size, grid_side=b.G, n_s=b.n_s, n_r=b.n_r, tau=b.tau,
        max_points=int(max(256, b.counts.max())), max_voxels=b.nvox, precision=a.precision))
    out = g.outputs(b.nvox, "cuda", init=bool(a.init))
    for r in range(a.reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        g.solve_csr(d["xyz"], d["offsets"], d["centres"], d["lam"], d["sf2"], d["sn2"], out=out,
                    init=bool(a.init))
        e1.record()
        torch.cuda.synchronize()
        print(f"rep {r} ms {e0.elapsed_time(e1):.3f}")
    g.close()


if __name__ == "__main__":
    main()
