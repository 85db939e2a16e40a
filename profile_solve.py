"""Run one batched solve on a prefix of a synthetic workload, for profilers (ncu).

    python profile_solve.py --nvox 10000 --precision 1
    python profile_solve.py --workload fixed --n 512 --nvox 296

prints the CUDA-event time of each repetition.  Workloads: quadric (the bench workload),
mixed (escalation workload), stress (1M-voxel workload), plane; with --path alg3 the
paper's Alg. 3 formulation (full covariance) on the chosen workload, with --path lp the
structure similarity loss of the workload's points against its initialised Gaussians, with
--path raster one 1920 x 1080 image of those Gaussians.
"""
from __future__ import annotations

import argparse
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))

import torch

from paper_2410_17084_b300 import build, gp_voxels as gv, synth


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--nvox", type=int, default=10000)
    ap.add_argument("--precision", type=int, default=gv.PREC_MIXED)
    ap.add_argument("--reps", type=int, default=1)
    ap.add_argument("--init", type=int, default=1)
    ap.add_argument("--workload", default="quadric",
                    choices=["quadric", "mixed", "stress", "plane", "serving", "fixed"])
    ap.add_argument("--n", type=int, default=512, help="points per voxel of the fixed workload")
    ap.add_argument("--scans", type=int, default=12)
    ap.add_argument("--path", default="solve", choices=["solve", "alg3", "lp", "raster"])
    ap.add_argument("--tc-mb", type=int, default=4096, help="tensor-core variance workspace")
    ap.add_argument("--tall-min", type=int, default=0, help="tall-matrix path above this n")
    a = ap.parse_args()
    build.build()
    if a.workload == "serving":  # scans one after another through the serving path
        from paper_2410_17084_b300 import serve
        scene = synth.lidar_scene()
        scans = [synth.lidar_scan(scene, k) for k in range(a.scans)]
        srv = serve.Server(serve.serving_config())
        lat, wall, _ = srv.run(scans, realtime=False, max_inflight=1)
        srv.close()
        print("per-scan ms", [round(x * 1e3, 1) for x in lat.tolist()])
        return
    if a.workload == "fixed":
        b = synth.fixed_batch(a.nvox, a.n)
    else:
        gen = {"quadric": synth.quadric_batch, "mixed": synth.mixed_batch,
               "stress": synth.stress_batch, "plane": synth.plane_batch}[a.workload]
        b = gen(a.nvox)
    d = gv.batch_to_device(b)
    g = gv.GpVoxels(gv.gp_voxels_config_default(
        voxel_size=b.size, grid_side=b.G, n_s=b.n_s, n_r=b.n_r, tau=b.tau,
        max_points=int(max(256, b.counts.max())), max_voxels=b.nvox, precision=a.precision,
        tc_workspace_mb=a.tc_mb, tall_min_points=a.tall_min))
    out = g.outputs(b.nvox, "cuda", init=bool(a.init) or a.path in ("lp", "raster"))
    if a.path != "solve":
        _other_path(a, b, d, g, out)
        g.close()
        return
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


def _other_path(a, b, d, g, out):
    import numpy as np
    Q = b.G * b.G
    if a.path == "alg3":
        axis = torch.empty(b.nvox, dtype=torch.uint8, device="cuda")
        mean = torch.empty(b.nvox, Q, device="cuda")
        cov = torch.empty(b.nvox, Q, Q, device="cuda")
        st = torch.empty(b.nvox, dtype=torch.int32, device="cuda")
        fn = lambda: gv.gp_voxels_solve_alg3(g.h, d["xyz"], d["offsets"], b.nvox, d["centres"],
                                             d["lam"], d["sf2"], d["sn2"], axis, mean, cov, st)
    else:
        g.solve_csr(d["xyz"], d["offsets"], d["centres"], d["lam"], d["sf2"], d["sn2"], out=out,
                    init=True)
        ok = torch.repeat_interleave((out["status"] & 0x15) == 0, b.n_s * b.n_s)
        gpos, gsc, gq = (out[k][ok].contiguous() for k in ("pos", "scale", "quat"))
        m = int(gpos.shape[0])
        if a.path == "lp":
            loss = torch.empty(1, dtype=torch.float64, device="cuda")
            npts = int(d["xyz"].shape[0])
            fn = lambda: gv.gp_voxels_structure_loss(g.h, gpos, gsc, m, d["xyz"], npts,
                                                     b.size / b.n_s, loss)
        else:
            rng = np.random.default_rng(81)
            gop = torch.from_numpy(rng.uniform(0.2, 1.0, m).astype(np.float32)).cuda()
            gcol = torch.from_numpy(rng.uniform(0.0, 1.0, (m, 3)).astype(np.float32)).cuda()
            W, H = 1920, 1080
            cam = gv.make_camera(np.diag([1.0, -1.0, -1.0]), [0.0, 0.0, 20.0], 700.0, 700.0,
                                 W / 2, H / 2, W, H, 0.2)
            img = torch.empty(H, W, 3, device="cuda")
            dep = torch.empty(H, W, device="cuda")
            sil = torch.empty(H, W, device="cuda")
            fn = lambda: gv.gp_voxels_render(g.h, gpos, gsc, gq, gop, gcol, m, cam, img, dep, sil)
    for r in range(a.reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        torch.cuda.synchronize()
        print(f"{a.path} rep {r} ms {e0.elapsed_time(e1):.3f}")


if __name__ == "__main__":
    main()
