"""Benchmark of the B300 Voxel-GPR path (GS-LIVM Sec. 3.1-3.2).

One step = one batched Voxel-GPR solve + fused Gaussian initialisation over the whole
workload: 50,000 voxels with lognormal point counts (median 64, clipped to 16..256) on
quadric surfaces, per-voxel lengthscale U[0.1, 0.4] and noise sd U[0.01, 0.05], a 16 x 16
query grid (n_s = n_r = 4), mixed precision (float-float with FP64 escalation).

Prints ONE JSON line (rank 0).  ``--impl reference`` times the FP64 CPU oracle on the
same workload instead (bounded sample per step).  Multi-GPU (torchrun): every rank
solves its own independent batch (weak scaling, no data-path collective).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("voxel GP solves/sec + predicted pts/sec (mixed vs plain FP32, same err); "
          "p50/p99 scan ms")
WORKLOAD = ("quadric50k: 50,000 voxels of 0.5 m, lognormal counts (median 64) clipped to "
            "[16,256], quadric surfaces (curvature U[-2,2]) with noise sd U[0.01,0.05] m, SE "
            "kernel lengthscale U[0.1,0.4], 16x16 query grid (n_s=n_r=4), value axis drawn "
            "per voxel; GPR + fused Gaussian init")


def algorithmic_flops(counts: np.ndarray, G: int) -> float:
    """Per voxel n^3/3 (Cholesky) + n^2 G^2 (triangular solve behind diag Sigma*) +
    4 n G^2 (mean and variance norms) + 4 n^2 (alpha solves); the explicit inverse and
    the full Sigma* that the method avoids are not counted."""
    n = counts.astype(np.float64)
    g2 = float(G * G)
    return float(np.sum(n ** 3 / 3.0 + n * n * g2 + 4.0 * n * g2 + 4.0 * n * n))


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during a region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = os.path.join(ROOT, "gpurun_out", f"clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self) -> dict:
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            p = [x.strip() for x in line.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax.append(float(p[2]))
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if p[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


def fp32_alu_peak_tflops(sm_mhz: float) -> float:
    """148 SMs x 128 FP32 lanes x 2 flops per FMA x clock."""
    return 148 * 128 * 2 * sm_mhz * 1e6 / 1e12


# FP32 instructions per float-float multiply-add (TwoProduct with two correction FMAs and
# a fast renormalisation = 7, accurate float-float addition = 20)
FF_OPS_PER_FMA = 27


def run_reference(args, rank, world):
    """The FP64 CPU oracle timed on the host cores on a bounded sample of the workload."""
    from oracle import oracle as O
    from paper_2410_17084_b300 import synth
    if rank != 0:
        return
    b = synth.quadric_batch()
    ncpu = os.cpu_count() or 1
    # size one step to ~2 s of host work
    probe = b.subset(np.arange(400))
    t = time.perf_counter()
    O.solve_batch(probe.xyz, probe.offsets, probe.centres, probe.lam, probe.sf2, probe.sn2,
                  b.size, b.G, b.tau, nthreads=ncpu)
    per = (time.perf_counter() - t) / 400
    k = int(min(b.nvox, max(400, 2.0 / max(per, 1e-9))))
    times = []
    for s in range(args.warmup + args.steps):
        idx = np.arange(s * k, (s + 1) * k) % b.nvox
        sub = b.subset(idx)
        t = time.perf_counter()
        r = O.solve_batch(sub.xyz, sub.offsets, sub.centres, sub.lam, sub.sf2, sub.sn2, b.size,
                          b.G, b.tau, nthreads=ncpu)
        O.init_batch(r["mean"], r["var"], r["axis"], sub.centres, sub.sf2, b.size, b.G, b.n_s,
                     b.n_r)
        if s >= args.warmup:
            times.append(time.perf_counter() - t)
    tt = sum(times)
    value = k * len(times) / tt
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "voxel solves/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * tt / len(times), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample_voxels_per_step": k},
        "cpu_baseline": {"value": value, "unit": "voxel solves/s", "cores": ncpu,
                         "kind": "oracle", "sample": f"{k} voxels of the workload per step"},
        "e2e": {"value": value, "unit": "voxel solves/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def cpu_baseline_leg(b, budget_s=12.0) -> dict:
    from oracle import oracle as O
    ncpu = os.cpu_count() or 1
    probe = b.subset(np.arange(300))
    t = time.perf_counter()
    O.solve_batch(probe.xyz, probe.offsets, probe.centres, probe.lam, probe.sf2, probe.sn2,
                  b.size, b.G, b.tau, nthreads=ncpu)
    per = (time.perf_counter() - t) / 300
    k = int(min(b.nvox, max(300, budget_s / max(per, 1e-9))))
    sub = b.subset(np.arange(k))
    t = time.perf_counter()
    r = O.solve_batch(sub.xyz, sub.offsets, sub.centres, sub.lam, sub.sf2, sub.sn2, b.size, b.G,
                      b.tau, nthreads=ncpu)
    O.init_batch(r["mean"], r["var"], r["axis"], sub.centres, sub.sf2, b.size, b.G, b.n_s, b.n_r)
    dt = time.perf_counter() - t
    return {"value": k / dt, "unit": "voxel solves/s", "cores": ncpu, "kind": "oracle",
            "sample": f"first {k} of {b.nvox} voxels of the workload (GPR + Gaussian init)",
            "seconds": dt}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip FP32 / one-per-launch legs")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import torch
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    from paper_2410_17084_b300 import build, gp_voxels as gv, synth
    if rank == 0:
        build.build()
    if dist is not None:
        dist.barrier()

    b = synth.quadric_batch(seed=1 + 1000 * rank)
    G = b.G
    flops = algorithmic_flops(b.counts, G)
    d = gv.batch_to_device(b)
    cfg = gv.gp_voxels_config_default(voxel_size=b.size, grid_side=G, n_s=b.n_s, n_r=b.n_r,
                                      tau=b.tau, max_points=256, max_voxels=b.nvox,
                                      precision=gv.PREC_MIXED, mean_mode=1)
    g = gv.GpVoxels(cfg)
    out = g.outputs(b.nvox, "cuda", init=True)
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def step(handle=g, o=out, flags=0):
        gv.gp_voxels_solve_csr(handle.h, d["xyz"], d["offsets"], b.nvox, d["centres"], d["lam"],
                               d["sf2"], d["sn2"], o["axis"], o["mean"], o["var"], o["status"],
                               o.get("pos"), o.get("scale"), o.get("quat"), flags, stream)

    def timed(fn, steps, warmup):
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize()
        evs = []
        for _ in range(steps):
            flush.fill_(1.0)  # evict L2 between timed steps (256 MiB > 126 MB L2)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            evs.append((e0, e1))
        torch.cuda.synchronize()
        return [a.elapsed_time(c) for a, c in evs]

    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        ms = timed(step, args.steps, args.warmup)
    t_step = sum(ms) / len(ms)
    if dist is not None:
        tt = torch.tensor([t_step], device="cuda")
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t_step = float(tt.item())
    value = world * b.nvox / (t_step * 1e-3)
    st = out["status"].cpu().numpy()
    n_esc = int(((st & gv.VOX_ESCALATED) != 0).sum())

    # ---- e2e: host buffers in, host buffers out, through the C ABI ------------------
    pin = {k: torch.from_numpy(getattr(b, k)).pin_memory() for k in
           ("xyz", "offsets", "centres", "lam", "sf2", "sn2")}
    host_out = {k: torch.empty(v.shape, dtype=v.dtype).pin_memory() for k, v in out.items()}
    h2d = sum(v.numel() * v.element_size() for v in pin.values())
    d2h = sum(v.numel() * v.element_size() for v in host_out.values())

    def e2e_step():
        for k, v in pin.items():
            d[k].copy_(v, non_blocking=True)
        step()
        for k, v in out.items():
            host_out[k].copy_(v, non_blocking=True)

    e2e_ms = timed(e2e_step, max(3, args.steps // 2), 2)
    t_e2e = sum(e2e_ms) / len(e2e_ms)

    extras = {}
    if not args.no_extras and rank == 0:
        # plain FP32 batched and the plain one-voxel-per-launch FP32 baseline
        cfg32 = gv.gp_voxels_config_default(voxel_size=b.size, grid_side=G, n_s=b.n_s,
                                            n_r=b.n_r, tau=b.tau, max_points=256,
                                            max_voxels=b.nvox, precision=gv.PREC_FP32)
        g32 = gv.GpVoxels(cfg32)
        o32 = g32.outputs(b.nvox, "cuda", init=True)
        m32 = timed(lambda: step(g32, o32), 3, 3)
        t32 = sum(m32) / len(m32)
        extras["fp32_batched"] = {"value": b.nvox / (t32 * 1e-3), "ms_per_step": t32}
        # one voxel per launch: time a 5,000-voxel prefix, scaled per voxel
        nsub = 5000
        bs = b.subset(np.arange(nsub))
        ds = gv.batch_to_device(bs)
        gsub = gv.GpVoxels(gv.gp_voxels_config_default(
            voxel_size=b.size, grid_side=G, n_s=b.n_s, n_r=b.n_r, tau=b.tau, max_points=256,
            max_voxels=nsub, precision=gv.PREC_FP32))
        osub = gsub.outputs(nsub, "cuda", init=True)

        def one_per_launch():
            gv.gp_voxels_solve_csr(gsub.h, ds["xyz"], ds["offsets"], nsub, ds["centres"],
                                   ds["lam"], ds["sf2"], ds["sn2"], osub["axis"], osub["mean"],
                                   osub["var"], osub["status"], osub["pos"], osub["scale"],
                                   osub["quat"], gv.SOLVE_ONE_PER_LAUNCH, stream)
        mpl = timed(one_per_launch, 2, 1)
        tpl = sum(mpl) / len(mpl)
        extras["fp32_one_voxel_per_launch"] = {"value": nsub / (tpl * 1e-3),
                                               "sample_voxels": nsub}
        extras["mixed_vs_one_per_launch"] = value / world / extras["fp32_one_voxel_per_launch"]["value"]
        g32.close()
        gsub.close()

    clocks = clk.summary()
    sm_mhz = clocks.get("sm_mhz") or 2032.0
    peak_fp32 = fp32_alu_peak_tflops(2032.0)
    peak_ff = peak_fp32 * 2.0 / FF_OPS_PER_FMA
    achieved = flops / (t_step * 1e-3) / 1e12
    line = {
        "metric": METRIC,
        "value": value,
        "unit": "voxel solves/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": t_step,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32x2",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "voxels_per_gpu": b.nvox, "grid": f"{G}x{G}",
                   "precision": "mixed (float-float + FP64 escalation)",
                   "l2": "flushed between timed steps (256 MiB write)",
                   "parallelism": f"independent batches per GPU x{world}"},
        "predicted_pts_per_s": value * G * G,
        "escalated_voxels": n_esc,
        "gpu_launches": None,
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak_ff, "unit": "TFLOP/s",
                     "frac": achieved / peak_ff, "traffic": None,
                     "peak_note": "float-float FMA rate = FP32 ALU peak (148 SMs x 128 lanes x "
                                  "2 x 2032 MHz) x 2 / 27 FP32 ops per float-float FMA"},
        "e2e": {"value": world * b.nvox / (t_e2e * 1e-3), "unit": "voxel solves/s",
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "clocks": clocks,
    }
    line.update(extras)
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_leg(b)
    if rank == 0:
        print(json.dumps(line), flush=True)
    g.close()
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
