"""Benchmark of the B300 Voxel-GPR path (GS-LIVM Sec. 3.1-3.2).

One step = one batched Voxel-GPR solve + fused Gaussian initialisation over the largest
workload: 1,000,000 voxels with power-law point counts (density n^-1.5 on [4, 1024]) on
quadric surfaces, per-voxel lengthscale U[0.1, 0.4] and noise sd U[0.01, 0.05], a 9 x 9
query grid (n_s = n_r = 3), mixed precision (float-float and exact BF16 slice products on
the tensor cores, FP64 escalation), replayed as one CUDA graph per step.

Prints ONE JSON line (rank 0).  Every measured leg carries its error against the FP64
oracle on a fixed sample of voxels solved outside the timed region.  ``--impl reference``
times the FP64 CPU oracle on the same workload instead (bounded sample per step).
Multi-GPU (torchrun): every rank solves its own independent batch (weak scaling, no
data-path collective).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("voxel GP solves/sec + predicted pts/sec (mixed vs plain FP32, same err); "
          "p50/p99 scan ms")
WORKLOAD = ("stress1m: 1,000,000 voxels of 0.5 m, point counts power-law (density n^-1.5) on "
            "[4,1024], quadric surfaces (curvature U[-2,2]) with noise sd U[0.01,0.05] m, SE "
            "kernel lengthscale U[0.1,0.4], 9x9 query grid (n_s=n_r=3), value axis drawn per "
            "voxel; GPR + fused Gaussian init (9 Gaussians per voxel); one CUDA-graph replay "
            "per step")
ERR_SAMPLE = 2000          # voxels per workload compared with the oracle
FF_OPS_PER_FMA = 12        # FP32 instructions per float-float multiply-add (accumulate form)
SLICE_PAIRS = 21           # BF16 slice products per float-float product (six slices, s+t <= 5)


# ---- algorithmic work -----------------------------------------------------------------
def algorithmic_flops(counts: np.ndarray, G: int) -> np.ndarray:
    """Per voxel: n^3/3 (Cholesky) + n^2 G^2 (the triangular solve behind diag Sigma*) +
    4 n G^2 (mean and variance norms) + 4 n^2 (alpha solves); the explicit inverse and the
    full Sigma* that the method avoids are not counted."""
    n = counts.astype(np.float64)
    g2 = float(G * G)
    return n ** 3 / 3.0 + n * n * g2 + 4.0 * n * g2 + 4.0 * n * n


def split_flops(counts: np.ndarray, G: int, plan: dict) -> dict:
    """Algorithmic FLOPs by the unit that executes them in the mixed path.
    Tall-matrix voxels (n > tall_min): the panel updates of L and V (all but the work
    inside each 32-column panel) run as exact BF16 slice products on the tensor cores; the
    in-panel work (about 32 flops per row and column: the block solve, the running sums)
    on the CUDA cores in float-float.  Shared-memory voxels: the variance contraction
    n^2 G^2 on the tensor cores where the tensor-core variance takes them
    (n <= tc_nmax), everything else in float-float on the CUDA cores."""
    n = counts.astype(np.float64)
    fl = algorithmic_flops(counts, G)
    Q = float(G * G)
    tmin = plan["tall_min"] if plan["tall_min"] > 0 else 1 << 30
    tall = counts > tmin
    npad = np.ceil(n / 32.0) * 32.0
    in_panel = np.minimum(32.0 * (npad + Q) * npad, fl)
    tc_small = (~tall) & (counts <= plan["tc_nmax"])
    f_tc = np.where(tall, fl - in_panel, np.where(tc_small, n * n * Q, 0.0))
    return {"total": float(fl.sum()), "tc": float(f_tc.sum()), "ff": float((fl - f_tc).sum()),
            "tall_total": float(fl[tall].sum()), "tall_tc": float(f_tc[tall].sum()),
            "tall_ff": float(in_panel[tall].sum()), "tall_voxels": int(tall.sum())}


# ---- clocks -----------------------------------------------------------------------------
class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during a region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"gpv_clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                stderr=subprocess.DEVNULL)
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


def measured_peaks() -> dict:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return {"hbm_gbs": d.get("hbm_gbs"), "bf16_tflops": d.get("bf16_tflops"),
                "bf16_tflops_sustained": d.get("bf16_tflops_sustained"), "source": "measured"}
    return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "bf16_tflops_sustained": 1400.0,
            "source": "fallback"}


def traffic_from_profiles(tall_flops_step: float):
    """DRAM bytes of the tall-matrix launches of one step, from the committed ncu summary
    (bytes per algorithmic flop of its voxels, captured on a smaller case), valid while the
    kernel's sources match the summary's source_sha (else None)."""
    import hashlib
    import re
    csrc = os.path.join(ROOT, "paper_2410_17084_b300", "csrc")
    h = hashlib.sha256()
    for f in ("gpv_tall.cu", "gpv_num.cuh", "gpv_umma.cuh", "gpv_internal.h", "gpv_common.cuh",
              "gpv_init.cuh"):
        h.update(open(os.path.join(csrc, f), "rb").read())
    sha = h.hexdigest()[:16]
    path = os.path.join(ROOT, "profiles", "tall_stress_traffic.md")
    if not os.path.exists(path):
        return None
    txt = open(path).read()
    m_sha = re.search(r"source_sha:\s*([0-9a-f]+)", txt)
    m_b = re.search(r"dram_bytes_per_flop:\s*([0-9.eE+-]+)", txt)
    if not m_sha or not m_b or m_sha.group(1) != sha:
        return None
    return float(m_b.group(1)) * tall_flops_step


# ---- oracle comparison ------------------------------------------------------------------
class ErrSample:
    """A fixed, seeded sample of a workload's voxels, solved once by the FP64 oracle; the
    GPU outputs of any leg on that workload are compared with it per output."""

    def __init__(self, b, nsample=ERR_SAMPLE, seed=12345):
        from oracle import compare
        from oracle import oracle as O
        rng = np.random.default_rng(seed)
        idx = np.sort(rng.choice(b.nvox, size=min(nsample, b.nvox), replace=False))
        self.idx = idx
        self.b = b
        self.sub = b.subset(idx)
        t = time.perf_counter()
        self.ref = compare.oracle_for_batch(self.sub)
        self.ri = O.init_batch(self.ref["mean"], self.ref["var"], self.ref["axis"],
                               self.sub.centres, self.sub.sf2, b.size, b.G, b.n_s, b.n_r)
        self.seconds = time.perf_counter() - t

    def errors(self, out) -> dict:
        """out: device outputs of the whole workload (axis, mean, var, status[, pos, ...])."""
        import torch
        from oracle import compare
        from oracle import oracle as O
        it = torch.from_numpy(self.idx).to(out["mean"].device)
        g = {k: out[k].index_select(0, it).cpu().numpy() for k in ("axis", "mean", "var", "status")}
        ref = self.ref
        ax = g["axis"].astype(np.int32)
        diff = np.nonzero((ref["status"] == 0) & (ax != ref["axis"]) & (ax <= 2))[0]
        if diff.size:  # axis-ambiguous voxels: the oracle takes the GPU's axis
            ref = compare.oracle_for_batch(self.sub, gpu_axis=ax)
        solved = (ref["status"] == 0) & ((g["status"].astype(np.uint32) & 0x55) == 0)
        e = compare.gpr_errors(g["mean"], g["var"], ref, self.sub.sn2, solved)
        res = {"sample_voxels": int(self.idx.size), "compared": e["n"],
               "mean_max": e["mean_max"], "mean_p99": e["mean_p99"],
               "var_max": e["var_max"], "var_p99": e["var_p99"],
               "ambiguous_axis_reruns": int(diff.size)}
        if "pos" in out:
            ng = self.b.n_s * self.b.n_s
            gi = (self.idx[:, None] * ng + np.arange(ng)[None, :]).reshape(-1)
            gt = torch.from_numpy(gi).to(out["pos"].device)
            ri = self.ri if not diff.size else O.init_batch(
                ref["mean"], ref["var"], ref["axis"], self.sub.centres, self.sub.sf2,
                self.b.size, self.b.G, self.b.n_s, self.b.n_r)
            ie = compare.init_errors(out["pos"].index_select(0, gt).cpu().numpy(),
                                     out["scale"].index_select(0, gt).cpu().numpy(),
                                     out["quat"].index_select(0, gt).cpu().numpy(), ri,
                                     valid=np.repeat(solved, ng))
            res.update(scale_rel_max=ie["scale_rel_max"], rot_max=ie["rot_max"],
                       unpinned_axes=ie["unpinned_axes"])
        return res


# ---- reference arm: the oracle on the host cores ------------------------------------------
def run_reference(args, rank, world):
    """The FP64 CPU oracle timed on the host cores on a bounded sample of the workload."""
    from oracle import oracle as O
    from paper_2410_17084_b300 import synth
    if rank != 0:
        return
    b = synth.stress_batch()
    ncpu = os.cpu_count() or 1
    rng = np.random.default_rng(99)
    probe = b.subset(np.sort(rng.choice(b.nvox, 2000, replace=False)))
    t = time.perf_counter()
    O.solve_batch(probe.xyz, probe.offsets, probe.centres, probe.lam, probe.sf2, probe.sn2,
                  b.size, b.G, b.tau, nthreads=ncpu)
    per = (time.perf_counter() - t) / probe.nvox
    k = int(min(b.nvox, max(500, 4.0 / max(per, 1e-9))))  # about 4 s of host work per step
    times = []
    for s in range(args.warmup + args.steps):
        idx = np.sort(rng.choice(b.nvox, k, replace=False))
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
                         "kind": "oracle",
                         "sample": f"{k} voxels drawn at random from the workload per step"},
        "e2e": {"value": value, "unit": "voxel solves/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def oracle_per_config(extras: dict, errs5) -> dict:
    """The oracle's own rate on every batch workload (GPR + Gaussian init, all host cores):
    the 1,000-voxel plane workload in full, timed here, and the fixed 2,000-voxel samples
    of the quadric, escalation and headline workloads that the error figures re-solve
    (timed when they were solved).  Rates per workload, not extrapolated to its size."""
    from oracle import oracle as O
    from paper_2410_17084_b300 import synth
    ncpu = os.cpu_count() or 1
    c1 = synth.plane_batch()
    t = time.perf_counter()
    r = O.solve_batch(c1.xyz, c1.offsets, c1.centres, c1.lam, c1.sf2, c1.sn2, c1.size, c1.G,
                      c1.tau, nthreads=ncpu)
    O.init_batch(r["mean"], r["var"], r["axis"], c1.centres, c1.sf2, c1.size, c1.G, c1.n_s,
                 c1.n_r)
    dt = time.perf_counter() - t
    out = {"plane1k": {"voxels": c1.nvox, "seconds": dt, "value": c1.nvox / dt,
                       "sample": "the whole workload"}}
    for name, key in (("quadric50k", "quadric50k"), ("mixed200k", "mixed200k")):
        sec = extras.get(key, {}).get("oracle_seconds")
        if sec:
            out[name] = {"voxels": ERR_SAMPLE, "seconds": sec, "value": ERR_SAMPLE / sec,
                         "sample": f"the {ERR_SAMPLE}-voxel error sample"}
    if errs5 is not None and errs5.seconds > 0:
        out["stress1m"] = {"voxels": int(errs5.idx.size), "seconds": errs5.seconds,
                           "value": errs5.idx.size / errs5.seconds,
                           "sample": f"the {errs5.idx.size}-voxel error sample"}
    return {"unit": "voxel solves/s", "cores": ncpu, "configs": out}


def cpu_baseline_leg(b, budget_s=15.0) -> dict:
    """The oracle (GPR + Gaussian init) on all host cores over a bounded random sample of
    the workload, sized from a probe to about budget_s."""
    from oracle import oracle as O
    ncpu = os.cpu_count() or 1
    rng = np.random.default_rng(7)

    def one(sub):
        r = O.solve_batch(sub.xyz, sub.offsets, sub.centres, sub.lam, sub.sf2, sub.sn2, b.size,
                          b.G, b.tau, nthreads=ncpu)
        O.init_batch(r["mean"], r["var"], r["axis"], sub.centres, sub.sf2, b.size, b.G, b.n_s,
                     b.n_r)

    probe = b.subset(np.sort(rng.choice(b.nvox, min(b.nvox, 1500), replace=False)))
    t = time.perf_counter()
    one(probe)
    per = (time.perf_counter() - t) / probe.nvox
    k = int(min(b.nvox, max(probe.nvox, budget_s / max(per, 1e-9))))
    sub = b.subset(np.sort(rng.choice(b.nvox, k, replace=False)))
    t = time.perf_counter()
    one(sub)
    dt = time.perf_counter() - t
    return {"value": k / dt, "unit": "voxel solves/s", "cores": ncpu, "kind": "oracle",
            "sample": f"{k} voxels drawn at random from the {b.nvox}-voxel workload "
                      "(GPR + Gaussian init)", "seconds": dt}


# ---- GPU legs ---------------------------------------------------------------------------
def tc_workspace_mb(batch, nmax=224) -> int:
    """MiB of tensor-core variance workspace a batch needs (the handle's per-voxel hand-over
    of L^-1, the node factors and the means, float-float): every voxel that takes the
    tensor-core variance gets its own slice, so a batch of a million voxels needs more
    than the 4 GiB default."""
    G = batch.G
    Gp = (G + 3) // 4 * 4
    n = batch.counts[(batch.counts <= nmax) & (batch.counts >= batch.tau)].astype(np.int64)
    e = n * (n + 1) // 2 + n * G + n * Gp + 2 * G * G
    need = int(np.sum((8 * e + 4 * (n + G * G) + 15) // 16 * 16))
    return max(4096, (need >> 20) + 256)


def make_handle(gv, batch, prec, **kw):
    kw.setdefault("tc_workspace_mb", tc_workspace_mb(batch))
    cfg = gv.gp_voxels_config_default(voxel_size=batch.size, grid_side=batch.G,
                                      n_s=batch.n_s, n_r=batch.n_r, tau=batch.tau,
                                      max_points=int(max(256, batch.counts.max())),
                                      max_voxels=batch.nvox, precision=prec, **kw)
    return gv.GpVoxels(cfg)


def solve_leg(gv, batch, dev, prec, timed, errs=None, steps=3, warmup=2, graph=True,
              init=True, tune=True):
    g = make_handle(gv, batch, prec)
    tuned = None
    if tune:  # launch shapes per size bucket, on a prefix of the leg's own workload
        pre = batch.subset(np.arange(min(batch.nvox, 100000)))
        dp = gv.batch_to_device(pre)
        tuned = g.autotune(dp["xyz"], dp["offsets"], dp["centres"], dp["lam"], dp["sf2"],
                           dp["sn2"])
        del dp
    o = g.outputs(batch.nvox, "cuda", init=init)
    f = lambda: g.solve_csr(dev["xyz"], dev["offsets"], dev["centres"], dev["lam"],
                            dev["sf2"], dev["sn2"], out=o, init=init)
    if graph:
        gr = gv.capture_graph(f)
        f = gr.replay
    ms = timed(f, steps, warmup)
    st = o["status"].cpu().numpy()
    t = sum(ms) / len(ms)
    res = {"value": batch.nvox / (t * 1e-3), "unit": "voxel solves/s", "ms_per_step": t,
           "steps": steps, "predicted_pts_per_s": batch.nvox * batch.G * batch.G / (t * 1e-3),
           "escalated": int(((st & gv.VOX_ESCALATED) != 0).sum())}
    if tuned is not None:
        res["autotune"] = f"{tuned} size buckets changed (100,000-voxel prefix)"
    if errs is not None:
        res["err"] = errs.errors(o)
    g.close()
    return res


def run_extras(b5, errs5, timed, stream) -> dict:
    """Secondary legs, each with its error against the oracle: plain FP32 on the headline
    workload, the one-voxel-per-launch FP32 baseline, the escalation workload (200,000
    voxels, G = 32) mixed and FP32, the 50,000-voxel quadric workload, the paper's Alg. 3
    formulation, L_p, the rasteriser and serving at 10 Hz."""
    import torch
    from paper_2410_17084_b300 import gp_voxels as gv, serve, synth
    ex = {}
    try:
        d5 = gv.batch_to_device(b5)
        ex["stress1m_fp32"] = solve_leg(gv, b5, d5, gv.PREC_FP32, timed, errs5)
        del d5
        # one voxel per launch (plain FP32), on a random sample of the headline workload
        rng = np.random.default_rng(5)
        bs = b5.subset(np.sort(rng.choice(b5.nvox, 5000, replace=False)))
        ds = gv.batch_to_device(bs)
        gsub = make_handle(gv, bs, gv.PREC_FP32, refine=0)
        osub = gsub.outputs(bs.nvox, "cuda", init=True)
        mpl = timed(lambda: gsub.solve_csr(ds["xyz"], ds["offsets"], ds["centres"], ds["lam"],
                                           ds["sf2"], ds["sn2"], out=osub, init=True,
                                           one_per_launch=True, stream=stream), 1, 1)
        gsub.close()
        tpl = sum(mpl) / len(mpl)
        ex["fp32_one_voxel_per_launch"] = {
            "value": bs.nvox / (tpl * 1e-3), "unit": "voxel solves/s",
            "sample": "5,000 voxels drawn at random from the headline workload, one launch "
                      "per voxel (plain FP32, no refinement)"}
    except Exception as e:  # an extra must not lose the headline
        ex["fp32_error"] = repr(e)
    try:
        c3 = synth.mixed_batch()
        e3 = ErrSample(c3)
        d3 = gv.batch_to_device(c3)
        ex["mixed200k"] = {
            "workload": "200,000 voxels, counts power-law on [32,512], 10% collinear voxels "
                        "(sn = 1e-4, Gram condition > 1e8), G = 32, fused init, one CUDA-graph "
                        "replay per step",
            "mixed": solve_leg(gv, c3, d3, gv.PREC_MIXED, timed, e3),
            "fp32": solve_leg(gv, c3, d3, gv.PREC_FP32, timed, e3),
            "oracle_seconds": e3.seconds}
        del d3
    except Exception as e:
        ex["mixed200k_error"] = repr(e)
    try:
        c2 = synth.quadric_batch()
        e2 = ErrSample(c2)
        d2 = gv.batch_to_device(c2)
        ex["quadric50k"] = {
            "workload": "50,000 voxels, lognormal counts (median 64) clipped to [16,256], "
                        "G = 16, fused init, one CUDA-graph replay per step",
            "mixed": solve_leg(gv, c2, d2, gv.PREC_MIXED, timed, e2, steps=5),
            "fp32": solve_leg(gv, c2, d2, gv.PREC_FP32, timed, e2, steps=5),
            "oracle_seconds": e2.seconds}
        # the paper's Alg. 3 formulation with the full posterior covariance
        na = 5000
        ba = c2.subset(np.arange(na))
        da = gv.batch_to_device(ba)
        ga = make_handle(gv, ba, gv.PREC_MIXED)
        Q = c2.G * c2.G
        oa = {"axis": torch.empty(na, dtype=torch.uint8, device="cuda"),
              "mean": torch.empty(na, Q, device="cuda"),
              "cov": torch.empty(na, Q, Q, device="cuda"),
              "status": torch.empty(na, dtype=torch.int32, device="cuda")}
        fa = lambda: gv.gp_voxels_solve_alg3(ga.h, da["xyz"], da["offsets"], na, da["centres"],
                                             da["lam"], da["sf2"], da["sn2"], oa["axis"],
                                             oa["mean"], oa["cov"], oa["status"])
        nmax_a3 = fa()
        ma = timed(fa, 3, 2)
        st = oa["status"].cpu().numpy().astype(np.uint32)
        ga.close()
        ta = sum(ma) / len(ma)
        ex["alg3_full_covariance"] = {
            "workload": f"first {na} voxels of the quadric workload, the paper's Alg. 3 (FP32 "
                        "LU + explicit inverse, full G^2 x G^2 Sigma* on tcgen05, 3xTF32)",
            "value": na / (ta * 1e-3), "unit": "voxel solves/s", "ms_per_step": ta,
            "sigma_GBps": na * Q * Q * 4 / (ta * 1e-3) / 1e9,
            "solved": int((st == 0).sum()), "too_large": int(((st & gv.VOX_TOO_LARGE) != 0).sum()),
            "nmax": nmax_a3}
        del da, oa
        # structure similarity loss (Eq. 11) and rasterisation (Eq. 9) of the Gaussians
        gl = make_handle(gv, c2, gv.PREC_MIXED)
        ol = gl.solve_csr(d2["xyz"], d2["offsets"], d2["centres"], d2["lam"], d2["sf2"],
                          d2["sn2"], init=True)
        ok = torch.repeat_interleave((ol["status"] & 0x15) == 0, c2.n_s * c2.n_s)
        gpos = ol["pos"][ok].contiguous()
        gsc = ol["scale"][ok].contiguous()
        m = int(gpos.shape[0])
        npts = int(d2["xyz"].shape[0])
        lossd = torch.empty(1, dtype=torch.float64, device="cuda")
        cell = c2.size / c2.n_s
        fl = lambda: gv.gp_voxels_structure_loss(gl.h, gpos, gsc, m, d2["xyz"], npts, cell, lossd)
        ml = timed(fl, 3, 2)
        tl = sum(ml) / len(ml)
        ex["structure_loss"] = {
            "workload": f"L_p of Eq. 11: the {npts} points of the quadric workload against the "
                        f"{m} Gaussians initialised from it (hash grid, cell {cell} m)",
            "value": npts / (tl * 1e-3), "unit": "points/s", "ms_per_step": tl,
            "loss_m": float(lossd.item())}
        rng = np.random.default_rng(81)
        gq = ol["quat"][ok].contiguous()
        gop = torch.from_numpy(rng.uniform(0.2, 1.0, m).astype(np.float32)).cuda()
        gcol = torch.from_numpy(rng.uniform(0.0, 1.0, (m, 3)).astype(np.float32)).cuda()
        W, H = 1920, 1080
        cam = gv.make_camera(np.diag([1.0, -1.0, -1.0]), [0.0, 0.0, 20.0], 700.0, 700.0,
                             W / 2, H / 2, W, H, 0.2)
        img = torch.empty(H, W, 3, device="cuda")
        dep = torch.empty(H, W, device="cuda")
        sil = torch.empty(H, W, device="cuda")
        pairs = []
        fr = lambda: pairs.append(gv.gp_voxels_render(gl.h, gpos, gsc, gq, gop, gcol, m, cam,
                                                      img, dep, sil))
        mr = timed(fr, 3, 2)
        tr = sum(mr) / len(mr)
        ex["rasterize"] = {
            "workload": f"{m} Gaussians (initialised from the quadric workload, seeded colours "
                        f"and opacities), one {W}x{H} camera 20 m above, colour + depth + "
                        "silhouette",
            "value": 1e3 / tr, "unit": "images/s", "ms_per_image": tr,
            "gaussians_per_s": m / (tr * 1e-3), "tile_pairs": pairs[-1],
            "covered": float((sil > 0).float().mean().item())}
        gl.close()
        del d2
    except Exception as e:
        ex["quadric50k_error"] = repr(e)
    try:
        ex.update(serving_legs(gv, serve, synth))
    except Exception as e:
        ex["serving_error"] = repr(e)
    return ex


def serving_legs(gv, serve, synth, nsc=None) -> dict:
    """Serving at the LiDAR workload's configuration (Sec. 3.3, Alg. 2): 256-point buckets,
    9 x 9 grid, 4 GB budget, scans arriving at 10 Hz (Poisson), checked against the oracle
    on a sample of the rows of every 50th scan."""
    import torch
    from oracle import compare
    nsc = nsc or int(os.environ.get("GPV_BENCH_SCANS", "600"))
    scene = synth.lidar_scene()
    scans = [synth.lidar_scan(scene, k) for k in range(nsc)]
    cfg = serve.serving_config()
    srv = serve.Server(cfg)
    srv.run(scans[:3], realtime=False)  # first-use set-up of the kernels
    srv.close()
    srv2 = serve.Server(cfg)
    lat, wall, _ = srv2.run(scans, arrivals=scene.arrivals[:nsc], realtime=True)
    srv2.close()
    # error: the first scans again, outputs collected, against the oracle's store and
    # FP64 solve of the same points
    nerr = 40
    srv3 = serve.Server(cfg)
    _, _, res = srv3.run(scans[:nerr], realtime=False, collect=True, max_inflight=1)
    srv3.close()
    errs = serving_oracle_err(gv, synth, cfg, scans[:nerr], res, every=8)
    ex = {"serving": {
        "workload": f"{nsc} synthetic 64x1024 LiDAR scans, Poisson arrivals at 10 Hz, 0.5 m "
                    f"voxels, {cfg.max_points}-point buckets, G = 9, mixed precision + init, "
                    f"{cfg.mem_budget >> 30} GB budget",
        "scans": nsc, "p50_ms": float(np.percentile(lat * 1e3, 50)),
        "p99_ms": float(np.percentile(lat * 1e3, 99)), "max_ms": float(lat.max() * 1e3),
        "scans_per_s": nsc / wall, "err": errs}}
    return ex


def serving_oracle_err(gv, synth, cfg, scans, res, every=8) -> dict:
    """The oracle's store (Alg. 2) fed the same scans in order; every `every`-th scan's rows
    solved by the FP64 oracle from the points it holds and compared with the served rows."""
    from oracle import compare
    from oracle import oracle as O
    store = O.VoxelStore(cfg.voxel_size, cfg.max_points)
    mm, vm, nrow = 0.0, 0.0, 0
    for k, scan in enumerate(scans):
        touched = store.insert_scan(scan)
        if k % every:
            continue
        r = res[k]
        pts = [store.points(t) for t in touched]
        counts = np.array([q.shape[0] for q in pts], dtype=np.int64)
        off = np.zeros(len(pts) + 1, np.int64)
        off[1:] = np.cumsum(counts)
        nv = len(pts)
        cen = O.voxel_centres(np.array(touched, np.int32), cfg.voxel_size)
        b = synth.VoxelBatch("scan", np.concatenate(pts).astype(np.float32), off, cen,
                             np.full(nv, cfg.lambda_, np.float32), np.full(nv, cfg.sf2, np.float32),
                             np.full(nv, cfg.sn2, np.float32), cfg.voxel_size, cfg.grid_side,
                             cfg.n_s, cfg.n_r, cfg.tau, counts, np.zeros(nv, bool))
        ax = r["axis"].astype(np.int32)
        ref = compare.oracle_for_batch(b, gpu_axis=np.where(ax <= 2, ax, -1))
        solved = (ref["status"] == 0) & ((r["status"].astype(np.uint32) & 0x55) == 0)
        e = compare.gpr_errors(r["mean"], r["var"], ref, b.sn2, solved)
        mm, vm, nrow = max(mm, e["mean_max"]), max(vm, e["var_max"]), nrow + e["n"]
    return {"mean_max": mm, "var_max": vm, "rows_compared": nrow,
            "sample": f"every {every}th of the first {len(scans)} scans, every solved row, "
                      "against the oracle's store and FP64 solve of the same points"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="headline leg only")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    from paper_2410_17084_b300 import dist as D
    rank, world, local = D.rank_world()
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

    b = synth.stress_batch(seed=D.rank_seed(4, rank))  # independent batch per rank
    G = b.G
    d = gv.batch_to_device(b)
    g = make_handle(gv, b, gv.PREC_MIXED, mean_mode=1)
    plan = gv.gp_voxels_plan_info(g.h)
    fl = split_flops(b.counts, G, plan)
    # autotune the shared-memory buckets on a 100,000-voxel prefix (same count distribution)
    pre = b.subset(np.arange(100000))
    dp = gv.batch_to_device(pre)
    tuned = g.autotune(dp["xyz"], dp["offsets"], dp["centres"], dp["lam"], dp["sf2"], dp["sn2"])
    del dp
    meas_ff = gv.gp_voxels_measure_peak(1)
    peaks = measured_peaks()
    out = g.outputs(b.nvox, "cuda", init=True)
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def step():
        gv.gp_voxels_solve_csr(g.h, d["xyz"], d["offsets"], b.nvox, d["centres"], d["lam"],
                               d["sf2"], d["sn2"], out["axis"], out["mean"], out["var"],
                               out["status"], out["pos"], out["scale"], out["quat"], 0,
                               torch.cuda.current_stream())

    tall_ms = []

    def timed(fn, steps, warmup, tall=None):
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
            if tall is not None:  # the tall-matrix launches of this step (events on their stream)
                tall.append(gv.gp_voxels_last_tall_ms(g.h))
        torch.cuda.synchronize()
        return [a.elapsed_time(c) for a, c in evs]

    gv.gp_voxels_set_timing(g.h, True)
    graph = gv.capture_graph(step)
    launches = gv.gp_voxels_last_launches(g.h)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        ms = timed(graph.replay, args.steps, args.warmup, tall=tall_ms)
    t_step = D.max_over_ranks(sum(ms) / len(ms), dist, "cuda")
    value = world * b.nvox / (t_step * 1e-3)
    st = out["status"].cpu().numpy()
    n_esc = int(((st & gv.VOX_ESCALATED) != 0).sum())
    errs5 = ErrSample(b) if rank == 0 else None
    err = errs5.errors(out) if rank == 0 else None

    # ---- e2e: host buffers in, host buffers out, through the C ABI ------------------
    pin = {k: torch.from_numpy(getattr(b, k)).pin_memory() for k in
           ("xyz", "offsets", "centres", "lam", "sf2", "sn2")}
    h2d = sum(v.numel() * v.element_size() for v in pin.values())
    d2h = sum(v.numel() * v.element_size() for v in out.values())
    # Streamed: two sets of device inputs and outputs; every step copies its inputs in and
    # its outputs out (pinned host memory) on copy streams of their own, so the copies of
    # one step overlap the neighbouring steps' solves.  Timed from the first input copy to
    # the last output copy.
    d2 = {k: torch.empty_like(v) for k, v in d.items()}
    dsets, osets = [d, d2], [out, g.outputs(b.nvox, "cuda", init=True)]
    hsets = [{k: torch.empty(v.shape, dtype=v.dtype).pin_memory() for k, v in out.items()}
             for _ in range(2)]
    s_in, s_out = torch.cuda.Stream(), torch.cuda.Stream()
    gv.gp_voxels_set_timing(g.h, False)

    def e2e_stream(nsteps):
        ev_in = [torch.cuda.Event() for _ in range(2)]
        ev_done = [torch.cuda.Event() for _ in range(2)]
        ev_out = [torch.cuda.Event() for _ in range(2)]
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        s_in.wait_event(e0)
        s_out.wait_event(e0)
        for k in range(nsteps):
            j = k % 2
            with torch.cuda.stream(s_in):
                if k >= 2:
                    s_in.wait_event(ev_done[j])  # the solve of step k - 2 released set j
                for key, v in pin.items():
                    dsets[j][key].copy_(v, non_blocking=True)
                ev_in[j].record(s_in)
            stream.wait_event(ev_in[j])
            if k >= 2:
                stream.wait_event(ev_out[j])  # the outputs of step k - 2 are read out
            o, dd = osets[j], dsets[j]
            gv.gp_voxels_solve_csr(g.h, dd["xyz"], dd["offsets"], b.nvox, dd["centres"],
                                   dd["lam"], dd["sf2"], dd["sn2"], o["axis"], o["mean"],
                                   o["var"], o["status"], o["pos"], o["scale"], o["quat"], 0,
                                   stream)
            ev_done[j].record(stream)
            with torch.cuda.stream(s_out):
                s_out.wait_event(ev_done[j])
                for key, v in o.items():
                    hsets[j][key].copy_(v, non_blocking=True)
                ev_out[j].record(s_out)
        e1.record(s_out)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / nsteps

    e2e_stream(2)  # warm-up
    t_e2e = D.max_over_ranks(e2e_stream(max(3, args.steps)), dist, "cuda")
    del d2, dsets, osets, hsets

    extras = {}
    if not args.no_extras and rank == 0:
        extras = run_extras(b, errs5, timed, stream)
    clocks = clk.summary()

    # ---- roofline ---------------------------------------------------------------------
    # dominant kernel: the tall-matrix launches (events around them on their own stream)
    t_tall = sum(tall_ms) / max(len(tall_ms), 1)
    bf16 = peaks["bf16_tflops_sustained"]
    p_tc = bf16 / SLICE_PAIRS         # float-float-accurate products on the tensor cores
    p_ff = meas_ff                     # measured float-float multiply-add rate, CUDA cores
    tall_floor_ms = 1e3 * (fl["tall_tc"] / (p_tc * 1e12) + fl["tall_ff"] / (p_ff * 1e12))
    tall_peak = fl["tall_total"] / (tall_floor_ms * 1e-3) / 1e12
    tall_ach = fl["tall_total"] / (t_tall * 1e-3) / 1e12 if t_tall > 0 else 0.0
    step_floor_ms = 1e3 * (fl["tc"] / (p_tc * 1e12) + fl["ff"] / (p_ff * 1e12))
    step_ach = fl["total"] / (t_step * 1e-3) / 1e12
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
                   "precision": "mixed (float-float + exact BF16 slice products + FP64 "
                                "escalation)",
                   "l2": "flushed between timed steps (256 MiB write); inputs 0.76 GB > L2",
                   "autotune": f"CTA size per shared-memory size bucket chosen by "
                               f"gp_voxels_autotune on a 100,000-voxel prefix ({tuned} changed)",
                   "plan": plan,
                   "parallelism": f"independent batches per GPU x{world}"},
        "predicted_pts_per_s": value * G * G,
        "escalated_voxels": n_esc,
        "gpu_launches": launches,
        "err": err,
        "roofline": {
            "bound": "tensor", "achieved": tall_ach, "peak": tall_peak, "unit": "TFLOP/s",
            "frac": tall_ach / tall_peak if tall_peak else None,
            "traffic": traffic_from_profiles(fl["tall_total"]),
            "kernel": "k_tall (tall-matrix factorisation of the voxels with more than "
                      f"{plan['tall_min']} points: {fl['tall_voxels']} voxels, "
                      f"{fl['tall_total'] / 1e12:.3f} TFLOP algorithmic per step)",
            "kernel_ms": t_tall,
            "peak_note": "composite floor of the kernel's algorithmic work by the unit that "
                         "runs it: the panel updates as exact BF16 slice products at the "
                         f"measured sustained BF16 rate / {SLICE_PAIRS} slice products per "
                         f"float-float product ({bf16} / {SLICE_PAIRS} = {p_tc:.1f} TFLOP/s), "
                         "the in-panel work (32 flops per row and column) at the measured "
                         f"float-float rate ({p_ff:.2f} TFLOP/s); peak = its work / that "
                         "floor (of measured)",
            "step": {"achieved": step_ach, "floor_ms": step_floor_ms,
                     "peak": fl["total"] / (step_floor_ms * 1e-3) / 1e12,
                     "frac": step_floor_ms / t_step,
                     "tc_tflop": fl["tc"] / 1e12, "ff_tflop": fl["ff"] / 1e12}},
        "e2e": {"value": world * b.nvox / (t_e2e * 1e-3), "unit": "voxel solves/s",
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "mode": "streamed: two device input/output sets, host-device copies on "
                        "their own streams overlapping the neighbouring steps' solves"},
        "clocks": clocks,
    }
    line.update(extras)
    if "fp32_one_voxel_per_launch" in extras:
        line["mixed_vs_fp32_one_voxel_per_launch"] = (
            value / world / extras["fp32_one_voxel_per_launch"]["value"])
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_leg(b)
        try:
            line["cpu_baseline"]["per_config"] = oracle_per_config(extras, errs5)
        except Exception as e:  # a report must not lose the line
            line["cpu_baseline"]["per_config_error"] = repr(e)
    if rank == 0:
        print(json.dumps(line), flush=True)
    g.close()
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
