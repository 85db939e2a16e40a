"""GPU parity of the posterior variance formed on the tensor cores (GS-LIVM Eq. 3,
diag(Sigma*) = sf2 - |L^-1 k_q|^2 by exact BF16 slice products, then the Gaussians of
Sec. 3.2) against the FP64 oracle, and against the same solve with the variance formed
on the CUDA cores (tc_workspace_mb = 0).

Tolerances: the oracle tolerances of the mixed path (mean 1e-4 m, variance 1e-3 relative
to max(var_ref, 1e-3 sigma^2), scale 1e-4, rotation 1e-3 rad).  Both variance paths carry
about 48 bits before the cancellation in sf2 - |v|^2, so they agree far more tightly:
|var_tc - var_cc| <= 1e-6 max(var_cc, 1e-3 sigma^2), and the means (which do not go through
the tensor cores) to 1e-7 m: the two runs may factor with different CTA sizes and panels.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

MEAN_TOL = 1e-4
VAR_TOL = 1e-3
SCALE_TOL = 1e-4
ROT_TOL = 1e-3
AGREE_TOL = 1e-6


@pytest.fixture(scope="module")
def gpv():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2410_17084_b300 import build, gp_voxels
    build.build()
    return gp_voxels


def _run(gpv, b, init=True, **kw):
    import torch
    d = dict(voxel_size=b.size, grid_side=b.G, n_s=b.n_s, n_r=b.n_r, tau=b.tau,
             max_points=int(max(b.counts.max(), b.tau, 8)), max_voxels=max(b.nvox, 1),
             precision=1, mean_mode=1, tall_min_points=-1)  # shared-memory kernels only
    d.update(kw)
    g = gpv.GpVoxels(gpv.gp_voxels_config_default(**d))
    dev = gpv.batch_to_device(b)
    out = g.solve_csr(dev["xyz"], dev["offsets"], dev["centres"], dev["lam"], dev["sf2"],
                      dev["sn2"], init=init)
    torch.cuda.synchronize()
    launches = gpv.gp_voxels_last_launches(g.h)
    res = {k: v.cpu().numpy() for k, v in out.items()}
    g.close()
    return res, launches


def _oracle_check(b, out, oracle, name, init=True):
    from oracle import compare
    ref = compare.oracle_for_batch(b, gpu_axis=out["axis"].astype(np.int32))
    solved = ref["status"] == 0
    assert np.array_equal(solved, (out["status"].astype(np.uint32) & 0x45) == 0), name
    err = compare.gpr_errors(out["mean"], out["var"], ref, b.sn2, solved)
    print(f"\n{name}: {err}")
    assert err["mean_max"] <= MEAN_TOL and err["var_max"] <= VAR_TOL, name
    if init:
        ri = oracle.init_batch(ref["mean"], ref["var"], ref["axis"], b.centres, b.sf2, b.size,
                               b.G, b.n_s, b.n_r)
        valid = np.repeat(solved, b.n_s * b.n_s)
        e = compare.init_errors(out["pos"], out["scale"], out["quat"], ri, valid=valid)
        print(f"{name} init: {e}")
        assert e["pos_max"] <= 1e-4 and e["scale_rel_max"] <= SCALE_TOL and e["rot_max"] <= ROT_TOL
    return solved


def _agree(b, tc, cc, solved, name, exact_mean=False):
    # the two runs may factor with different launch configurations (the variant without the
    # contraction has defaults and a shared-memory plan of its own): means agree to rounding
    if exact_mean:
        assert np.array_equal(tc["mean"], cc["mean"]), name
    assert np.abs(tc["mean"] - cc["mean"])[solved].max() <= 1e-7, name
    floor = 1e-3 * b.sn2.astype(np.float64)[:, None]
    rel = np.abs(tc["var"].astype(np.float64) - cc["var"]) / np.maximum(cc["var"], floor)
    worst = float(rel[solved].max()) if solved.any() else 0.0
    print(f"{name}: tensor-core vs CUDA-core variance, max rel {worst:.2e}")
    assert worst <= AGREE_TOL, name


def _quadric(nvox, seed, lo=16, hi=192, pool=None):
    from paper_2410_17084_b300 import synth
    full = synth.quadric_batch(pool or nvox * 4, seed=seed)
    idx = np.nonzero((full.counts >= lo) & (full.counts <= hi))[0][:nvox]
    return full.subset(idx)


def test_tc_quadric_against_oracle_and_cuda_cores(gpv, oracle):
    """16 x 16 grid (two M tiles of 128 queries), counts 16..192 (one or two passes of
    96 rows of L^-1), fused Gaussian init."""
    b = _quadric(600, seed=31)
    tc, l_tc = _run(gpv, b)
    cc, l_cc = _run(gpv, b, tc_workspace_mb=0)
    assert l_tc > l_cc + 2  # k_var_tc per bucket, the re-solve of what was not handed over, k_init_tc
    solved = _oracle_check(b, tc, oracle, "tc quadric G=16")
    _agree(b, tc, cc, solved, "tc quadric G=16")


@pytest.mark.parametrize("shape", ["G9", "G32"])
def test_tc_grid_sides(gpv, oracle, shape):
    """One partly filled M tile (G = 9: 81 queries) and eight (G = 32)."""
    from paper_2410_17084_b300 import synth
    if shape == "G9":
        full = synth.stress_batch(3000, seed=33)
        idx = np.nonzero(full.counts <= 192)[0][:400]
    else:
        full = synth.mixed_batch(1500, seed=34)
        idx = np.nonzero(~full.degenerate & (full.counts <= 160))[0][:150]
    b = full.subset(idx)
    tc, l_tc = _run(gpv, b)
    cc, l_cc = _run(gpv, b, tc_workspace_mb=0)
    assert l_tc > l_cc + 2
    solved = _oracle_check(b, tc, oracle, f"tc {shape}")
    _agree(b, tc, cc, solved, f"tc {shape}")


def test_tc_largest_eligible_voxels(gpv, oracle):
    """n = 180..200 across the 192-point bound of the regular shared-memory plan: above it
    the tensor-core variant still factors in shared memory (bucket up to 224 points)."""
    b = _quadric(120, seed=35, lo=180, hi=200, pool=20000)
    assert (b.counts > 192).any() and (b.counts <= 192).any()
    tc, _ = _run(gpv, b, max_points=256)
    cc, _ = _run(gpv, b, max_points=256, tc_workspace_mb=0)
    solved = _oracle_check(b, tc, oracle, "tc n 180..200")
    # with the tensor-core variance on, 193..224-point voxels factor in shared memory (the
    # variant's smaller plan fits them); off, in the global workspace: the means agree to
    # rounding, not bit for bit
    _agree(b, tc, cc, solved, "tc n 180..200")


def test_tc_global_workspace_voxels(gpv, oracle):
    """n = 216..256 across the 224-point bound of the variant's shared-memory plan: above it
    the factor lives in the global workspace and the variance still goes to the tensor cores
    up to 255 points; 256-point voxels form it on the CUDA cores."""
    b = _quadric(120, seed=39, lo=216, hi=256, pool=40000)
    assert (b.counts <= 224).any() and ((b.counts > 224) & (b.counts < 256)).any()
    assert (b.counts == 256).any()
    tc, l_tc = _run(gpv, b, max_points=256)
    cc, l_cc = _run(gpv, b, max_points=256, tc_workspace_mb=0)
    assert l_tc > l_cc + 2
    solved = _oracle_check(b, tc, oracle, "tc n 216..256")
    _agree(b, tc, cc, solved, "tc n 216..256")


def test_tc_workspace_too_small_falls_back_whole_call(gpv):
    """A call whose eligible voxels need more workspace than configured forms every
    variance on the CUDA cores (the regular kernel re-solves them): it agrees with the
    solve with the workspace off to summation order, and repeats bit for bit."""
    b = _quadric(600, seed=36, lo=110, hi=160, pool=8000)  # ~600 x 100 KB > 16 MB
    small, _ = _run(gpv, b, tc_workspace_mb=16)
    again, _ = _run(gpv, b, tc_workspace_mb=16)
    off, _ = _run(gpv, b, tc_workspace_mb=0)
    for k in ("mean", "var", "status", "pos", "scale", "quat"):
        assert np.array_equal(small[k], again[k]), k
    assert np.array_equal(small["status"], off["status"])
    solved = (off["status"].astype(np.uint32) & 0x45) == 0
    _agree(b, small, off, solved, "workspace full")


def test_tc_repeatable(gpv):
    """Same inputs, same outputs (the work queues hand voxels out in any order)."""
    b = _quadric(500, seed=37)
    a, _ = _run(gpv, b)
    c, _ = _run(gpv, b)
    for k in ("mean", "var", "status", "pos", "scale", "quat"):
        assert np.array_equal(a[k], c[k]), k


def test_tc_workspace_within_memory_budget(gpv, oracle):
    """Under mem_budget the workspace takes what the budget leaves (here about 64 MB): a
    batch that fits takes the tensor-core variance, and the handle stays within budget."""
    b = _quadric(300, seed=38)
    # room for 5,000 voxels: the budget, not max_voxels, bounds the workspace
    base = dict(voxel_size=b.size, grid_side=b.G, n_s=b.n_s, n_r=b.n_r, tau=b.tau,
                max_points=int(b.counts.max()), max_voxels=5000, precision=1, mean_mode=1)
    rest = gpv.gp_voxels_query_sizes(gpv.gp_voxels_config_default(tc_workspace_mb=0, **base))
    budget = rest + (64 << 20)
    unbounded = gpv.gp_voxels_query_sizes(gpv.gp_voxels_config_default(**base))
    assert unbounded > budget
    assert gpv.gp_voxels_query_sizes(gpv.gp_voxels_config_default(mem_budget=budget, **base)) <= budget
    tc, l_tc = _run(gpv, b, mem_budget=budget, max_voxels=5000)
    cc, l_cc = _run(gpv, b, tc_workspace_mb=0, max_voxels=5000)
    assert l_tc > l_cc + 2  # the tensor-core variance ran
    solved = _oracle_check(b, tc, oracle, "tc under a memory budget")
    _agree(b, tc, cc, solved, "tc under a memory budget")
