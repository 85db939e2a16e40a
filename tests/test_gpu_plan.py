"""The launch plan and its conditioning rule on the GPU: size buckets as gp_voxels_bucket_info
reports them (consistent with the tall-matrix threshold, CTAs at least as large as their
shared-memory buckets, before and after gp_voxels_autotune), and the FP32 rule that a
factor without significant digits is reported not positive definite (GS-LIVM Sec. 3.1:
the Cholesky of K + D, Eq. 2-3), with the prior as output."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gpv():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2410_17084_b300 import build, gp_voxels
    build.build()
    return gp_voxels


def _handle(gpv, b, precision, **kw):
    d = dict(voxel_size=b.size, grid_side=b.G, n_s=b.n_s, n_r=b.n_r, tau=b.tau,
             max_points=int(max(b.counts.max(), b.tau, 8)), max_voxels=max(b.nvox, 1),
             precision=precision, mean_mode=1)
    d.update(kw)
    return gpv.GpVoxels(gpv.gp_voxels_config_default(**d))


def _check_plan(gpv, g, max_points):
    plan = gpv.gp_voxels_plan_info(g.h)
    buckets = gpv.gp_voxels_bucket_info(g.h)
    assert len(buckets) == plan["buckets"]
    his = [b["hi"] for b in buckets]
    assert his == sorted(his) and len(set(his)) == len(his)
    assert his[-1] == max_points
    tall_min = plan["tall_min"]
    for b in buckets:
        if tall_min > 0 and b["hi"] > tall_min:
            assert b["path"] == "tall", b
        else:
            assert b["path"] in ("shared", "shared+tc", "workspace"), b
        if b["path"] in ("shared", "shared+tc"):
            # the shared-memory kernels give every point of a voxel its own thread
            assert b["threads"] >= b["hi"] and b["threads"] in (32, 64, 128, 256, 512), b
            assert b["panel"] in (4, 8, 16), b
    return buckets


@pytest.mark.parametrize("precision", [1, 0])
def test_bucket_info_matches_the_routing(gpv, precision):
    """The 1M-voxel stress shapes (counts up to 1024, G = 9): buckets above the tall-matrix
    threshold take that path, the ones below it shared memory; after the autotuner the plan
    keeps those rules and the solve still matches the plan's routing."""
    import torch
    from paper_2410_17084_b300 import synth
    b = synth.stress_batch(20000)
    g = _handle(gpv, b, precision, max_points=1024)
    before = _check_plan(gpv, g, 1024)
    plan = gpv.gp_voxels_plan_info(g.h)
    assert plan["tall_min"] == (128 if precision == 1 else 160)
    if precision == 1:  # one and two warps per voxel for the smallest float-float buckets
        small = [x for x in before if x["hi"] <= 16]
        assert small and all(x["threads"] == 32 for x in small)
    d = gpv.batch_to_device(b)
    g.autotune(d["xyz"], d["offsets"], d["centres"], d["lam"], d["sf2"], d["sn2"])
    after = _check_plan(gpv, g, 1024)
    assert [x["hi"] for x in after] == [x["hi"] for x in before]
    out = g.solve_csr(d["xyz"], d["offsets"], d["centres"], d["lam"], d["sf2"], d["sn2"])
    torch.cuda.synchronize()
    st = out["status"].cpu().numpy()
    assert ((st & 0x55) == 0).mean() > 0.99
    g.close()


def test_fp32_reports_ill_conditioned_voxels_not_spd(gpv):
    """Collinear voxels with sn = 1e-4 (Gram condition beyond 1e8): the mixed path escalates
    them to FP64; plain FP32 cannot resolve them and reports GPV_VOX_NOT_SPD with the prior
    (mean = the data mean, variance = sf^2), while the well-conditioned voxels solve."""
    import torch
    from paper_2410_17084_b300 import synth
    full = synth.mixed_batch(3000)
    deg = np.nonzero(full.degenerate)[0][:60]
    good = np.nonzero(~full.degenerate)[0][:200]
    b = full.subset(np.concatenate([deg, good]))
    isdeg = np.zeros(b.nvox, bool)
    isdeg[:deg.size] = True
    res = {}
    for prec in (1, 0):
        g = _handle(gpv, b, prec)
        d = gpv.batch_to_device(b)
        out = g.solve_csr(d["xyz"], d["offsets"], d["centres"], d["lam"], d["sf2"], d["sn2"])
        torch.cuda.synchronize()
        res[prec] = {k: v.cpu().numpy() for k, v in out.items()}
        g.close()
    st32 = res[0]["status"].astype(np.uint32)
    stmx = res[1]["status"].astype(np.uint32)
    esc = (stmx & gpv.VOX_ESCALATED) != 0
    assert esc[isdeg].mean() > 0.5
    notspd = (st32 & gpv.VOX_NOT_SPD) != 0
    print(f"\nFP32 not SPD: {int(notspd[isdeg].sum())} of {int(isdeg.sum())} collinear, "
          f"{int(notspd[~isdeg].sum())} of {int((~isdeg).sum())} others")
    assert notspd[isdeg].mean() > 0.9
    assert not notspd[~isdeg].any()
    # the prior: variance sf^2 at every query, mean constant over the grid
    sf2 = b.sf2.astype(np.float32)
    for v in np.nonzero(notspd)[0]:
        assert np.all(res[0]["var"][v] == sf2[v])
        assert np.all(res[0]["mean"][v] == res[0]["mean"][v][0])
