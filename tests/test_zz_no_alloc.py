"""The allocation-free batched solve (gp_voxels_solve_csr_noalloc) against the handle
entry point (gp_voxels_solve_csr), called through the C ABI.

That entry point exists for callers that may not allocate device memory, such as code
embedded in a host application that owns every device allocation, or an op of another
framework that can only use the tensors it is given; it keeps its work queues in a
static scratch area of the library instead.  Two calls in a row must both match the
handle path (the second one sees the scratch left by the first), within the tolerance of
the other parity tests: posterior mean 1e-4 m, variance 1e-3 relative.

The file is named to be collected after the other GPU tests; it passes alone in a fresh
process as well as after them (the static scratch keeps whatever earlier calls left).
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

MEAN_TOL = 1e-4
VAR_TOL = 1e-3


def _batch():
    from paper_2410_17084_b300 import synth
    full = synth.quadric_batch(6000, seed=31)
    keep = np.nonzero(full.counts <= 160)[0][:3000]
    return full.subset(keep)


@pytest.mark.parametrize("precision,panel", [(1, 0), (0, 0), (1, 8)])
def test_noalloc_matches_handle_solve_twice(precision, panel):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2410_17084_b300 import build, gp_voxels as gv
    build.build()
    b = _batch()
    d = gv.batch_to_device(b)
    cfg = gv.gp_voxels_config_default(voxel_size=b.size, grid_side=b.G, n_s=b.n_s, n_r=b.n_r,
                                      tau=b.tau, max_points=160, max_voxels=b.nvox,
                                      precision=precision, factor_panel=panel)
    g = gv.GpVoxels(cfg)
    ref = g.solve_csr(d["xyz"], d["offsets"], d["centres"], d["lam"], d["sf2"], d["sn2"],
                      init=True)
    torch.cuda.synchronize()
    ref = {k: v.cpu().numpy() for k, v in ref.items()}
    g.close()
    solved = (ref["status"] & 0x15) == 0
    assert solved.sum() > 0.9 * b.nvox
    for call in range(2):
        out = gv.GpVoxels.outputs(g, b.nvox, "cuda", init=True)
        for v in out.values():
            v.fill_(7)  # stale values must be overwritten
        gv.gp_voxels_solve_csr_noalloc(cfg, d["xyz"], d["offsets"], b.nvox, d["centres"],
                                       d["lam"], d["sf2"], d["sn2"], out["axis"], out["mean"],
                                       out["var"], out["status"], out["pos"], out["scale"],
                                       out["quat"])
        torch.cuda.synchronize()
        o = {k: v.cpu().numpy() for k, v in out.items()}
        assert np.array_equal(o["status"], ref["status"]), f"call {call}: status"
        assert np.array_equal(o["axis"], ref["axis"]), f"call {call}: axis"
        m = solved
        assert np.abs(o["mean"][m] - ref["mean"][m]).max() <= MEAN_TOL
        floor = 1e-3 * b.sn2[m][:, None]
        rel = np.abs(o["var"][m] - ref["var"][m]) / np.maximum(ref["var"][m], floor)
        assert rel.max() <= VAR_TOL
        ng = b.n_s * b.n_s
        gm = np.repeat(m, ng)
        assert np.allclose(o["pos"][gm], ref["pos"][gm], rtol=0, atol=1e-5)
        assert np.allclose(o["scale"][gm], ref["scale"][gm], rtol=1e-4, atol=1e-9)


def test_noalloc_limits():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2410_17084_b300 import gp_voxels as gv
    from paper_2410_17084_b300 import synth
    cfg = gv.gp_voxels_config_default(voxel_size=0.5, grid_side=16, n_s=4, n_r=4, tau=16,
                                      max_points=2048, precision=gv.PREC_MIXED)
    # more voxels than the static scratch holds: rejected before any work is queued
    n = gv.NOALLOC_MAX_VOXELS + 1
    z = torch.zeros(n, device="cuda")
    off = torch.zeros(n + 1, dtype=torch.int64, device="cuda")
    with pytest.raises(gv.GpvError) as ei:
        gv.gp_voxels_solve_csr_noalloc(cfg, z, off, n, z, z, z, z, z, z, z, z)
    assert ei.value.code == gv.GPV_EINVAL
    # a panel width the handle path rejects is rejected here too
    bad = gv.gp_voxels_config_default(voxel_size=0.5, grid_side=16, n_s=4, n_r=4, tau=16,
                                      max_points=256, precision=gv.PREC_MIXED, factor_panel=5)
    with pytest.raises(gv.GpvError) as ei:
        gv.gp_voxels_solve_csr_noalloc(bad, z, off, 1, z, z, z, z, z, z, z, z)
    assert ei.value.code == gv.GPV_EINVAL
    # a voxel too large for shared memory is reported, not solved
    b = synth.quadric_batch(50, seed=32)
    big = synth.stress_batch(4000, seed=33)
    sel = np.argsort(big.counts)[-1:]
    bb = big.subset(sel)
    assert bb.counts[0] > 300
    d = gv.batch_to_device(bb)
    axis = torch.empty(1, dtype=torch.uint8, device="cuda")
    mean = torch.empty(1, 256, device="cuda")
    var = torch.empty(1, 256, device="cuda")
    st = torch.empty(1, dtype=torch.int32, device="cuda")
    gv.gp_voxels_solve_csr_noalloc(cfg, d["xyz"], d["offsets"], 1, d["centres"], d["lam"],
                                   d["sf2"], d["sn2"], axis, mean, var, st)
    torch.cuda.synchronize()
    assert int(st.item()) == gv.VOX_TOO_LARGE
    assert float(var[0, 0].item()) == float(bb.sf2[0])
    del b
