"""GPU parity of the paper's own solve formulation (supplementary Alg. 3: LU with partial
pivoting, explicit inverse, mu* = k_k* f, FULL Sigma* = K** - k_k* K*; FP32 as the paper,
the last product on tcgen05 tensor cores as three TF32 products) against the FP64
oracle's full posterior covariance.

Tolerance, derived from the arithmetic: FP32 LU and inverse of ky = K + sigma^2 I carry
a relative error of order u kappa(ky) (u = 2^-24, kappa the 2-norm condition number), and
Sigma* = K** - K*^T ky^-1 K* inherits it on the scale of sf2.  The test asserts, per voxel,
max |Sigma* - ref| <= 8 u kappa(ky) sf2 and max |mu* - ref| <= 8 u kappa(ky) max|f - m| +
1e-6 m, with kappa computed here in FP64.  A well-conditioned batch (kappa ~ 1e3) makes
this a tight check of the implementation; the less conditioned ones show the bound holds
where FP32 loses digits (the diagonal-only mixed-precision solve is the accurate path).
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
U32 = 2.0 ** -24


@pytest.fixture(scope="module")
def gv():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2410_17084_b300 import build, gp_voxels
    build.build()
    return gp_voxels


def _solve(gv, b, max_points=None):
    import torch
    mp = int(max(b.counts.max(), b.tau)) if max_points is None else max_points
    cfg = gv.gp_voxels_config_default(voxel_size=b.size, grid_side=b.G, n_s=b.n_s, n_r=b.n_r,
                                      tau=b.tau, max_points=mp, max_voxels=b.nvox)
    g = gv.GpVoxels(cfg)
    d = gv.batch_to_device(b)
    Q = b.G * b.G
    axis = torch.empty(b.nvox, dtype=torch.uint8, device="cuda")
    mean = torch.full((b.nvox, Q), float("nan"), device="cuda")
    cov = torch.full((b.nvox, Q, Q), float("nan"), device="cuda")
    st = torch.empty(b.nvox, dtype=torch.int32, device="cuda")
    nmax = gv.gp_voxels_solve_alg3(g.h, d["xyz"], d["offsets"], b.nvox, d["centres"], d["lam"],
                                   d["sf2"], d["sn2"], axis, mean, cov, st)
    torch.cuda.synchronize()
    out = dict(axis=axis.cpu().numpy(), mean=mean.cpu().numpy(), cov=cov.cpu().numpy(),
               status=st.cpu().numpy().astype(np.uint32), nmax=nmax)
    g.close()
    return out


def _kappa(pts, axis, centre, lam, sf2, sn2):
    p1, p2 = {0: (1, 2), 1: (2, 0), 2: (0, 1)}[axis]
    X = np.stack([pts[:, p1].astype(np.float64) - centre[p1],
                  pts[:, p2].astype(np.float64) - centre[p2]], 1)
    K = sf2 * np.exp(-lam * ((X[:, None, :] - X[None, :, :]) ** 2).sum(-1))
    return float(np.linalg.cond(K + sn2 * np.eye(len(X))))


def _check(gv, oracle, b, label, expect_tight=None):
    from oracle import compare
    o = _solve(gv, b)
    worst_ratio, worst_abs, n = 0.0, 0.0, 0
    for v in range(b.nvox):
        pts = b.xyz[b.offsets[v]:b.offsets[v + 1]]
        st = int(o["status"][v])
        assert st == 0, f"{label} voxel {v}: status {st}"
        ax = int(o["axis"][v])
        ov = ax if compare.axis_ambiguous(pts) else -1
        r = oracle.solve_voxel_fullcov(pts, b.centres[v], b.size, b.G, float(b.lam[v]),
                                       float(b.sf2[v]), float(b.sn2[v]), 1, ov)
        assert r[0] == 0 and r[1] == ax
        kap = _kappa(pts, ax, b.centres[v].astype(np.float64), float(b.lam[v]),
                     float(b.sf2[v]), float(b.sn2[v]))
        bound = 8 * U32 * kap * float(b.sf2[v])
        f = pts[:, ax].astype(np.float64) - b.centres[v][ax]
        ec = float(np.abs(o["cov"][v] - r[3]).max())
        em = float(np.abs(o["mean"][v] - r[2]).max())
        assert ec <= bound, f"{label} voxel {v}: cov error {ec:.2e} > {bound:.2e} (kappa {kap:.1e})"
        assert em <= 8 * U32 * kap * np.abs(f - f.mean()).max() + 1e-6, f"{label} voxel {v}: mean"
        worst_ratio = max(worst_ratio, ec / bound)
        worst_abs = max(worst_abs, ec / float(b.sf2[v]))
        n += 1
    print(f"\n{label}: {n} voxels, worst cov error {worst_abs:.2e} sf2 = {worst_ratio:.3f} of bound")
    if expect_tight is not None:
        assert worst_abs <= expect_tight
    return o


def test_alg3_well_conditioned(gv, oracle):
    from paper_2410_17084_b300 import synth
    p = synth.plane_batch(1000, seed=0)
    b = p.subset(np.nonzero(p.counts <= 32)[0][:150])
    b.sn2[:] = 0.2 ** 2  # kappa ~ 1e2-1e3
    _check(gv, oracle, b, "plane sn 0.2", expect_tight=2e-4)


def test_alg3_less_conditioned(gv, oracle):
    from paper_2410_17084_b300 import synth
    p = synth.plane_batch(1000, seed=0)
    _check(gv, oracle, p.subset(np.arange(200)), "plane sn 0.02 (configs as the paper)")
    q = synth.quadric_batch(3000, seed=52)
    _check(gv, oracle, q.subset(np.nonzero(q.counts <= 112)[0][:40]), "quadric G16")


def test_alg3_large_grid_tiles(gv, oracle):
    """G = 32: Sigma* is 1024 x 1024 per voxel, 8 x 4 tensor-core tiles."""
    from paper_2410_17084_b300 import synth
    m = synth.mixed_batch(400, seed=53)
    b = m.subset(np.nonzero((m.counts <= 48) & ~m.degenerate)[0][:6])
    b.sn2[:] = 0.1 ** 2
    _check(gv, oracle, b, "G32")


def test_alg3_voxels_beyond_shared_memory(gv, oracle):
    """Voxels too large for one CTA's shared memory (ky in a global-memory slice, the
    persistent class of kernel A), up to 520 points at G = 9, against the oracle's full
    covariance within the same FP32 bound."""
    from paper_2410_17084_b300 import synth
    s = synth.stress_batch(20000, seed=55)
    pick = np.nonzero((s.counts >= 240) & (s.counts <= 520))[0]
    order = pick[np.argsort(s.counts[pick])]
    b = s.subset(order[np.linspace(0, order.size - 1, 10).astype(int)])
    b.sn2[:] = 0.1 ** 2  # kappa ~ 1e3-1e4: FP32 LU keeps a tight bound
    o = _check(gv, oracle, b, "beyond shared memory")
    assert o["nmax"] >= b.counts.max()


def test_alg3_unsolved_voxels_get_the_prior(gv):
    from paper_2410_17084_b300 import synth
    s = synth.stress_batch(3000, seed=54)
    small = np.nonzero(s.counts < 8)[0][:3]
    big = np.nonzero(s.counts > 600)[0][:2]
    ok = np.nonzero((s.counts >= 20) & (s.counts <= 40))[0][:3]
    b = s.subset(np.concatenate([small, big, ok]))
    b.tau = 8
    o = _solve(gv, b, max_points=560)
    assert o["nmax"] == 560 and b.counts[3:5].min() > 560
    st = o["status"]
    assert np.all(st[:3] == gv.VOX_BELOW_TAU) and np.all(st[3:5] == gv.VOX_TOO_LARGE)
    assert np.all(st[5:] == 0)
    G = b.G
    nd = -b.size / 2 + (np.arange(G) + 0.5) * b.size / G
    uu = np.repeat(nd, G)
    vv = np.tile(nd, G)
    for v in range(5):
        lam, sf2 = float(b.lam[v]), float(b.sf2[v])
        Kss = sf2 * np.exp(-lam * (uu[:, None] - uu[None, :]) ** 2) * np.exp(-lam * (vv[:, None] - vv[None, :]) ** 2)
        assert np.allclose(o["cov"][v], Kss, rtol=1e-5, atol=1e-7)
        assert np.all(o["mean"][v] == 0) and o["axis"][v] == 255
