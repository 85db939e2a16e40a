"""Host-side accounting of the benchmark line (no GPU): the algorithmic work per voxel that
the roofline divides by, its split between the tensor cores and the CUDA cores, and the
oracle's per-workload rate.

Mistakes each test is meant to catch: a dropped term of the per-voxel count (n^3/3 for the
Cholesky, n^2 G^2 for the triangular solve behind the variance, 4 n G^2 for the mean and
the variance norms, 4 n^2 for the alpha solves), a voxel counted on both units or on none,
the tall-matrix threshold applied with the wrong inequality, and a per-workload rate that
divides by the wrong sample size."""
import types

import numpy as np
import pytest


def test_algorithmic_flops_closed_form():
    import bench
    n, G = np.array([1, 8, 64, 1024]), 9
    expect = n ** 3 / 3 + n ** 2 * 81 + 4 * n * 81 + 4 * n ** 2
    assert np.allclose(bench.algorithmic_flops(n, G), expect, rtol=0, atol=1e-6)
    # the 512-point voxel of the tall-matrix capture: 67.2 MFLOP
    assert bench.algorithmic_flops(np.array([512]), 9)[0] == pytest.approx(67.19e6, rel=1e-3)


def test_split_flops_partitions_the_work():
    import bench
    rng = np.random.default_rng(0)
    counts = rng.integers(4, 1025, 5000)
    plan = {"tall_min": 128, "tc_nmax": 224}
    fl = bench.split_flops(counts, 9, plan)
    assert fl["tc"] + fl["ff"] == pytest.approx(fl["total"], rel=1e-12)
    tall = counts > 128
    assert fl["tall_voxels"] == int(tall.sum())
    assert fl["tall_total"] == pytest.approx(bench.algorithmic_flops(counts[tall], 9).sum(),
                                             rel=1e-12)
    assert fl["tall_tc"] + fl["tall_ff"] == pytest.approx(fl["tall_total"], rel=1e-12)
    # shared-memory voxels: only the variance contraction n^2 G^2 on the tensor cores
    small = counts[~tall].astype(np.float64)
    assert fl["tc"] - fl["tall_tc"] == pytest.approx((small ** 2 * 81).sum(), rel=1e-12)
    # a voxel of exactly tall_min points stays on the shared-memory kernels
    one = bench.split_flops(np.array([128]), 9, plan)
    assert one["tall_voxels"] == 0
    # the in-panel work of a tall voxel: 32 flops per row and column of the padded matrix
    big = bench.split_flops(np.array([300]), 9, plan)
    npad = 320.0
    assert big["tall_ff"] == pytest.approx(32.0 * (npad + 81) * npad, rel=1e-12)


def test_split_flops_without_tall_path():
    import bench
    counts = np.array([10, 100, 200, 300])
    fl = bench.split_flops(counts, 16, {"tall_min": 0, "tc_nmax": 224})
    assert fl["tall_voxels"] == 0 and fl["tall_total"] == 0.0
    # the 300-point voxel is beyond the tensor-core variance: all of it on the CUDA cores
    tc = (np.array([10, 100, 200], np.float64) ** 2 * 256).sum()
    assert fl["tc"] == pytest.approx(tc, rel=1e-12)


def test_oracle_per_config_rates():
    import bench
    fake5 = types.SimpleNamespace(idx=np.arange(2000), seconds=4.0)
    ex = {"quadric50k": {"oracle_seconds": 2.0}, "mixed200k": {"oracle_seconds": 8.0}}
    r = bench.oracle_per_config(ex, fake5)["configs"]
    assert r["plane1k"]["voxels"] == 1000 and r["plane1k"]["value"] > 0
    assert r["quadric50k"]["value"] == pytest.approx(bench.ERR_SAMPLE / 2.0)
    assert r["mixed200k"]["value"] == pytest.approx(bench.ERR_SAMPLE / 8.0)
    assert r["stress1m"]["value"] == pytest.approx(500.0)
    # legs that did not run are left out, not reported as zero
    assert set(bench.oracle_per_config({}, None)["configs"]) == {"plane1k"}
