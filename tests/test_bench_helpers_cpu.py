"""bench.py's roofline and option helpers on synthetic per-solve statistics:
the roofline objects carry the keys the JSON line needs and their
fractions follow from the stated work, time and peak.  CPU only."""

import types

import pytest

import bench

PK = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}
KEYS = {"bound", "achieved", "peak", "unit", "frac", "traffic"}


def stats(**kw):
    base = {"flops_filter": 0.0, "t_filter": 0.0, "flops_rr_product": 0.0, "t_rr_product": 0.0,
            "lanczos_matvecs": 0, "t_lanczos": 0.0}
    base.update(kw)
    return base


def test_split_filter_roofline_counts_28_slice_pairs():
    s = [stats(flops_filter=4.0e13, t_filter=1.0)]  # 40 TFLOP/s FP64-equivalent
    main, other = bench.roofline_entry(s, PK, "measured", "split_rr")
    assert KEYS <= set(main)
    assert main["fp64_equivalent_tflops"] == pytest.approx(40.0)
    assert main["achieved"] == pytest.approx(28 * 40.0)
    assert main["frac"] == pytest.approx(28 * 40.0 / 1700.0, rel=1e-3)
    assert other["kernel"].startswith("zgemm_split_kernel")


def test_fp64_rr_product_is_dominant_when_it_takes_longer():
    # H Q: 1.3e12 algorithmic FLOPs in 1 s, filter 0.5 s
    s = [stats(flops_filter=2.0e13, t_filter=0.5, flops_rr_product=1.3e12, t_rr_product=1.0)]
    main, other = bench.roofline_entry(s, PK, "measured", "split")
    assert main["kernel"].startswith("zgemm_tma_kernel")
    peak = 1900.0 * 1.25 / 2250.0
    assert main["peak"] == pytest.approx(peak, rel=1e-3)
    assert main["achieved"] == pytest.approx(0.75 * 1.3, rel=1e-3)  # 3M: 6 of 8 FLOPs executed
    assert main["frac"] == pytest.approx(0.75 * 1.3 / peak, rel=1e-3)
    assert other["kernel"].startswith("zgemm_split_kernel")


def test_fp64_filter_roofline():
    s = [stats(flops_filter=1.35e12, t_filter=1.0)]
    main, other = bench.roofline_entry(s, PK, "fallback", "fp64")
    assert other is None and KEYS <= set(main)
    assert main["algorithmic_tflops"] == pytest.approx(1.35)
    assert "fallback" in main["peak_source"]


def test_lanczos_entry_rates():
    n = 8000
    s = [stats(lanczos_matvecs=25, t_lanczos=0.0142)]
    e = bench.lanczos_entry(s, n, PK, "measured")
    flops = 8.0 * n * n * 25
    assert e["achieved"] == pytest.approx(flops / 0.0142 / 1e12, rel=1e-3)
    assert e["hbm_gbs"] == pytest.approx(16.0 * n * n * 25 / 0.0142 / 1e9, rel=1e-3)
    assert bench.lanczos_entry([stats()], n, PK, "measured") is None


def test_deg_extra_defaults():
    from paper_1805_10121_gb300 import chase
    args = types.SimpleNamespace(deg_extra=None)
    assert bench.deg_extra_for(args, chase.CHASE_FP64) == 2
    assert bench.deg_extra_for(args, chase.CHASE_SPLIT_BF16) == bench.SPLIT_DEG_EXTRA
    assert bench.deg_extra_for(types.SimpleNamespace(deg_extra=4), chase.CHASE_FP64) == 4


def test_split_algorithmic_bytes_per_launch():
    # one K segment of the N = 30000 filter: 7 slice planes of H (30000 rows)
    # and of the block (3000 real rows) over K = 30000, and the FP64 result
    n, b, k = 30000, 1500, 30000
    got = bench.split_algorithmic_bytes(n, b, k)
    assert got == pytest.approx(7 * 2 * (30000 + 3000) * 30000 + 16 * 30000 * 1500)


def test_blas_threads_round_trip():
    import numpy as np
    a = np.ones((64, 64))
    a @ a  # load the BLAS
    bt = bench.BlasThreads(1)
    if not bt.ok:
        pytest.skip("no OpenBLAS thread control in this NumPy")
    before = int(bt.get_fn()) if bt.get_fn else None
    with bt:
        if bt.get_fn:
            assert int(bt.get_fn()) == 1
    if bt.get_fn:
        assert int(bt.get_fn()) == before


def test_degree_caps_by_precision():
    # DEGMAX 64 with a split filter, Table 1's 36 with FP64; --deg-max wins
    from paper_1805_10121_gb300 import chase
    args = types.SimpleNamespace(deg_max=None, deg_extra=None)
    assert bench.deg_max_for(args, chase.CHASE_SPLIT_BF16) == bench.SPLIT_DEG_MAX == 64
    assert bench.deg_max_for(args, chase.CHASE_FP64) == chase.chase_opts_default().deg_max == 36
    assert bench.deg_extra_for(args, chase.CHASE_FP64) == 2
    assert bench.deg_extra_for(args, chase.CHASE_SPLIT_BF16) == bench.SPLIT_DEG_EXTRA
    args = types.SimpleNamespace(deg_max=48, deg_extra=4)
    assert bench.deg_max_for(args, chase.CHASE_FP64) == 48
    assert bench.deg_extra_for(args, chase.CHASE_SPLIT_BF16) == 4
