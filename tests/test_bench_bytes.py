"""The algorithmic byte counts behind the bench line's roofline fractions,
checked against counts written out by hand for small cases, and the
roofline traffic figure against the capture it is scaled from."""
import importlib.util
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_spmv_bytes_by_hand(bench):
    # 3 block rows, 7 blocks: values 7 x 32, columns 7 x 4, row pointers 4 x 4,
    # x read and y written 3 x (16 + 16)
    assert bench.spmv_bytes(3, 7) == 224 + 28 + 16 + 96
    # the two sizes of the roofline capture and of the bench (block rows and
    # blocks of the 200x200x20 and 200x200x50 fields)
    assert bench.spmv_bytes(1600025, 7905025) == 342181804
    assert bench.spmv_bytes(4000025, 19882525) == 859771804


def test_roofline_traffic_is_the_capture_scaled(bench):
    t = bench.TIMED_TRAFFIC[(200, 200, 50, 0)]
    captured = 316643072 + 21299968
    assert t == round(captured * bench.spmv_bytes(4000025, 19882525)
                      / bench.spmv_bytes(1600025, 7905025))
    assert 0.95 < t / bench.spmv_bytes(4000025, 19882525) < 1.0


def test_sweep_bytes_by_hand(bench):
    # 4 block rows, 10 blocks: (10 - 4) / 2 = 3 L and 3 U blocks; level 0 with
    # 10 entries; the first colour 2 rows and 3 entries
    b = bench.sweep_bytes(4, 10, 2, 3, first_fused=True)
    assert b["k_ilu_fwd"] == 20 * 3 + 44 * 4
    assert b["k_ilu_bwd"] == 20 * 3 + 52 * 4
    post = 8 * 10 + 24 * 4
    pre_fused = post - 8 * 3 - 24 * 2
    assert b["k_gs_c"] == (pre_fused + post) // 2
    b = bench.sweep_bytes(4, 10, 2, 3, first_fused=False)
    assert b["k_gs_c"] == (post - 8 * 3 - 12 * 2 + post) // 2


def test_coarse_cycle_bytes_by_hand(bench):
    levels = [dict(n=100, nnz=500, nagg=10, p_nnz=200, smoother=0),
              dict(n=10, nnz=60, nagg=3, p_nnz=20, smoother=1),
              dict(n=3, nnz=9, nagg=0, p_nnz=0, smoother=2)]
    # level 1 (FP32 values: 8 B an entry): two smoothings, restriction, prolongation
    smooth = 2 * (8 * 60 + 4 * 11 + 16 * 10)
    restrict = 8 * 20 + 4 * 4 + 4 * 10 + 4 * 3
    prolong = 8 * 20 + 4 * 11 + 4 * 3 + 8 * 10
    # level 2: the dense FP64 inverse and b, x
    coarsest = 8 * 9 + 8 * 3
    assert bench.coarse_cycle_bytes(levels, 1) == smooth + restrict + prolong + coarsest
    # BF16 values (6 B an entry) on level 1 with precision 2
    smooth2 = 2 * (6 * 60 + 4 * 11 + 16 * 10)
    restrict2 = 6 * 20 + 4 * 4 + 4 * 10 + 4 * 3
    prolong2 = 6 * 20 + 4 * 11 + 4 * 3 + 8 * 10
    assert bench.coarse_cycle_bytes(levels, 2) == smooth2 + restrict2 + prolong2 + coarsest
    # a smoothed coarsest level: its two sweeps
    levels[2]["smoother"] = 1
    assert (bench.coarse_cycle_bytes(levels, 1)
            == smooth + restrict + prolong + 2 * (8 * 9 + 4 * 4 + 16 * 3))


def test_assembly_bytes_by_hand(bench):
    assert bench.assembly_bytes(5, 13, 4) == 44 * 13 + 56 * 4 + 24 * 5


def test_spmv_fp64_side(bench):
    r = bench.spmv_fp64(19882525, 0.1515)
    assert r["flops_per_launch"] == 8 * 19882525
    assert abs(r["achieved_tflops"] - 8 * 19882525 / 0.1515e-3 / 1e12) < 1e-12
    assert 0.8 < r["frac"] < 0.95
