"""Host logic of bench.py (no GPU): algorithmic bytes per step and the keys of the committed
ncu traffic table."""
import argparse
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

INFO = {"grid_x": 1000, "grid_k": 1012, "n_xi": 50_000, "n_records": 25_000, "nnz": 2_000_000, "stencil_x": 8}


def test_spmv_bytes_follow_the_stored_value_type():
    n = 10_000
    fp32 = bench.stage_bytes(INFO, n, 1, "fp32", esz=8)["spmv"]
    fp64 = bench.stage_bytes(INFO, n, 1, "fp64", esz=8)["spmv"]
    near32 = bench.stage_bytes(INFO, n, 1, "fp32", esz=8, near32=True)["spmv"]
    # D is float64 in both forms (column index 4 B + value 8 B per non-zero); the
    # float32-D flag stores 4 B values
    assert fp64 == fp32 == 12 * INFO["nnz"] + 8 * (n + 1) + 2 * 8 * n
    assert fp32 - near32 == 4 * INFO["nnz"]
    helm32 = bench.stage_bytes(INFO, n, 1, "fp32", esz=16, near32=True)["spmv"]
    assert helm32 == (4 + 8) * INFO["nnz"] + 8 * (n + 1) + 2 * 16 * n
    helm = bench.stage_bytes(INFO, n, 1, "fp32", esz=16)["spmv"]
    assert helm == (4 + 16) * INFO["nnz"] + 8 * (n + 1) + 2 * 16 * n


def test_laplace_steps_count_half_the_grid_and_no_node_data():
    """The node step moves a read and a write of the half plane's cells; node data counts 0 (the
    nodes are a function of (p, m)); the stored records it streams are reported apart."""
    b = bench.stage_bytes(INFO, 10_000, 1, "fp32", esz=8)
    m, nk = INFO["grid_x"], INFO["grid_k"]
    assert b["node"] == 8 * nk * nk
    assert bench.stage_bytes(INFO, 10_000, 1, "fp32", esz=16)["node"] == 2 * 8 * nk * nk
    assert bench.node_records_bytes(INFO, "fp32") == 24 * INFO["n_records"]
    assert b["fft_fwd"] == 8 * (m * m // 2 + nk * nk // 2)
    assert b["spread"] == 16 * 10_000 + 8 * 10_000 + 8 * m * m // 2


def test_traffic_keys_name_size_and_alpha():
    a = argparse.Namespace(workload="laplace_curves", n=1_000_000, nrhs=1)
    assert bench.traffic_key(a, 0.0) == "laplace_curves"
    assert bench.traffic_key(a, 0.125) == "laplace_curves_alpha0.125"
    a.n = 300_000
    assert bench.traffic_key(a, 0.0) == "laplace_curves_n300000_rhs1"
    assert bench.traffic_for("node", "no_such_workload", "fp32") is None


def test_step_bytes_scale_with_right_hand_sides():
    one = bench.stage_bytes(INFO, 10_000, 1, "fp32", esz=8)
    four = bench.stage_bytes(INFO, 10_000, 4, "fp32", esz=8)
    for st in ("fft_fwd", "fft_inv", "sum", "node"):
        assert four[st] == 4 * one[st]
    # the point records are read once per launch, the grids and values once per right-hand side
    assert four["spread"] - 16 * 10_000 == 4 * (one["spread"] - 16 * 10_000)
