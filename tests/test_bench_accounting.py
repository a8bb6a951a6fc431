"""CPU checks of bench.py's accounting, which turns measured times into
roofline fractions: the algorithmic bytes and flops per COCG iteration
against the per-mode formulas written out here term by term, the band-block
count of the block incomplete Cholesky mode against a count over the
oracle's band split, and the recorded DRAM traffic, which is used only while
the solve kernel's sources are unchanged."""
import importlib.util
from pathlib import Path

import numpy as np
import pytest

from oracle import fem, precond
from paper_0704_2344_gb300 import workloads as W

ROOT = Path(__file__).resolve().parents[1]

INFO = {"nnzb": 1000, "n_nodes": 50, "n_dof": 150}
SYS = {"nnzb": 1000, "blocks_explicit": 400, "rows_general": 3, "rows_diagonal": 20}


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", ROOT / "bench.py")
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_fp64_iteration_bytes(bench):
    # every stored block (9 complex128 + a column index), row pointers; per dof and
    # column: u in, w out, r and u for the dots, u p s x r and w in, p s x r u out,
    # the block-Jacobi row
    per_dof = 16 + 16 + 2 * 16 + 5 * 16 + 16 + 5 * 16 + 3 * 16
    assert per_dof == 288
    for R in (1, 2, 8):
        _, inner, outer = bench.algorithmic_bytes(INFO, SYS, "fp64", 1, 0, R=R)
        assert inner == 1000 * (9 * 16 + 4) + 51 * 4 + 150 * R * per_dof
        assert outer == 1000 * (9 * 16 + 4) + 51 * 4 + 150 * R * 240


def test_complex64_iteration_bytes(bench):
    # explicit blocks only, 27 column indices per stencil row, and the complex64 copy of u
    per_dof = 8 + 8 + 2 * 16 + 5 * 16 + 8 + 5 * 16 + 8 + 3 * 16
    assert per_dof == 272
    _, inner, outer = bench.algorithmic_bytes(INFO, SYS, "mixed", 1, 0, R=1)
    assert inner == 400 * (9 * 8 + 4) + 23 * 27 * 4 + 51 * 4 + 150 * per_dof
    assert outer == 1000 * (9 * 16 + 4) + 51 * 4 + 150 * (240 + 8)
    total, inner, outer = bench.algorithmic_bytes(INFO, SYS, "df", 7, 2, R=1)
    assert total == 7 * inner + 2 * outer


def test_iteration_flops(bench):
    prod, f64 = bench.algorithmic_flops(INFO, SYS, "fp64", 1, 0, R=4)
    assert prod == 72 * 1000 * 4 and f64 == 76 * 150 * 4
    prod, _ = bench.algorithmic_flops(INFO, SYS, "df", 1, 0, R=1)
    assert prod == 60 * (9 * 400 + 27 * 9 * 3 + 27 * 1.5 * 20)
    _, f64 = bench.algorithmic_flops(INFO, SYS, "mixed", 0, 3, R=2)
    assert f64 == 3 * (72 * 1000 * 2 + 34 * 150 * 2)


@pytest.mark.parametrize("n_band", [1, 3, 17, "per_node"])
def test_bicp_band_blocks(bench, n_band):
    prob = W.random_small_grid(6, n_max=7, n_pec_boxes=2)
    maps = fem.mesh_maps(prob)
    S = maps.n_act if n_band == "per_node" else n_band
    band = precond.node_subdomain(maps.n_act, S)
    count = 0
    for I in range(maps.n_act):
        for J in maps.col_idx[maps.row_ptr[I]:maps.row_ptr[I + 1]]:
            count += int(J < I and band[J] == band[I])
    assert bench.bicp_band_blocks(maps.row_ptr, maps.col_idx, S) == count
    if S == maps.n_act:
        assert count == 0


def test_recorded_traffic_follows_the_kernel_sources(bench, monkeypatch):
    text = (ROOT / "profiles" / "k_solve_config2_traffic.txt").read_text()
    recorded = next(l.split("=", 1)[1].strip() for l in text.splitlines() if l.startswith("kernel_hash="))
    monkeypatch.setattr(bench, "kernel_hash", lambda: recorded)   # the sources as captured
    for mode in ("fp64", "mixed", "df", "fp64_bicp"):
        t = bench.recorded_traffic("config2", mode)
        assert isinstance(t, int) and t > 0, mode
    assert bench.recorded_traffic("config3", "df") is None
    monkeypatch.setattr(bench, "kernel_hash", lambda: "0" * 16)
    assert bench.recorded_traffic("config2", "df") is None


def test_method_bytes_per_product_match_the_worked_figures(bench):
    # Worked figures for the 3-wavelength cube (748 658 blocks,
    # 29 666 nodes, 88 998 unknowns), one column: 58.4 MB per complex64
    # product and 113.8 MB per complex128 (or FP32-pair) product.
    c2 = {"nnzb": 748658, "n_nodes": 29666, "n_dof": 88998}
    assert bench.product_bytes(c2, 8, 1) == 748658 * 76 + 29667 * 4 + 2 * 88998 * 8
    assert round(bench.product_bytes(c2, 8, 1) / 1e6, 1) == 58.4
    assert round(bench.product_bytes(c2, 16, 1) / 1e6, 1) == 113.8
    # R columns: the vectors scale, the matrix does not
    assert bench.product_bytes(c2, 8, 32) - bench.product_bytes(c2, 8, 1) == 2 * 88998 * 8 * 31


def test_method_products_count_the_slowest_column_of_each_launch(bench):
    rep = [{"iterations": 10, "outer": 3}, {"iterations": 12, "outer": 2},
           {"iterations": 7, "outer": 2}, {"iterations": 9, "outer": 4}]
    # two launches of two columns: 12 + (3 - 2) and 9 + (4 - 2) inner products;
    # 3 + 4 true-residual products
    assert bench.method_products(rep, 2) == (12 + 1 + 9 + 2, 3 + 4)
    # one column per launch: a column with two passes has no intermediate refresh
    assert bench.method_products(rep[:1], 1) == (10 + 1, 3)
    assert bench.method_products(rep[1:2], 1) == (12, 2)


def test_reference_arm_reports_the_time_it_ran(bench, capsys):
    """The reference arm times bounded samples of the oracle's solve: its
    line's rate is the solves those samples did over the time they ran, so
    rate, solves per step and time per step agree, and the time it claims
    fits in the time the call took."""
    import argparse
    import json
    args = argparse.Namespace(workload="config2", cpu_sample_s=3.0, steps=2, warmup=0, gpus=1)
    bench.run_reference(args)
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["value"] == pytest.approx(line["solves_per_step"] * 1e3 / line["ms_per_step"], rel=1e-3)
    assert line["ms_per_step"] * line["steps"] <= 1e3 * line["wall_s"]
    assert line["config"]["workload"].startswith("config2: ") and "88998 unknowns" in line["config"]["workload"]
