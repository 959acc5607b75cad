"""Host arithmetic of bench.py that feeds the reported numbers (no GPU):
the algorithmic flops and bytes behind roofline.achieved, the G difference
reported for every reduced-precision form, and the lookup of the committed
ncu traffic record."""
import json
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_setup_flops_and_bytes_by_hand():
    # row 0 keeps P = {0} (no step); row 1 grows 1 -> 2 -> 3 entries (s = 1)
    rowptr_G = np.array([0, 1, 4])
    steps = np.array([0, 2])
    flops = bench.setup_flops(rowptr_G, steps, 1, 5.0)
    # step 1: m = 2, |P_0| = 1: 8/3 + 2*4 + 2*5*1; step 2: m = 3, |P_1| = 2: 27/3 + 2*9 + 2*5*2
    assert flops == pytest.approx(8 / 3 + 8 + 10 + 9 + 18 + 20)
    touched = bench.setup_touched_bytes(rowptr_G, steps, 1, 5.0)
    # G rows written: 4 entries x 12 B; step 1 reads 1 + 1 rows of A, step 2 reads 2 + 1,
    # each 12 B x 5 entries + 8 B of row pointers
    assert touched == pytest.approx(4 * 12 + (2 + 3) * (12 * 5 + 8))


def test_spmv_and_pcg_bytes():
    assert bench.spmv_bytes(10, 30) == 30 * 12 + 4 * 11 + 10 * 8 + 10 * 8
    assert bench.spmv_bytes(10, 30, val_bytes=4, x_bytes=8, y_bytes=4) == 30 * 8 + 4 * 11 + 80 + 40

    class A:
        n, nnz = 100, 700

    fp64 = bench.pcg_iteration_bytes(A, {"nnz_G": 400}, "fp64")
    mixed = bench.pcg_iteration_bytes(A, {"nnz_G": 400}, "mixed")
    assert fp64 == 12 * 700 + 2 * 12 * 400 + 12 * 100 + 140 * 100
    assert fp64 - mixed == 2 * 4 * 400  # FP32 G saves 4 B per entry of G and G^T


def _lower(n, rng):
    rp, ci, va = [0], [], []
    for i in range(n):
        cols = sorted(set(rng.choice(i + 1, size=min(i + 1, 3), replace=False).tolist()) | {i})
        ci += cols
        va += rng.uniform(0.5, 1.5, size=len(cols)).tolist()
        rp.append(len(ci))
    return np.array(rp), np.array(ci), np.array(va)


def test_g_difference():
    rng = np.random.default_rng(3)
    n = 50
    rp, ci, va = _lower(n, rng)
    same = bench.g_difference((rp, ci, va), (rp, ci, va.copy()), n)
    assert same == {"rel_frobenius": 0.0, "max_rel_same_pattern_rows": 0.0, "rows_same_pattern": 1.0}
    # one value off by 1e-3 (relative)
    v2 = va.copy()
    v2[7] *= 1.0 + 1e-3
    d = bench.g_difference((rp, ci, va), (rp, ci, v2), n)
    assert d["max_rel_same_pattern_rows"] == pytest.approx(1e-3, rel=1e-9)
    assert d["rel_frobenius"] == pytest.approx(abs(va[7]) * 1e-3 / np.linalg.norm(va), rel=1e-9)
    assert d["rows_same_pattern"] == 1.0
    # one row with another pattern (same length): it leaves the entrywise comparison
    i = 20  # at least one off-diagonal entry (3 drawn columns plus the diagonal)
    b, e = rp[i], rp[i + 1]
    assert e - b >= 2 and ci[b] < i
    free = sorted(set(range(i)) - set(ci[b:e].tolist()))
    c2 = ci.copy()
    c2[b] = free[0]
    c2[b:e] = np.sort(c2[b:e])
    d = bench.g_difference((rp, ci, va), (rp, c2, va), n)
    assert d["rows_same_pattern"] == pytest.approx((n - 1) / n)
    assert d["max_rel_same_pattern_rows"] == 0.0
    assert d["rel_frobenius"] > 0.0


def test_measured_traffic_follows_the_source_digest(tmp_path, monkeypatch):
    src = os.path.join("tests", "conftest.py")
    rec = {"k": {"dram_bytes": 1000.0, "units": 10, "capture": "test", "sources": [src],
                 "source_digest": bench.source_digest([src])}}
    f = tmp_path / "traffic.json"
    f.write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(f))
    v, note = bench.measured_traffic("k", 25)
    assert v == pytest.approx(2500.0) and "scaled" in note
    rec["k"]["source_digest"] = "0" * 16
    f.write_text(json.dumps(rec))
    assert bench.measured_traffic("k", 25) == (None, "kernel changed since the ncu capture")
    assert bench.measured_traffic("absent", 25) == (None, "no ncu record")


def test_pcg_kernel_table_bounds():
    class A:
        n, nnz = 1000, 7000

    # FP64 G: the G SpMV moves 12 B per entry for one FP64 fma; at the
    # measured bandwidth and the derived FP64 rate the bytes bind
    t = bench.pcg_kernel_table(A, 10000, "fp64", [0.1, 0.02, 0.1, 0.1, 0.02])
    g = [k for k in t if k["key"] == "pcg_G"][0]
    assert g["bytes"] == 12 * 10000 + 4 * 1001 + 16 * 1000 and g["dfma"] == 10000
    assert g["bound"] == "hbm"
    assert g["achieved"] == pytest.approx(g["bytes"] / 1e-4 / 1e9)
    assert g["frac"] == pytest.approx(g["achieved"] / bench.MEASURED_HBM_GBS)
    # FP32 G: 8 B per entry, no FP64 fma in the product
    t32 = bench.pcg_kernel_table(A, 10000, "mixed", [0.1] * 5)
    g32 = [k for k in t32 if k["key"] == "pcg_G"][0]
    assert g32["bytes"] == 8 * 10000 + 4 * 1001 + 16 * 1000 and g32["dfma"] == 0
