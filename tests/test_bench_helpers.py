"""Host logic of bench.py: the roofline's algorithmic bytes and the guard on
the measured DRAM traffic (reported only for the kernel code it was taken
on)."""
import bench


def test_algorithmic_bytes_terms():
    n = 10
    cells = n * (n - 1) // 2
    sum_m = n * (n + 1) // 2 - 1
    updated = (n - 1) * (n - 2) // 2
    base = 4 * cells + 8 * n + 8 * sum_m + 12 * updated + 12 * (n - 1)
    b, note = bench.algorithmic_bytes(n, 1, None)
    assert b == base and "missing" in note
    b, _ = bench.algorithmic_bytes(n, 1, {"rescan_cells": 7})
    assert b == base + 28
    b, _ = bench.algorithmic_bytes(n, 1, {"rescan_cells": 7, "rowi_cells": 5})
    assert b == base + 28 + 20  # the merged rows' recomputed minima
    b, _ = bench.algorithmic_bytes(n, 3, {"rescan_cells": 0})
    assert b == base + 4 * sum_m  # Ward also reads the sizes


def test_traffic_only_for_the_measured_workload_and_code():
    assert bench.measured_traffic("gmm16384q", 1) is None
    assert bench.measured_traffic("conformer65536", 3) is None
    v = bench.measured_traffic("conformer65536", 1)
    same = bench.kernel_source_sha256() == bench.MEASURED_TRAFFIC["kernel_sha256"]
    assert (v == bench.MEASURED_TRAFFIC["bytes_per_launch"]) if same else v is None


def test_kernel_hash_ignores_comments(tmp_path, monkeypatch):
    import os
    src = tmp_path / "paper_1709_06816_gb300" / "csrc"
    src.mkdir(parents=True)
    (src / "lw_merge.cu").write_text("int a = 1;  // one\n// note\n\nint b = 2;\n")
    (src / "lw_internal.h").write_text("#pragma once\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h1 = bench.kernel_source_sha256()
    (src / "lw_merge.cu").write_text("int a = 1;  // another note\nint b = 2;  // two\n")
    assert bench.kernel_source_sha256() == h1
    (src / "lw_merge.cu").write_text("int a = 1;\nint b = 3;\n")
    assert bench.kernel_source_sha256() != h1
