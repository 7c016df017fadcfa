"""Host-side logic that needs no GPU: the batched form's size classes, the autotuner's cache key,
the benchmark's op counting and its traffic record's source check."""
import hashlib
import json
import os

import pytest

import bench
from paper_2604_16725_gb300.batched import class_sizes
from paper_2604_16725_gb300.tune import signature


def test_class_sizes_cover_and_bound_padding():
    s = class_sizes(8, 22)
    assert s == sorted(set(s)) and s[0] == 256 and s[-1] == 1 << 22
    assert all(x % 256 == 0 for x in s)
    worst = {1024: 0.0, 8192: 0.0}
    j = 0
    for n in range(1, (1 << 22) + 1, 13):
        while s[j] < n:
            j += 1
        pad = (s[j] - n) / s[j]
        for lo in worst:
            if n >= lo:
                worst[lo] = max(worst[lo], pad)
    assert worst[1024] < 0.20 and worst[8192] < 0.18
    assert len([x for x in s if 1 << 12 <= x < 1 << 13]) == 4    # four classes per power of two


def test_tune_signature():
    a = signature(64, 1 << 20, [512, 256, 4096], (0.6, 0.15, 0.05, 0.1, 0.1))
    assert a == signature(64, 1 << 20, [4096, 512, 256], (0.6, 0.15, 0.05, 0.1, 0.1))   # order of sizes
    assert a != signature(32, 1 << 20, [512, 256, 4096], (0.6, 0.15, 0.05, 0.1, 0.1))
    assert a != signature(64, 1 << 21, [512, 256, 4096], (0.6, 0.15, 0.05, 0.1, 0.1))
    assert a != signature(64, 1 << 20, [512, 256, 4096], (0.5, 0.25, 0.05, 0.1, 0.1))


def test_bench_op_counts():
    ops = bench.ops_per_step(log_q=24, log_r=18, log_u=20)
    assert ops == dict(lookup=1 << 24, successor=1 << 24, range=1 << 18, insert=1 << 20, delete=1 << 20)
    n = sum(ops.values())
    assert bench.whole_job_mops(n, 1, 5.0) == pytest.approx(n / 5e-3 / 1e6)
    assert bench.whole_job_mops(n, 4, 5.0) == pytest.approx(4 * n / 5e-3 / 1e6)     # every rank's ops
    assert bench.max_over_ranks(3.5, 1) == 3.5


def test_traffic_record_follows_the_marked_source(tmp_path, monkeypatch):
    src_dir = tmp_path / "paper_2604_16725_gb300" / "csrc"
    src_dir.mkdir(parents=True)
    (tmp_path / "profiles").mkdir()
    head, body, tail = "// header\n", "namespace flix {\nint pass_kernel;\n", "// ---- pass plan\nint plan;\n"
    (src_dir / "flix_sort.cu").write_text(head + body + tail)
    rec = {"sort_onesweep": {"dram_bytes_per_item": 20.0, "items_per_launch": 16, "source": "flix_sort.cu",
                             "from": "namespace flix {", "until": "// ---- pass plan",
                             "sha256": hashlib.sha256(body.encode()).hexdigest()}}
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.traffic_record("sort_onesweep")["dram_bytes_per_item"] == 20.0
    # edits outside the marked region keep the record; an edit inside it voids the record
    (src_dir / "flix_sort.cu").write_text("// other header\n" + body + tail + "int more;\n")
    assert bench.traffic_record("sort_onesweep") is not None
    (src_dir / "flix_sort.cu").write_text(head + body.replace("pass_kernel", "pass_kernel2") + tail)
    assert bench.traffic_record("sort_onesweep") is None
    assert bench.traffic_record("no_such_kernel") is None


def test_algorithmic_bytes_and_fractions():
    """The bench line's algorithmic bytes per step follow the kernel table's formulas (uint64 keys
    and values, node size 64, half-full nodes), and a kernel's fraction is bytes / time / peak."""
    by = bench.step_bytes(rcap=1000, log_load=12, log_q=10, log_r=4, log_u=6)
    n, B, R, U, ks, h = 1 << 12, 1 << 10, 1 << 4, 1 << 6, 8, 32
    nb = n // h
    assert by["gather"] == n * 2 * (ks + ks)
    assert by["sort_hist"] == (2 * B + R + 2 * U) * ks
    # windowed delivery: tag written with the result, then (tag, result) read and the result written,
    # for lookups (8-byte values) and successors (8-byte keys and values)
    assert by["read_unsort"] == (B * 4 + B * (4 + 8) + B * 8) + (B * 4 + B * (4 + 16) + B * 16)
    assert by["range_fill"] == 1000 * 2 * (ks + ks) + R * (4 + 12 + 16)
    assert by["partition"] == 2 * (nb * ks + B * ks + 4 * B) + (nb * ks + R * ks + 4 * R) + 2 * (nb * ks + U * ks + 4 * nb)
    prof = {"gather": {"ms": 2.0, "launches": 2, "bytes": 0.0}}
    out = bench.apply_rooflines(prof, 2, 1000.0, "measured", rcap=1000)
    g = out["gather"]
    assert g["ms_per_step"] == 1.0 and g["frac"] == pytest.approx(g["achieved"] / 1000.0, abs=1e-3)
    assert g["achieved"] == pytest.approx(bench.step_bytes(1000)["gather"] / 1e-3 / 1e9, abs=0.1)   # rounded to 0.1
