"""Host-side logic of the benchmark and the autotuner, on the CPU: the kernel
source digest that keys recorded profiles, the lookup of recorded DRAM
traffic, the path roofline arithmetic, and the autotuner's candidate list."""

import json
import os
import shutil

import pytest

import bench
from paper_2401_02756_gb300 import autotune

CSRC = ("dbg_insert.cu", "dbg_binned.cu", "dbg_binned.cuh", "dbg_tiles.cuh", "dbg_internal.cuh",
        "dbg_tma.cuh")


@pytest.fixture
def tree(tmp_path, monkeypatch):
    """A copy of the kernel sources under a temporary root."""
    src = os.path.join(bench.ROOT, "paper_2401_02756_gb300", "csrc")
    dst = tmp_path / "paper_2401_02756_gb300" / "csrc"
    dst.mkdir(parents=True)
    for f in CSRC:
        shutil.copy(os.path.join(src, f), dst / f)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    return dst


def test_digest_ignores_comments_and_blank_lines_only(tree):
    d0 = bench.kernel_source_digest()
    p = tree / "dbg_binned.cu"
    text = p.read_text()
    p.write_text("// a new comment line\n\n" + text.replace("\n", "  // trailing note\n", 3))
    assert bench.kernel_source_digest() == d0
    p.write_text(text.replace("kTiledShift = 21", "kTiledShift = 20"))
    assert bench.kernel_source_digest() != d0


def test_recorded_traffic_needs_the_same_kernels(tree, tmp_path):
    prof = tmp_path / "profiles"
    prof.mkdir()
    rec = {"wl": {"bin_apply": {"dram_bytes_per_launch": 123, "kernel_source_digest": "x"}}}
    (prof / "insert_traffic.json").write_text(json.dumps(rec))
    assert bench.recorded_traffic("wl", "bin_apply") is None  # another digest
    rec["wl"]["bin_apply"]["kernel_source_digest"] = bench.kernel_source_digest()
    (prof / "insert_traffic.json").write_text(json.dumps(rec))
    assert bench.recorded_traffic("wl", "bin_apply") == 123
    assert bench.recorded_traffic("wl", "bin_split") is None
    assert bench.recorded_traffic("other", "bin_apply") is None


def test_committed_traffic_record_is_well_formed():
    # every entry: bytes per launch, the kernels it sums, the digest of the
    # code it was taken on, and an ncu command that leaves the clocks alone
    rec = json.load(open(os.path.join(bench.ROOT, "profiles", "insert_traffic.json")))
    for wl, kernels in rec.items():
        assert wl in ("100mbp_30x_k31", "5mbp_50x_k31", "2mbp_30x_k31")
        for name, e in kernels.items():
            assert name in ("bin_count", "bin_scatter", "bin_split", "bin_apply", "bin_deferred")
            assert e["dram_bytes_per_launch"] > 0 and e["kernels"]
            assert len(e["kernel_source_digest"]) == 16
            assert "ncu " in e["command"] and "--clock-control none" in e["command"]


def test_path_roofline_arithmetic():
    # 120 edges, 121 touches, 45.5 input bytes: 64.91 B per edge; 1 s at 6.5 TB/s
    r = bench.path_roofline(120, 121, 45.5, 1.0, 6500.0, None)
    assert r["bytes_per_edge"] == pytest.approx((121 * 64 + 45.5) / 120)
    assert r["hbm_ceiling"] == pytest.approx(6500e9 / r["bytes_per_edge"])
    assert r["achieved"] == 120.0 and r["atomic_ceiling"] is None
    probe = {"load_red_touches_per_s": 2.42e10}
    r = bench.path_roofline(120, 121, 45.5, 1.0, 6500.0, probe)
    assert r["atomic_ceiling"] == pytest.approx(2.42e10 * 120 / 121)
    assert r["roofline"] == min(r["hbm_ceiling"], r["atomic_ceiling"])
    # the binned insert does not touch the table at random: the atomic rate
    # is the direct path's ceiling only, and the roofline is HBM's
    r = bench.path_roofline(120, 121, 45.5, 1.0, 6500.0, probe, binned=True)
    assert r["atomic_ceiling"] is None and r["roofline"] == r["hbm_ceiling"]
    assert r["direct_path_atomic_ceiling"] == pytest.approx(2.42e10 * 120 / 121)
    assert r["frac_of_roofline"] == r["frac_of_hbm_ceiling"]


def test_autotune_candidates():
    direct = autotune.candidates(31, binned=False)
    assert all(c["insert_path"] == 1 for c in direct) and len(direct) == 8
    both = autotune.candidates(31, binned=True)
    binned = [c for c in both if c["insert_path"] == 2]
    assert {c["apply_mode"] for c in binned} == {1, 2}
    assert {c["region_log2"] for c in binned if c["apply_mode"] == 2} == {0, 20, 22}
    # 64-bit events carry keys of at most 60 bits: no binned candidates for k = 32
    assert all(c["insert_path"] == 1 for c in autotune.candidates(32, binned=True))


def test_autotune_covers_the_binned_shapes():
    binned = [c for c in autotune.candidates(31, binned=True) if c.get("apply_mode") == 2]
    assert {c["scatter_reads"] for c in binned} >= {0, 256, 512}
    assert {c["split_threads"] for c in binned} >= {0, 1024}
    batch = autotune.batch_candidates()
    assert all(c["insert_path"] == 2 and c["apply_mode"] == 2 for c in batch)
    assert len({tuple(sorted(c.items())) for c in batch}) == len(batch)
    for c in batch:  # every field is one the C library accepts
        assert set(c) <= set(bench_tuning_fields())
        assert c["scatter_reads"] in (0,) or 32 <= c["scatter_reads"] <= 512
        assert c["split_threads"] in (0, 256, 512, 1024)


def bench_tuning_fields():
    from paper_2401_02756_gb300 import dbg
    return dbg.Graph.TUNING_FIELDS
