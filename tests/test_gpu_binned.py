"""The binned insert (events grouped by table region, applied region by
region) against the oracle, bit for bit, including its fall-back to the
direct kernel and its interplay with streams, resets and errors."""

import numpy as np
import pytest

from gpu_util import assert_same_graph, capacity_for, oracle_export, to_device
from paper_2401_02756_gb300 import build, dbg, synth

pytestmark = pytest.mark.gpu

MULTI_REGION = 5_000_000  # slots: five regions of 2^20 slots


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    build.build()
    dbg.load()


def binned_graph(rs, capacity=MULTI_REGION, **tuning):
    g = dbg.Graph(rs.k, capacity)
    g.set_tuning(insert_path=2, **tuning)
    return g


@pytest.mark.parametrize("k", [2, 5, 21, 31, 32])
def test_binned_matches_oracle(k):
    rs = synth.ragged_reads(3000, 300, k, 2000 + k, lead=k % 5)
    g = binned_graph(rs)
    packed, offsets = to_device(rs)
    g.insert(packed, offsets)
    assert g.status() == dbg.OK
    if k <= 31:
        assert g.info()["event_capacity"] > 0
    if k >= 21:  # (k = 2, 5: a handful of keys overflow a region's bucket: direct insert)
        assert g.binned_counters()["binned"] == (k <= 31)  # 64-bit events need k <= 31
    assert_same_graph(g.export(), oracle_export(rs))
    g.close()


def test_binned_single_region_table():
    rs = synth.ragged_reads(2000, 200, 21, 33)
    g = binned_graph(rs, capacity=capacity_for(rs))
    packed, offsets = to_device(rs)
    g.insert(packed, offsets)
    assert_same_graph(g.export(), oracle_export(rs))
    g.close()


def test_binned_falls_back_when_events_do_not_fit():
    rs = synth.ragged_reads(20000, 200, 21, 34)
    g = binned_graph(rs)
    positions = int(np.maximum(rs.lengths() - rs.k + 2, 0).sum())
    g.reserve_events(1000)  # far fewer than the vertex positions (plus the buckets' margin)
    assert 1000 <= g.info()["event_capacity"] < positions
    packed, offsets = to_device(rs)
    g.insert(packed, offsets)
    assert g.status() == dbg.OK
    assert_same_graph(g.export(), oracle_export(rs))
    g.close()


def test_binned_calls_on_two_streams_and_repeated():
    import torch
    rs = synth.ragged_reads(2500, 220, 25, 35, lead=2)
    g = binned_graph(rs, capacity=MULTI_REGION)
    packed, offsets = to_device(rs)
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    torch.cuda.synchronize()
    cuts = [0, 600, 1700, rs.n_reads]
    for i in range(3):
        g.insert(packed, offsets[cuts[i]:cuts[i + 1] + 1], stream=s1 if i % 2 else s2)
    torch.cuda.synchronize()
    assert_same_graph(g.export(), oracle_export(rs))
    # a second pass doubles every counter and adds no vertex
    g.insert(packed, offsets)
    keys, counts = g.export()
    ek, ec = oracle_export(rs)
    assert np.array_equal(keys, ek) and np.array_equal(counts, 2 * ec)
    g.reset()
    g.insert(packed, offsets)
    assert_same_graph(g.export(), oracle_export(rs))
    g.close()


def test_binned_with_host_buffers_and_low_complexity():
    reads = ["A" * 150] * 200 + ["AC" * 75] * 100
    rs0 = synth.ragged_reads(1500, 200, 31, 36)
    rs = synth.from_strings(reads + [rs0.read_ascii(i) for i in range(rs0.n_reads)], 31)
    g = binned_graph(rs)
    g.insert_host(rs.packed, rs.offsets)
    assert g.status() == dbg.OK
    assert_same_graph(g.export(), oracle_export(rs))
    g.close()


def test_binned_capacity_overflow_is_reported():
    rs = synth.ragged_reads(800, 150, 21, 37)
    g = binned_graph(rs, capacity=300)
    packed, offsets = to_device(rs)
    g.insert(packed, offsets)
    assert g.status() == dbg.ERR_CAPACITY
    g.close()


def test_auto_path_picks_binned_for_large_tables():
    rs = synth.ragged_reads(1000, 150, 21, 38)
    g = dbg.Graph(rs.k, (256 << 20) // 32)  # exactly the automatic threshold
    packed, offsets = to_device(rs)
    assert g.binned_counters() == {"binned": False, "deferred": 0, "overflow": 0}  # no call yet
    g.insert(packed, offsets)
    assert g.info()["event_capacity"] > 0
    assert g.binned_counters()["binned"]
    assert_same_graph(g.export(), oracle_export(rs))
    g.close()
    small = dbg.Graph(rs.k, capacity_for(rs))
    small.insert(packed, offsets)
    assert small.info()["event_capacity"] == 0
    assert not small.binned_counters()["binned"]  # the direct path: no binned call
    small.close()


def test_kernel_timer_records_the_kernels_each_path_launches():
    rs = synth.ragged_reads(1500, 200, 21, 39)
    packed, offsets = to_device(rs)
    K = len(dbg.Graph.KERNELS)
    for tuning, launched in ((dict(insert_path=1), [0]),
                             # tiled: bucket sizing (under "bin_count") replaces count + scan
                             (dict(insert_path=2), [1, 3, 4, 5, 6, 7]),
                             (dict(insert_path=2, apply_mode=1), [1, 2, 3, 5, 7])):
        g = dbg.Graph(rs.k, MULTI_REGION)
        g.set_tuning(**tuning)
        g.enable_kernel_timing(4)
        for _ in range(6):  # more calls than kept: the oldest are dropped
            g.insert(packed, offsets)
        t = g.kernel_times()
        assert t.shape == (4, K)
        for j in range(K):
            if j in launched:
                assert (t[:, j] >= 0).all(), (tuning, j, t)
            else:
                assert (t[:, j] == -1).all(), (tuning, j, t)
        g.close()


@pytest.mark.parametrize("tuning", [
    # the streaming apply and its launch shapes
    dict(apply_mode=1), dict(apply_mode=1, apply_unroll=2), dict(apply_mode=1, apply_unroll=8),
    dict(apply_mode=1, apply_chunk=4), dict(apply_mode=1, apply_chunk=16),
    dict(apply_mode=1, apply_ctas=1), dict(apply_mode=1, apply_counters=1),
    dict(apply_mode=1, apply_counters=64), dict(apply_mode=1, region_log2=16),
    dict(apply_mode=1, region_log2=26, apply_chunk=4, apply_unroll=2),
    # the tiled apply over region sizes of 32 .. 4096 tiles (2^26: streaming fall-back)
    dict(apply_mode=2), dict(apply_mode=2, region_log2=16), dict(apply_mode=2, region_log2=20),
    dict(apply_mode=2, region_log2=23), dict(apply_mode=2, region_log2=26),
    # the direct kernel's tiles (512 reads) differ from the binned walk's
    dict(block_threads=512), dict(block_threads=512, apply_mode=1),
    dict(block_threads=128, tile_reads=96),
])
def test_binned_tuning_independence(tuning):
    rs = synth.ragged_reads(2500, 250, 27, 40, lead=1)
    g = binned_graph(rs, **tuning)
    packed, offsets = to_device(rs)
    g.insert(packed, offsets)
    assert g.status() == dbg.OK
    assert_same_graph(g.export(), oracle_export(rs))
    g.close()


@pytest.mark.parametrize("fill", [1.1, 1.3, 1.5])
def test_tiled_apply_at_high_load_defers_exactly(fill):
    # a nearly full table: long probe runs, many of them past a tile's end
    rs = synth.ragged_reads(6000, 300, 25, 41, lead=2)
    exp = oracle_export(rs)
    cap = int(len(exp[0]) * fill) + 1
    for mode in (1, 2):
        g = dbg.Graph(rs.k, cap)
        g.set_tuning(insert_path=2, apply_mode=mode)
        packed, offsets = to_device(rs)
        g.insert(packed, offsets)
        assert g.status() == dbg.OK
        c = g.binned_counters()
        assert c["binned"]
        if mode == 2:  # long probe runs cross tile ends
            assert c["deferred"] > 0
        assert_same_graph(g.export(), exp)
        g.close()


def test_tile_bucket_overflow_goes_to_the_global_pass():
    # one read repeated 1000 times: each of its keys brings 1000 events to its
    # tile, well past the tile's bucket (the region's mean per tile, about
    # 1500, plus the slack); the rest goes to the overflow area and the
    # global pass applies it, still on the binned path
    base = synth.ragged_reads(20000, 200, 21, 43)
    rep = synth.codes_to_ascii(synth.random_genome(150, 44))
    rs = synth.from_strings([base.read_ascii(r) for r in range(base.n_reads)] + [rep] * 1000, 21)
    exp = oracle_export(rs)
    g = binned_graph(rs, apply_mode=2)
    packed, offsets = to_device(rs)
    g.insert(packed, offsets)
    assert g.status() == dbg.OK
    c = g.binned_counters()
    assert c["binned"] and c["overflow"] > 0, c
    assert_same_graph(g.export(), exp)
    g.close()


def test_tiled_apply_respects_max_probes_with_a_spill():
    rs = synth.ragged_reads(4000, 250, 21, 42)
    exp = oracle_export(rs)
    g = dbg.Graph(rs.k, int(len(exp[0]) * 1.05) + 1, max_probes=16)
    g.set_tuning(insert_path=2, apply_mode=2)
    g.set_spill(2_000_000)
    packed, offsets = to_device(rs)
    g.insert(packed, offsets)
    st = g.status()
    assert st in (dbg.OK, dbg.ERR_NEEDS_GROW)
    if st == dbg.ERR_NEEDS_GROW:
        g.grow(4 * g.info()["n_slots"])
    assert g.status() == dbg.OK
    assert_same_graph(g.export(), exp)
    g.close()


def test_bucket_overflow_from_repeated_keys_falls_back_exactly():
    # one read repeated many times puts most positions in few regions: a
    # bucket (expected size + six standard deviations) overflows, and the
    # direct insert does the call instead -- the same graph either way
    rs = synth.from_strings(["ACGTTGCAAGGCTTAACCGTAGGCATCGATCGGATC" * 4] * 20000, 21)
    exp = oracle_export(rs)
    g = binned_graph(rs)
    g.enable_kernel_timing(2)
    packed, offsets = to_device(rs)
    g.insert(packed, offsets)
    assert g.status() == dbg.OK
    assert_same_graph(g.export(), exp)
    t = g.kernel_times()
    fallback = dbg.Graph.KERNELS.index("direct_fallback")
    assert t[-1, fallback] >= 0
    assert not g.binned_counters()["binned"]
    g.close()
