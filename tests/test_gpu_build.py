"""dbg_build_reads (discard the graph, then insert, in one call) against the
oracle, bit for bit, on every path: the direct insert, the binned insert with
the tiled apply (whose tiles start EMPTY in shared memory and are all written
once, which is the reset), the streaming apply, 128-bit keys, the binned
fall-back to the direct insert, and host buffers.  Every build goes into a
table that already holds another graph, so a slot the build forgot to empty
shows up as a wrong vertex."""

import numpy as np
import pytest

from gpu_util import assert_same_graph, capacity_for, oracle_export, to_device
from paper_2401_02756_gb300 import build, dbg, synth

pytestmark = pytest.mark.gpu

MULTI_REGION = 5_000_003  # slots: several regions, a last tile of 1,795 slots


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    build.build()
    dbg.load()


def dirty(g, k, seed=77):
    """Fill the graph with an unrelated read set first."""
    other = synth.ragged_reads(1500, 200, k, seed)
    g.insert(*to_device(other))


@pytest.mark.parametrize("k,capacity,tuning", [
    (21, None, dict(insert_path=1)),                         # direct
    (31, MULTI_REGION, dict(insert_path=2)),                 # binned, tiled apply
    (25, MULTI_REGION, dict(insert_path=2, region_log2=16)), # tiled, 32 tiles per region
    (27, MULTI_REGION, dict(insert_path=2, apply_mode=1)),   # binned, streaming apply
    (51, None, None),                                        # 128-bit keys
])
def test_build_discards_what_the_table_held(k, capacity, tuning):
    rs = synth.ragged_reads(3000, 260, k, 3100 + k, lead=k % 4)
    g = dbg.Graph(k, capacity or capacity_for(rs))
    if tuning:
        g.set_tuning(**tuning)
    dirty(g, k)
    packed, offsets = to_device(rs)
    g.build(packed, offsets)
    assert g.status() == dbg.OK
    if tuning and tuning.get("insert_path") == 2:
        assert g.binned_counters()["binned"]
    exp = oracle_export(rs)
    assert_same_graph(g.export(), exp)
    # the vertex and edge totals: counted by the tiled build itself, or by a
    # pass over the table
    assert g.stats() == (len(exp[0]), rs.n_edges())
    g.build(packed, offsets)  # again: the same graph, not twice the counts
    assert_same_graph(g.export(), exp)
    assert g.stats() == (len(exp[0]), rs.n_edges())
    g.insert(packed, offsets)  # an insert after a build adds as usual
    assert g.stats() == (len(exp[0]), 2 * rs.n_edges())
    keys, counts = g.export()
    assert np.array_equal(keys, exp[0]) and np.array_equal(counts, 2 * exp[1])
    g.normalize(2.0)  # (the counters change: the totals are counted again)
    assert g.stats() == (len(exp[0]), rs.n_edges())
    g.close()


def test_build_writes_tiles_without_events():
    # a few reads into a large table: most tiles receive no event and must
    # still come out EMPTY, including the short last tile
    rs = synth.ragged_reads(40, 150, 31, 3200)
    g = dbg.Graph(31, MULTI_REGION)
    g.set_tuning(insert_path=2)
    dirty(g, 31, seed=78)
    g.build(*to_device(rs))
    assert g.status() == dbg.OK
    assert g.binned_counters()["binned"]
    assert_same_graph(g.export(), oracle_export(rs))
    assert g.stats() == (len(oracle_export(rs)[0]), rs.n_edges())
    g.close()


@pytest.mark.parametrize("fill", [1.1, 1.5])
def test_build_at_high_load_defers_exactly(fill):
    rs = synth.ragged_reads(6000, 300, 25, 3300, lead=2)
    exp = oracle_export(rs)
    g = dbg.Graph(rs.k, int(len(exp[0]) * fill) + 1)
    g.set_tuning(insert_path=2, apply_mode=2)
    g.insert(*to_device(synth.ragged_reads(400, 200, 25, 3301)))
    g.build(*to_device(rs))
    assert g.status() == dbg.OK
    c = g.binned_counters()
    assert c["binned"] and c["deferred"] > 0, c
    assert_same_graph(g.export(), exp)
    assert g.stats() == (len(exp[0]), rs.n_edges())  # deferred vertices counted too
    g.close()


def test_build_falls_back_to_the_direct_insert_on_an_emptied_table():
    # a read repeated 20,000 times overflows a region bucket: no binned kernel
    # touches the table, so the build's gated emptying pass runs before the
    # direct insert does the work
    rs = synth.from_strings(["ACGTTGCAAGGCTTAACCGTAGGCATCGATCGGATC" * 4] * 20000, 21)
    g = dbg.Graph(21, MULTI_REGION)
    g.set_tuning(insert_path=2)
    dirty(g, 21, seed=79)
    g.enable_kernel_timing(1)
    g.build(*to_device(rs))
    assert g.status() == dbg.OK
    assert not g.binned_counters()["binned"]
    t = g.kernel_times()
    assert t[-1, dbg.Graph.KERNELS.index("direct_fallback")] >= 0
    exp = oracle_export(rs)
    assert_same_graph(g.export(), exp)
    assert g.stats() == (len(exp[0]), rs.n_edges())  # the fall-back counts nothing itself
    g.close()


def test_build_clears_an_earlier_error():
    big = synth.ragged_reads(3000, 200, 21, 3400)
    small = synth.ragged_reads(20, 120, 21, 3401)
    g = dbg.Graph(21, capacity_for(small, 4.0))
    g.insert(*to_device(big))
    assert g.status() == dbg.ERR_CAPACITY
    g.build(*to_device(small))
    assert g.status() == dbg.OK
    assert_same_graph(g.export(), oracle_export(small))
    g.close()


@pytest.mark.parametrize("path", [1, 2])
def test_build_host_and_empty_build(path):
    rs = synth.ragged_reads(2500, 240, 29, 3500 + path, lead=3)
    g = dbg.Graph(rs.k, MULTI_REGION)
    g.set_tuning(insert_path=path)
    dirty(g, rs.k, seed=80)
    g.build_host(rs.packed, rs.offsets)
    assert g.status() == dbg.OK
    assert_same_graph(g.export(), oracle_export(rs))
    # offsets that decrease are refused (checked while the input is copied)
    # before any kernel runs: the graph stays as it was
    bad = rs.offsets.copy()
    bad[1000] = bad[999] - 1
    with pytest.raises(dbg.DbgError) as e:
        g.build_host(rs.packed, bad)
    assert e.value.code == dbg.ERR_INVALID_ARG
    assert g.status() == dbg.OK
    assert_same_graph(g.export(), oracle_export(rs))
    empty = np.zeros(1, dtype=np.uint64)
    g.build_host(np.zeros(1, np.uint8), empty)  # no reads: the table is only emptied
    assert g.stats() == (0, 0)
    g.close()
