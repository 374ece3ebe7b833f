"""Parity of the CUDA insert path with the CPU oracle, element by element
(integer work: bit-exact), on seeded inputs that span many tiles and end in a
ragged tile, plus the edge cases of the method."""

import os

import numpy as np
import pytest

from gpu_util import (assert_same_graph, capacity_for, gpu_export, gpu_graph, oracle_export,
                      to_device)
from paper_2401_02756_gb300 import build, dbg, synth

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    build.build()
    dbg.load()


def test_fig1_worked_example():
    from test_oracle import load_golden
    read, k, rows = load_golden("fig1_acgacgacgc_k4.txt")
    rs = synth.from_strings([read], k)
    keys, counts = gpu_export(rs)
    got = {"".join("ACGT"[(int(x) >> (2 * (k - 2 - j))) & 3] for j in range(k - 1)): tuple(int(v) for v in c)
           for x, c in zip(keys, counts)}
    assert got == rows
    assert list(got) == sorted(got)


def test_10kb_workload():
    rs = synth.workload_10kb()
    got = gpu_export(rs)
    assert_same_graph(got, oracle_export(rs))
    assert int(got[1].astype(np.int64).sum()) == 80_000
    assert got[0].size <= 9_981


@pytest.mark.parametrize("k", [2, 3, 4, 5, 11, 21, 31, 32])
def test_ragged_reads(k):
    rs = synth.ragged_reads(3000, 300, k, 1000 + k, lead=k % 7)
    assert_same_graph(gpu_export(rs), oracle_export(rs))


def test_stats_match_oracle():
    rs = synth.ragged_reads(2000, 250, 21, 4242)
    g = gpu_graph(rs)
    nv, ne = g.stats()
    ek, ec = oracle_export(rs)
    assert (nv, ne) == (ek.size, int(ec.astype(np.int64).sum())) == (ek.size, rs.n_edges())
    g.close()


@pytest.mark.parametrize("tuning", [
    dict(block_threads=128), dict(block_threads=512), dict(tile_reads=1), dict(tile_reads=7),
    dict(tile_reads=100, block_threads=128), dict(grid_ctas=1), dict(grid_ctas=3),
    dict(warp_aggregate=1), dict(warp_aggregate=1, block_threads=512, tile_reads=33),
    dict(warp_aggregate=0), dict(warp_aggregate=0, block_threads=128, tile_reads=50),
])
def test_launch_shape_independence(tuning):
    rs = synth.ragged_reads(1500, 220, 31, 77, lead=3)
    assert_same_graph(gpu_export(rs, tuning=tuning), oracle_export(rs))


def test_split_calls_and_streams():
    import torch
    rs = synth.ragged_reads(2500, 200, 25, 99, lead=1)
    packed, offsets = to_device(rs)
    g = dbg.Graph(rs.k, capacity_for(rs))
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    torch.cuda.synchronize()
    cuts = [0, 700, 701, 1900, rs.n_reads]
    for i in range(len(cuts) - 1):
        a, b = cuts[i], cuts[i + 1]
        g.insert(packed, offsets[a:b + 1], stream=s1 if i % 2 else s2)
    torch.cuda.synchronize()
    assert g.status() == dbg.OK
    assert_same_graph(g.export(), oracle_export(rs))
    g.close()


@pytest.mark.parametrize("pinned", [False, True])
def test_insert_from_host_buffers(pinned):
    import torch
    rs = synth.ragged_reads(3000, 180, 21, 5, lead=2)
    g = dbg.Graph(rs.k, capacity_for(rs))
    pk = torch.from_numpy(rs.packed.copy())
    of = torch.from_numpy(rs.offsets.view(np.int64).copy())
    if pinned:
        pk, of = pk.pin_memory(), of.pin_memory()
    g.insert_host(pk, of)
    assert g.status() == dbg.OK
    assert_same_graph(g.export(), oracle_export(rs))
    g.close()


def test_batch_of_graphs_with_mixed_k():
    sets = [synth.ragged_reads(400 + 50 * i, 160, k, 300 + i) for i, k in
            enumerate([21, 31, 5, 21, 32, 2])]
    graphs = [dbg.Graph(rs.k, capacity_for(rs)) for rs in sets]
    devs = [to_device(rs) for rs in sets]
    dbg.insert_batch([(g, p, o) for g, (p, o) in zip(graphs, devs)])
    for g, rs in zip(graphs, sets):
        assert g.status() == dbg.OK
        assert_same_graph(g.export(), oracle_export(rs))
        g.close()


def test_batch_larger_than_one_launch():
    sets = [synth.ragged_reads(20, 60, 9, 7000 + i) for i in range(150)]
    graphs = [dbg.Graph(rs.k, capacity_for(rs)) for rs in sets]
    devs = [to_device(rs) for rs in sets]
    dbg.insert_batch([(g, p, o) for g, (p, o) in zip(graphs, devs)])
    for g, rs in zip(graphs[::7], sets[::7]):
        assert_same_graph(g.export(), oracle_export(rs))
    for g in graphs:
        g.close()


def test_reads_wider_than_the_window():
    # 64 Ki bases fit the shared-memory window: these reads need sub-tiles and
    # the global-memory path
    g0 = synth.random_genome(400_000, 17)
    s = synth.codes_to_ascii(g0)
    reads = [s[:70_000], "ACGT" * 10, s[1000:201_000], "", s[5:300], s[:65_530], s[7:65_600]]
    rs = synth.from_strings(reads, 31, lead=5)
    assert_same_graph(gpu_export(rs), oracle_export(rs))
    assert_same_graph(gpu_export(rs, tuning=dict(tile_reads=2, block_threads=128)), oracle_export(rs))


@pytest.mark.parametrize("agg", [0, 1])
def test_low_complexity_reads(agg):
    reads = ["A" * 150] * 300 + ["AC" * 75] * 200 + ["ACG" * 50] * 100 + ["AAAAT" * 30] * 50
    rs = synth.from_strings(reads, 31)
    got = gpu_export(rs, tuning=dict(warp_aggregate=agg))
    assert_same_graph(got, oracle_export(rs))
    # the homopolymer vertex counts every one of its k-mers
    assert int(got[0][0]) == 0 and int(got[1][0, 0]) == 300 * 120


def test_unaligned_packed_pointer():
    rs = synth.ragged_reads(800, 200, 21, 31337, lead=1)
    for shift in (1, 3, 8, 13):
        assert_same_graph(gpu_export(rs, shift=shift), oracle_export(rs))


def test_reset_empties_the_graph():
    rs = synth.ragged_reads(500, 150, 21, 8)
    g = gpu_graph(rs)
    g.reset()
    assert g.stats() == (0, 0)
    packed, offsets = to_device(rs)
    g.insert(packed, offsets)
    assert_same_graph(g.export(), oracle_export(rs))
    g.close()


def test_capacity_overflow_is_reported_not_hung():
    rs = synth.ragged_reads(500, 150, 21, 9)
    g = dbg.Graph(rs.k, 100)  # far fewer slots than vertices
    packed, offsets = to_device(rs)
    g.insert(packed, offsets)
    assert g.status() == dbg.ERR_CAPACITY
    with pytest.raises(dbg.DbgError) as e:
        g.export()
    assert e.value.code == dbg.ERR_CAPACITY
    g.reset()
    assert g.status() == dbg.OK
    g.close()


def test_bad_offsets_are_reported():
    rs = synth.ragged_reads(600, 100, 11, 10)
    packed, offsets = to_device(rs)
    bad = offsets.clone()
    bad[300] = bad[302] + 5  # offsets[300] > offsets[301]
    g = dbg.Graph(rs.k, capacity_for(rs))
    g.insert(packed, bad)
    assert g.status() == dbg.ERR_BAD_OFFSETS
    g.close()
    g = dbg.Graph(rs.k, capacity_for(rs))
    g.insert(packed, offsets[:1].clone(), n_reads=0)  # nothing to do
    assert g.stats() == (0, 0)
    g.close()


def test_export_size_query_and_device_export():
    import ctypes
    rs = synth.ragged_reads(700, 120, 15, 11)
    g = gpu_graph(rs)
    lib = dbg.load()
    n = ctypes.c_uint64()
    keys = np.zeros(4, dtype=np.uint64)
    st = lib.dbg_export_sorted(g.handle, keys.ctypes.data, None, 4, ctypes.byref(n), None)
    assert st == dbg.ERR_BUFFER_TOO_SMALL and n.value > 4
    assert not keys.any()  # nothing written
    hk, hc = g.export()
    dk, dc = g.export_device()
    assert np.array_equal(dk.cpu().numpy().view(np.uint64), hk)
    assert np.array_equal(dc.cpu().numpy().view(np.uint32), hc)
    g.close()


def test_short_and_empty_reads_only():
    rs = synth.from_strings(["", "ACG", "", "ACGTACGTACGT"[:10], "A"], 11, lead=2)
    assert_same_graph(gpu_export(rs), oracle_export(rs))
    rs = synth.from_strings(["ACGTACGTAC"], 10)  # len == k: one edge, two vertices
    got = gpu_export(rs)
    assert got[0].size == 2 and int(got[1].sum()) == 1


def test_export_with_caller_scratch():
    import torch
    rs = synth.ragged_reads(3000, 250, 31, 4400, lead=2)
    g = gpu_graph(rs)
    D, _ = g.stats()
    keys = torch.empty(D, dtype=torch.int64, device="cuda")
    counts = torch.empty((D, 4), dtype=torch.int32, device="cuda")
    xs = dbg.export_scratch_bytes(31, D, g.info()["n_slots"])
    assert xs >= 4 * D
    scratch = torch.empty(xs, dtype=torch.uint8, device="cuda")
    for _ in range(2):  # the scratch holds the first call's contents the second time
        assert g.export_with(keys, counts, scratch) == D
        assert_same_graph((keys.cpu().numpy().view(np.uint64), counts.cpu().numpy().view(np.uint32)),
                          oracle_export(rs))
    with pytest.raises(dbg.DbgError) as e:  # too small a scratch is refused
        g.export_with(keys, counts, scratch[:xs // 2])
    assert e.value.code == dbg.ERR_INVALID_ARG
    g.close()


@pytest.mark.parametrize("n_shared", [20, 200, 2100])
def test_export_keys_sharing_a_prefix(n_shared):
    # keys of k = 31 are sorted by their top 32 bits (16 bases) first; reads
    # whose first 16 bases agree give runs of keys with one prefix: a run of
    # 20 is put in order by a warp, one of 200 by a CTA in shared memory, and
    # one of 2100 (over 2048) makes the export fall back to the full-width
    # sort -- the same graph every way
    import torch
    rng = np.random.default_rng(n_shared)
    head = "ACGTTGCAAGGCTTAA"
    reads = [head + "".join(rng.choice(list("ACGT"), size=40)) for _ in range(n_shared)]
    base = synth.ragged_reads(500, 200, 31, 4500)
    rs = synth.from_strings(reads + [base.read_ascii(i) for i in range(base.n_reads)], 31)
    g = gpu_graph(rs)
    exp = oracle_export(rs)
    assert_same_graph(g.export(), exp)  # host outputs
    keys, counts = g.export_device()    # device outputs: the sort runs inside them
    assert_same_graph((keys.cpu().numpy().view(np.uint64), counts.cpu().numpy().view(np.uint32)),
                      exp)
    g.close()


def test_export_into_larger_and_smaller_device_buffers():
    # the in-place export lays its sort out over all max_n rows of the
    # outputs and counts the vertices while it compacts: rows beyond D are
    # scratch, and too few rows give BUFFER_TOO_SMALL with the count
    import ctypes

    import torch
    rs = synth.ragged_reads(2500, 220, 31, 4600, lead=1)
    g = gpu_graph(rs)
    exp = oracle_export(rs)
    D = exp[0].size
    lib = dbg.load()
    for rows in (D, D + 1, 3 * D + 7):
        keys = torch.empty(rows, dtype=torch.int64, device="cuda")
        counts = torch.empty((rows, 4), dtype=torch.int32, device="cuda")
        assert g.export_into(keys, counts) == D
        assert_same_graph((keys[:D].cpu().numpy().view(np.uint64),
                           counts[:D].cpu().numpy().view(np.uint32)), exp)
    keys = torch.empty(D - 1, dtype=torch.int64, device="cuda")
    counts = torch.empty((D - 1, 4), dtype=torch.int32, device="cuda")
    n = ctypes.c_uint64()
    st = lib.dbg_export_sorted(g.handle, keys.data_ptr(), counts.data_ptr(), D - 1, ctypes.byref(n),
                               None)
    assert st == dbg.ERR_BUFFER_TOO_SMALL and n.value == D
    assert g.stats()[0] == D  # the graph is untouched
    g.close()
