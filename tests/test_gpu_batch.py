"""The batched insert captured into a CUDA graph and replayed: direct and
binned items in one captured call give the same graphs as one plain insert
per item, and the same again on every replay."""

import numpy as np
import pytest

import oracle
from gpu_util import capacity_for, to_device
from paper_2401_02756_gb300 import build, dbg, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    build.build()
    dbg.load()


def make_graphs(sets, paths):
    gs = []
    for rs, path in zip(sets, paths):
        g = dbg.Graph(rs.k, capacity_for(rs))
        g.set_tuning(insert_path=path)
        gs.append(g)
    return gs


def test_captured_batch_equals_plain_inserts():
    import torch
    sets = [synth.ragged_reads(n, 260, k, 7000 + i, lead=i % 4)
            for i, (n, k) in enumerate([(900, 21), (3000, 31), (50, 31), (2500, 21), (1200, 31)])]
    paths = [1, 2, 1, 1, 2]  # two items take the binned path inside the batch
    dev = [to_device(rs) for rs in sets]
    ref = make_graphs(sets, paths)
    for g, (pk, of) in zip(ref, dev):
        g.insert(pk, of)
    expect = [g.export() for g in ref]
    for g in ref:
        g.close()

    gs = make_graphs(sets, paths)
    items = [(g, pk, of) for g, (pk, of) in zip(gs, dev)]
    dbg.insert_batch(items)  # first call allocates the binned items' scratch
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s):
        dbg.insert_batch(items, s)
    for _ in range(2):
        for g in gs:
            g.reset()
        graph.replay()
        torch.cuda.synchronize()
        for g, (keys, counts) in zip(gs, expect):
            assert g.status() == dbg.OK
            k2, c2 = g.export()
            assert np.array_equal(k2, keys) and np.array_equal(c2, counts)
    o = oracle.build_graph(sets[1].packed, sets[1].offsets, 31)
    assert np.array_equal(expect[1][0], o.keys) and np.array_equal(expect[1][1], o.counts)
    for g in gs:
        g.close()


# --- binned chains: many tables per launch of each binned kernel --------------

def _dirty(g, k, seed):
    g.insert(*to_device(synth.ragged_reads(300, 180, k, seed)))


def _expect(rs):
    o = oracle.build_graph(rs.packed, rs.offsets, rs.k)
    return o.keys, o.counts


def _check(g, exp):
    assert g.status() == dbg.OK
    keys, counts = g.export()
    assert np.array_equal(keys, exp[0]) and np.array_equal(counts, exp[1])


@pytest.mark.parametrize("build", [False, True])
def test_binned_chain_of_many_tables(build):
    # twelve binned graphs of mixed k and size, two of several regions (2^21
    # slots each), one with no reads, all in one chain; a build goes into
    # tables that hold other graphs
    specs = [(21, 1200, 600_000), (31, 2500, 5_000_000), (25, 40, 90_000), (31, 0, 70_000),
             (27, 1800, 2_500_000), (21, 900, 300_000), (31, 3000, 4_300_000), (23, 700, 200_000),
             (29, 1500, 1_000_000), (21, 60, 100_000), (31, 2200, 800_000), (25, 1000, 400_000)]
    sets = [synth.ragged_reads(n, 260, k, 7100 + i, lead=i % 4) for i, (k, n, _) in enumerate(specs)]
    graphs = []
    for (k, _, cap), rs in zip(specs, sets):
        g = dbg.Graph(k, cap)
        g.set_tuning(insert_path=2)
        if build:
            _dirty(g, k, 7300 + len(graphs))
        graphs.append(g)
    items = [(g, *to_device(rs)) for g, rs in zip(graphs, sets)]
    (dbg.build_batch if build else dbg.insert_batch)(items)
    for g, rs in zip(graphs, sets):
        _check(g, _expect(rs))
    for g in graphs:
        g.close()


def test_binned_chains_split_by_items_and_regions():
    # 140 binned graphs (more than one chain holds), then 30 graphs of 77
    # regions each (2^16-slot regions: more regions than one chain holds)
    sets = [synth.ragged_reads(40 + 3 * i, 200, 21 + (i % 3) * 5, 7500 + i) for i in range(140)]
    graphs = []
    for rs in sets:
        g = dbg.Graph(rs.k, capacity_for(rs) + 300_000)
        g.set_tuning(insert_path=2)
        graphs.append(g)
    dbg.insert_batch([(g, *to_device(rs)) for g, rs in zip(graphs, sets)])
    for g, rs in zip(graphs, sets):
        _check(g, _expect(rs))
        g.close()
    sets = [synth.ragged_reads(200, 200, 31, 7700 + i) for i in range(30)]
    graphs = []
    for rs in sets:
        g = dbg.Graph(31, 5_000_000)
        g.set_tuning(insert_path=2, region_log2=16)
        graphs.append(g)
    dbg.build_batch([(g, *to_device(rs)) for g, rs in zip(graphs, sets)])
    for g, rs in zip(graphs, sets):
        _check(g, _expect(rs))
        g.close()


def test_build_batch_mixes_paths_and_replays_from_a_graph():
    import torch
    # direct (small tables), binned (insert_path=2) and 128-bit keys in one
    # build, captured after one uncaptured call and replayed into dirty tables
    specs = [(21, 800, 1), (31, 2000, 2), (51, 300, 0), (25, 1500, 2), (31, 50, 1), (63, 200, 0)]
    sets = [synth.ragged_reads(n, 240, k, 7900 + i, lead=i % 3) for i, (k, n, _) in enumerate(specs)]
    graphs = []
    for (k, _, path), rs in zip(specs, sets):
        g = dbg.Graph(k, capacity_for(rs) + 200_000)
        if path:
            g.set_tuning(insert_path=path)
        graphs.append(g)
    dev = [to_device(rs) for rs in sets]
    items = [(g, pk, of) for g, (pk, of) in zip(graphs, dev)]
    dbg.build_batch(items)
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    cg = torch.cuda.CUDAGraph()
    with torch.cuda.graph(cg, stream=s):
        dbg.build_batch(items, s)
    exp = [_expect(rs) for rs in sets]
    for rep in range(2):
        for i, g in enumerate(graphs):
            _dirty(g, g.k, 8000 + 10 * rep + i)
        torch.cuda.synchronize()
        cg.replay()
        torch.cuda.synchronize()
        for g, e in zip(graphs, exp):
            _check(g, e)
    for g in graphs:
        g.close()


def test_captured_batch_without_scratch_takes_the_direct_insert():
    import torch
    # the library's buffers released: a first call inside a capture cannot
    # allocate them, so the chain's graphs are inserted by the direct kernel
    sets = [synth.ragged_reads(900 + 200 * i, 220, 27, 8100 + i) for i in range(3)]
    graphs = []
    for rs in sets:
        g = dbg.Graph(27, capacity_for(rs) + 100_000)
        g.set_tuning(insert_path=2)
        graphs.append(g)
    dev = [to_device(rs) for rs in sets]
    torch.cuda.synchronize()
    dbg.release_scratch()
    s = torch.cuda.Stream()
    cg = torch.cuda.CUDAGraph()
    with torch.cuda.graph(cg, stream=s):
        dbg.build_batch([(g, pk, of) for g, (pk, of) in zip(graphs, dev)], s)
    cg.replay()
    torch.cuda.synchronize()
    for g, rs in zip(graphs, sets):
        _check(g, _expect(rs))
        g.close()


def test_chain_falls_back_to_the_direct_insert_exactly():
    # one graph's read repeated 20,000 times overflows its region's bucket:
    # the whole chain is done by the direct insert (and, for a build, its
    # tables are emptied first)
    rep = synth.from_strings(["ACGTTGCAAGGCTTAACCGTAGGCATCGATCGGATC" * 4] * 20000, 21)
    sets = [synth.ragged_reads(1000, 200, 21, 8200), rep, synth.ragged_reads(700, 200, 31, 8201)]
    graphs = []
    for rs in sets:
        g = dbg.Graph(rs.k, 3_000_000)
        g.set_tuning(insert_path=2)
        _dirty(g, rs.k, 8210 + len(graphs))
        graphs.append(g)
    dbg.build_batch([(g, *to_device(rs)) for g, rs in zip(graphs, sets)])
    for g, rs in zip(graphs, sets):
        _check(g, _expect(rs))
        g.close()
