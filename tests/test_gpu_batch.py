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
