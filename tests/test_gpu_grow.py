"""Grow-and-rebuild: a graph in a table that is too small keeps the vertices
it has no room for in a spill buffer; dbg_grow moves it to a larger table
and replays them, and the result equals the oracle's graph exactly."""

import numpy as np
import pytest

from gpu_util import assert_same_graph, oracle_export, to_device
from paper_2401_02756_gb300 import build, dbg, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    build.build()
    dbg.load()


@pytest.mark.parametrize("path", [1, 2])
def test_spill_then_grow_is_exact(path):
    rs = synth.ragged_reads(2500, 220, 21, 501, lead=2)
    ek, ec = oracle_export(rs)
    g = dbg.Graph(rs.k, int(ek.size * 0.6), max_probes=128)  # far too small
    g.set_tuning(insert_path=path)
    g.set_spill(rs.n_edges() + rs.n_reads)
    packed, offsets = to_device(rs)
    g.insert(packed, offsets)
    assert g.status() == dbg.ERR_NEEDS_GROW
    with pytest.raises(dbg.DbgError) as e:
        g.export()
    assert e.value.code == dbg.ERR_NEEDS_GROW
    g.grow(int(ek.size * 1.6))
    assert g.status() == dbg.OK
    assert_same_graph(g.export(), (ek, ec))
    # the grown graph keeps working: a second pass doubles every counter
    g.insert(packed, offsets)
    assert g.status() == dbg.OK
    k2, c2 = g.export()
    assert np.array_equal(k2, ek) and np.array_equal(c2, 2 * ec)
    g.close()


def test_grow_twice_and_default_doubling():
    rs = synth.ragged_reads(1500, 200, 31, 502)
    ek, ec = oracle_export(rs)
    g = dbg.Graph(rs.k, int(ek.size * 0.3), max_probes=128)
    g.set_spill(rs.n_edges() + rs.n_reads)
    packed, offsets = to_device(rs)
    g.insert(packed, offsets)
    with pytest.raises(dbg.DbgError) as e:
        g.grow()  # twice 0.3 x D: still too small, and the graph is kept
    assert e.value.code == dbg.ERR_CAPACITY
    assert g.status() == dbg.ERR_NEEDS_GROW
    g.grow(int(ek.size * 2))
    assert g.status() == dbg.OK
    assert_same_graph(g.export(), (ek, ec))
    g.close()


def test_grow_into_a_too_small_table_keeps_the_graph():
    rs = synth.ragged_reads(800, 150, 21, 503)
    ek, ec = oracle_export(rs)
    g = dbg.Graph(rs.k, int(ek.size * 0.5), max_probes=128)
    g.set_spill(rs.n_edges() + rs.n_reads)
    packed, offsets = to_device(rs)
    g.insert(packed, offsets)
    assert g.status() == dbg.ERR_NEEDS_GROW
    with pytest.raises(dbg.DbgError) as e:
        g.grow(int(ek.size * 0.7))
    assert e.value.code == dbg.ERR_CAPACITY
    assert g.status() == dbg.ERR_NEEDS_GROW  # still pending, nothing lost
    g.grow(int(ek.size * 1.5))
    assert_same_graph(g.export(), (ek, ec))
    g.close()


def test_full_spill_buffer_is_a_capacity_error():
    rs = synth.ragged_reads(800, 150, 21, 504)
    g = dbg.Graph(rs.k, 200, max_probes=16)
    g.set_spill(100)
    packed, offsets = to_device(rs)
    g.insert(packed, offsets)
    assert g.status() == dbg.ERR_CAPACITY
    with pytest.raises(dbg.DbgError):
        g.grow(100000)
    g.close()
