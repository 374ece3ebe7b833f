"""Graphs with k > 32 (128-bit keys; the paper's default k = 51) against the
oracle, bit for bit: keys as (high, low) word pairs, counters, across read
shapes, pointer alignments, batches and normalization."""

import numpy as np
import pytest

import oracle
from gpu_util import assert_same_graph, capacity_for, gpu_export, oracle_export, to_device
from oracle import contigs as oc
from paper_2401_02756_gb300 import build, dbg, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    build.build()
    dbg.load()


@pytest.mark.parametrize("k", [33, 34, 40, 51, 63, 64])
def test_wide_ragged_sets_match_oracle(k):
    rs = synth.ragged_reads(2500, 3 * k, k, 8000 + k, lead=k % 4)
    assert_same_graph(gpu_export(rs), oracle_export(rs))


@pytest.mark.parametrize("shift", [0, 3, 5])
def test_wide_genome_reads_unaligned(shift):
    g = synth.random_genome(20_000, 77)
    rs = synth.sample_reads(g, 3000, 150, 0.01, 77, 51, "k51")
    assert_same_graph(gpu_export(rs, shift=shift), oracle_export(rs))


def test_wide_reads_wider_than_the_staging_window():
    # tiles whose bytes exceed the shared-memory window read global memory
    long = [synth.codes_to_ascii(synth.random_genome(90_000, 5)),
            synth.codes_to_ascii(synth.random_genome(70_001, 6))]
    rs = synth.from_strings(long + ["ACGT" * 30], 51, lead=3)
    assert_same_graph(gpu_export(rs), oracle_export(rs))


def test_wide_repeats_and_homopolymers():
    reads = ["A" * 200, "AC" * 80, "ACGT" * 60, "GATTACA" * 30, "T" * 64, "TTTTG" * 40]
    for k in (33, 51, 64):
        rs = synth.from_strings(reads * 20, k, lead=2)
        assert_same_graph(gpu_export(rs), oracle_export(rs))


def test_wide_two_calls_host_input_and_batches():
    import torch
    a = synth.ragged_reads(800, 160, 45, 8100)
    b = synth.ragged_reads(900, 170, 45, 8101)
    both = synth.from_strings([a.read_ascii(r) for r in range(a.n_reads)] +
                              [b.read_ascii(r) for r in range(b.n_reads)], 45)
    g = dbg.Graph(45, capacity_for(both))
    pa, oa = to_device(a)
    g.insert(pa, oa)
    g.insert_host(b.packed, b.offsets)
    assert g.status() == dbg.OK
    assert_same_graph(g.export(), oracle_export(both))
    assert g.stats() == (len(oracle_export(both)[0]), both.n_edges())
    g.close()
    # a batch mixing 64-bit and 128-bit keys
    sets = [synth.ragged_reads(300, 150, k, 8200 + k) for k in (21, 51, 31, 33, 64)]
    gs = [dbg.Graph(rs.k, capacity_for(rs)) for rs in sets]
    dev = [to_device(rs) for rs in sets]
    dbg.insert_batch([(g, pk, of) for g, (pk, of) in zip(gs, dev)])
    torch.cuda.synchronize()
    for g, rs in zip(gs, sets):
        assert_same_graph(g.export(), oracle_export(rs))
        g.close()


def test_wide_overflow_normalize_and_refusals():
    rs = synth.ragged_reads(1500, 150, 51, 8300)
    g = dbg.Graph(51, 1000)  # far too small
    pk, of = to_device(rs)
    g.insert(pk, of)
    assert g.status() == dbg.ERR_CAPACITY
    g.close()
    g = dbg.Graph(51, capacity_for(rs))
    g.insert(pk, of)
    o = oracle.build_graph(rs.packed, rs.offsets, 51)
    div = 0.7
    g.normalize(div)
    keys, counts = g.export()
    assert np.array_equal(keys, o.keys) and np.array_equal(counts, oc.normalize(o.counts, div))
    with pytest.raises(dbg.DbgError):
        g.set_spill(1000)
    with pytest.raises(dbg.DbgError):
        g.grow()
    with pytest.raises(dbg.DbgError):
        g.contigs()
    g.close()
