"""Normalization and contigs (Section "Normalization of graph", Section
"Finding contigs", Alg. 5) on the GPU against the oracle, exactly: the
normalized counters bit for bit, the contigs string for string in order."""

import numpy as np
import pytest

import oracle
from gpu_util import gpu_graph
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


def oracle_contigs(rs, divisor=None):
    g = oracle.build_graph(rs.packed, rs.offsets, rs.k)
    counts = g.counts if divisor is None else oc.normalize(g.counts, divisor)
    return g.keys, counts, oc.find_contigs(g.keys, counts, rs.k)


def gpu_contigs(rs, divisor=None, **kw):
    g = gpu_graph(rs, **kw)
    assert g.status() == dbg.OK
    if divisor is not None:
        g.normalize(divisor)
    keys, counts = g.export()
    out = g.contigs()
    g.close()
    return keys, counts, out


def test_hand_worked_cases():
    cases = [("ACGACGACGC", 4, ["ACGACG", "ACGC"]), ("GGACGTACGTA", 4, ["GGACGTACG"]),
             ("ACGTACGTA", 4, [])]
    for read, k, expect in cases:
        rs = synth.from_strings([read], k)
        assert gpu_contigs(rs)[2] == expect


@pytest.mark.parametrize("k", [2, 3, 4, 7, 15, 21, 31, 32])
def test_raw_graph_contigs_match_oracle(k):
    rs = synth.ragged_reads(1500, 200, k, 5100 + k, lead=k % 4)
    assert gpu_contigs(rs)[2] == oracle_contigs(rs)[2]


def test_cycles_and_repeats():
    reads = ["A" * 60, "ACACACACACACACACAC", "ACGTACGTACGTACGT", "TTTTGGACGTACGTACGTA",
             "GATTACA" * 9, "CCCCCCCCCCCGGGGGGGGGGG"]
    for k in (3, 4, 5, 8):
        rs = synth.from_strings(reads, k, lead=1)
        assert gpu_contigs(rs)[2] == oracle_contigs(rs)[2]


@pytest.mark.parametrize("seed", [0, 1])
def test_normalized_sample_counts_and_contigs_match_oracle(seed):
    rs = synth.batch_sample(seed, 61, gmax=1.2e5)
    div = oc.divisor(rs.n_edges(), rs.meta["genome_len"])
    keys, counts, contigs = oracle_contigs(rs, div)
    gk, gc, gcon = gpu_contigs(rs, div)
    assert np.array_equal(gk, keys) and np.array_equal(gc, counts)
    assert gcon == contigs
    assert len(contigs) > 0


def test_normalized_10kb_workload():
    rs = synth.workload_10kb()
    div = oc.divisor(rs.n_edges(), 10_000)
    keys, counts, contigs = oracle_contigs(rs, div)
    gk, gc, gcon = gpu_contigs(rs, div)
    assert np.array_equal(gc, counts) and gcon == contigs


def test_normalization_rounding_edges():
    # counters around the rounding boundary: c / 2.5 + 0.5 for c = 0..40
    reads = ["ACGTTGCA" + "C" * 3] * 40
    rs = synth.from_strings(reads, 5)
    for div in (2.5, 3.0, 7.0, 0.75, 1e-3):
        _, counts, _ = oracle_contigs(rs, div)
        _, gc, _ = gpu_contigs(rs, div)
        assert np.array_equal(gc, counts), div


def test_size_query_and_errors():
    import ctypes
    rs = synth.ragged_reads(500, 120, 11, 5300)
    g = gpu_graph(rs)
    L = dbg.load()
    n, b = ctypes.c_uint64(), ctypes.c_uint64()
    assert L.dbg_find_contigs(g.handle, None, 0, None, 0, ctypes.byref(n), ctypes.byref(b),
                              None) == dbg.ERR_BUFFER_TOO_SMALL
    expect = oracle_contigs(rs)[2]
    assert n.value == len(expect) and b.value == sum(len(c) for c in expect)
    assert L.dbg_normalize(g.handle, 0.0, None) == dbg.ERR_INVALID_ARG
    assert L.dbg_normalize(g.handle, float("nan"), None) == dbg.ERR_INVALID_ARG
    # contigs can be found twice; the graph is unchanged by it
    assert g.contigs() == expect and g.contigs() == expect
    g.close()
    empty = dbg.Graph(11, 1000)
    assert empty.contigs() == []
    empty.close()
