"""The sketch kernel (HyperLogLog registers of the vertex keys) against the
oracle's own register computation, bit for bit, and the host estimator
against the oracle's formula."""

import numpy as np
import pytest

import oracle
from gpu_util import to_device
from paper_2401_02756_gb300 import build, dbg, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    build.build()
    dbg.load()


def gpu_sketch(rs, shift=0):
    packed, offsets = to_device(rs, shift=shift)
    regs = dbg.sketch(rs.k, packed, offsets).cpu().numpy().view(np.uint32)
    assert regs[-1] == dbg.OK
    return regs[:-1]


@pytest.mark.parametrize("k", [2, 5, 21, 31, 32])
def test_sketch_registers_match_oracle(k):
    rs = synth.ragged_reads(3000, 300, k, 1100 + k, lead=k % 3)
    assert np.array_equal(gpu_sketch(rs), oracle.sketch(rs.packed, rs.offsets, k))


def test_sketch_of_workloads_and_unaligned_input():
    rs = synth.workload_10kb()
    exp = oracle.sketch(rs.packed, rs.offsets, rs.k)
    assert np.array_equal(gpu_sketch(rs), exp)
    assert np.array_equal(gpu_sketch(rs, shift=5), exp)
    wide = synth.from_strings([synth.codes_to_ascii(synth.random_genome(90_000, 4))], 31)
    assert np.array_equal(gpu_sketch(wide), oracle.sketch(wide.packed, wide.offsets, 31))


def test_estimator_matches_the_formula_and_the_truth():
    rs = synth.ragged_reads(5000, 250, 31, 1200)
    regs = gpu_sketch(rs)
    est = dbg.sketch_estimate(regs)
    assert est == pytest.approx(oracle.hll_estimate(regs), rel=1e-12)
    D = oracle.build_graph(rs.packed, rs.offsets, 31).n_vertices
    assert abs(est - D) <= 0.13 * D


def test_batched_sketch_equals_one_by_one_and_oracle():
    import torch
    sets = [synth.ragged_reads(40 + 7 * i, 120, (21, 31, 5)[i % 3], 1300 + i, lead=i % 4)
            for i in range(260)]  # two launches of up to 256 items; mixed k
    sets[3] = synth.from_strings([], 21)  # an empty read set
    dev = [to_device(rs) for rs in sets]
    regs = torch.full((len(sets), dbg.SKETCH_REGISTERS + 1), 7, dtype=torch.int32, device="cuda")
    dbg.sketch_batch([(rs.k, pk, of, regs[i]) for i, (rs, (pk, of)) in enumerate(zip(sets, dev))])
    got = regs.cpu().numpy().view(np.uint32)
    for i, (rs, (pk, of)) in enumerate(zip(sets, dev)):
        assert got[i, -1] == dbg.OK
        one = dbg.sketch(rs.k, pk, of).cpu().numpy().view(np.uint32)
        assert np.array_equal(got[i], one)
        if i % 26 == 0:
            assert np.array_equal(got[i, :-1], oracle.sketch(rs.packed, rs.offsets, rs.k))
