"""Pins for the CPU oracle: each test checks it against something that does not
come from the oracle itself -- the paper's Fig. 1 example, brute force on
small inputs, the k=2 closed form, invariants of the construction and the
Eulerian re-spelling of reads.  No GPU needed."""

import itertools
import os

import numpy as np
import pytest

import oracle
from paper_2401_02756_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def load_golden(name):
    read, k, rows = None, None, {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            parts = line.split()
            if parts[0] == "read":
                read = parts[1]
            elif parts[0] == "k":
                k = int(parts[1])
            else:
                rows[parts[0]] = tuple(int(x) for x in parts[1:5])
    return read, k, rows


def brute_force(reads, k):
    """Definition written as a list scan, O(vertices x edges): every k-substring
    is an edge prefix -> suffix; the prefix counts its last letter."""
    kmers = [r[j:j + k] for r in reads for j in range(len(r) - k + 1)]
    verts = sorted(set([x[:-1] for x in kmers] + [x[1:] for x in kmers]))
    return {v: tuple(sum(1 for x in kmers if x[:-1] == v and x[-1] == b) for b in "ACGT")
            for v in verts}


def oracle_dict(reads, k, lead=0, **kw):
    rs = synth.from_strings(reads, k, lead=lead)
    g = oracle.build_graph(rs.packed, rs.offsets, k, strings=True, **kw)
    return g.as_dict(), g


# --------------------------------------------------------------------------
# the paper's worked example
# --------------------------------------------------------------------------

def test_fig1_golden():
    read, k, rows = load_golden("fig1_acgacgacgc_k4.txt")
    assert (read, k) == ("ACGACGACGC", 4)
    d, g = oracle_dict([read], k)
    assert d == rows
    # the vertex set printed with the paper's Fig. 3 caption
    assert set(d) == {"ACG", "CGC", "CGA", "GAC"}
    assert list(d) == sorted(d)  # A<C<G<T order


def test_fig1_eulerian_path_respells_read():
    read, k, _ = load_golden("fig1_acgacgacgc_k4.txt")
    _, g = oracle_dict([read], k)
    path = oracle.eulerian_path(g.keys, g.counts, k)
    assert oracle.spell(path, k) == read
    # unique: ACG->CGC first would dead-end, so the path is forced
    assert [oracle.decode_key(v, k) for v in path] == \
        ["ACG", "CGA", "GAC", "ACG", "CGA", "GAC", "ACG", "CGC"]


# --------------------------------------------------------------------------
# brute force
# --------------------------------------------------------------------------

@pytest.mark.parametrize("k", [2, 3, 4])
def test_every_single_read_up_to_len5(k):
    for L in range(0, 6):
        for t in itertools.product("ACGT", repeat=L):
            r = "".join(t)
            d, _ = oracle_dict([r], k)
            assert d == brute_force([r], k), r


@pytest.mark.parametrize("k", [2, 3, 4])
@pytest.mark.parametrize("L", [6, 7])
def test_all_reads_of_length_as_one_set(k, L):
    reads = ["".join(t) for t in itertools.product("ACGT", repeat=L)]
    d, _ = oracle_dict(reads, k, lead=3)
    assert d == brute_force(reads, k)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_random_ragged_vs_brute_force(seed):
    rs = synth.ragged_reads(60, 40, 5, seed, lead=seed)
    reads = [rs.read_ascii(r) for r in range(rs.n_reads)]
    for k in (2, 5, 9):
        g = oracle.build_graph(rs.packed, rs.offsets, k, strings=True)
        assert g.as_dict() == brute_force(reads, k)


@pytest.mark.parametrize("lead", [0, 1, 2, 3, 5])
def test_unpack_every_bit_position(lead):
    # k = read length: exactly one edge, prefix -> suffix, counting the last letter
    rng = np.random.default_rng(lead)
    for L in (2, 3, 7, 31, 32):
        r = "".join(rng.choice(list("ACGT"), size=L))
        d, _ = oracle_dict([r], L, lead=lead)
        exp = {r[:-1]: [0, 0, 0, 0], r[1:]: [0, 0, 0, 0]}
        exp[r[:-1]]["ACGT".index(r[-1])] += 1
        assert d == {v: tuple(c) for v, c in exp.items()}


def test_key_encoding_matches_strings():
    rs = synth.ragged_reads(50, 80, 31, 7)
    for k in (2, 17, 31, 32):
        g = oracle.build_graph(rs.packed, rs.offsets, k, strings=True)
        assert [oracle.decode_key(x, k) for x in g.keys] == g.strings
        assert all(int(a) < int(b) for a, b in zip(g.keys[:-1], g.keys[1:]))
        if k == 32:  # 62-bit keys never reach the all-ones word
            assert int(g.keys.max()) < (1 << 62)


# --------------------------------------------------------------------------
# closed form at k = 2: vertices are bases, counters are dinucleotide counts
# --------------------------------------------------------------------------

@pytest.mark.parametrize("seed", [11, 12])
def test_k2_closed_form(seed):
    rs = synth.ragged_reads(300, 60, 2, seed)
    M = np.zeros((4, 4), dtype=np.int64)
    present = np.zeros(4, dtype=bool)
    for r in range(rs.n_reads):
        a, b = int(rs.offsets[r]), int(rs.offsets[r + 1])
        c = rs.codes[a:b].astype(np.int64)
        if c.size >= 2:
            np.add.at(M, (c[:-1], c[1:]), 1)
            present[c] = True
    g = oracle.build_graph(rs.packed, rs.offsets, 2)
    assert list(g.keys) == [i for i in range(4) if present[i]]
    assert np.array_equal(g.counts.astype(np.int64), M[present])


# --------------------------------------------------------------------------
# invariants
# --------------------------------------------------------------------------

def _in_degrees(keys, counts, k):
    m = k - 1
    mask = (1 << (2 * m)) - 1
    ind = {int(v): 0 for v in keys}
    for v, c in zip(keys, counts):
        for b in range(4):
            if c[b]:
                ind[((int(v) << 2) | b) & mask] += int(c[b])
    return ind


@pytest.mark.parametrize("k", [3, 8, 21, 31, 32])
def test_invariants_ragged(k):
    rs = synth.ragged_reads(400, 120, k, 100 + k, lead=k % 4)
    g = oracle.build_graph(rs.packed, rs.offsets, k)
    ln = rs.lengths()
    assert int(g.counts.astype(np.int64).sum()) == int(np.maximum(ln - k + 1, 0).sum())
    assert g.n_vertices <= int(np.maximum(ln - k + 2, 0).sum())
    ind = _in_degrees(g.keys, g.counts, k)   # raises if a target is missing
    out = {int(v): int(c.sum()) for v, c in zip(g.keys, g.counts)}
    starts, ends = {}, {}
    for r in range(rs.n_reads):
        s = rs.read_ascii(r)
        if len(s) >= k:
            key_s = sum("ACGT".index(ch) << (2 * (k - 2 - i)) for i, ch in enumerate(s[:k - 1]))
            key_e = sum("ACGT".index(ch) << (2 * (k - 2 - i)) for i, ch in enumerate(s[-(k - 1):]))
            starts[key_s] = starts.get(key_s, 0) + 1
            ends[key_e] = ends.get(key_e, 0) + 1
    for v in out:
        assert out[v] - ind[v] == starts.get(v, 0) - ends.get(v, 0)


def test_10kb_workload_distinct_bound():
    rs = synth.workload_10kb()
    g = oracle.build_graph(rs.packed, rs.offsets, rs.k)
    assert int(g.counts.astype(np.int64).sum()) == rs.n_edges() == 80_000
    # error-free reads of a 10 kb genome: at most 10,000 - 20 + 1 distinct 20-mers
    assert g.n_vertices <= 9_981
    # every vertex is a substring of the genome
    gen = synth.codes_to_ascii(rs.meta["genome"])
    gset = {gen[i:i + 20] for i in range(len(gen) - 19)}
    assert all(oracle.decode_key(x, 21) in gset for x in g.keys[:500])


# --------------------------------------------------------------------------
# Eulerian re-spelling
# --------------------------------------------------------------------------

@pytest.mark.parametrize("seed", [1, 2, 3, 4])
def test_single_error_free_read_is_respelled(seed):
    g0 = synth.random_genome(400, seed)
    s = synth.codes_to_ascii(g0)
    k = 21
    assert len({s[i:i + k - 1] for i in range(len(s) - k + 2)}) == len(s) - k + 2
    _, g = oracle_dict([s], k)
    assert oracle.spell(oracle.eulerian_path(g.keys, g.counts, k), k) == s


def test_eulerian_path_with_repeats_uses_every_edge():
    s = "ACGTACGTTTACGTACGAAACGT"
    k = 4
    _, g = oracle_dict([s], k)
    path = oracle.eulerian_path(g.keys, g.counts, k)
    E = int(g.counts.sum())
    assert len(path) == E + 1
    assert len(oracle.spell(path, k)) == E + k - 1
    used = {}
    for a, b in zip(path, path[1:]):
        used[(a, b & 3)] = used.get((a, b & 3), 0) + 1
    exp = {(int(v), bb): int(c[bb]) for v, c in zip(g.keys, g.counts) for bb in range(4) if c[bb]}
    assert used == exp


def test_eulerian_path_absent_for_two_disjoint_reads():
    _, g = oracle_dict(["AAAAC", "GGGGT"], 3)
    assert oracle.eulerian_path(g.keys, g.counts, 3) is None


# --------------------------------------------------------------------------
# sharding and threads are exact partitions of the same graph
# --------------------------------------------------------------------------

def test_shards_and_threads_partition_the_graph():
    rs = synth.ragged_reads(500, 150, 21, 77, lead=2)
    full = oracle.build_graph(rs.packed, rs.offsets, 21)
    thr = oracle.build_graph(rs.packed, rs.offsets, 21, threads=4)
    assert np.array_equal(full.keys, thr.keys) and np.array_equal(full.counts, thr.counts)
    parts = [oracle.build_graph(rs.packed, rs.offsets, 21, shard_mod=5, shard_id=p) for p in range(5)]
    keys = np.concatenate([p.keys for p in parts])
    cnts = np.concatenate([p.counts for p in parts])
    o = np.argsort(keys)
    assert np.array_equal(keys[o], full.keys) and np.array_equal(cnts[o], full.counts)
    sh = oracle.shard_of_keys(full.keys, 21, 5)
    for p in range(5):
        assert np.array_equal(full.keys[sh == p], parts[p].keys)


def test_invalid_arguments_rejected():
    rs = synth.from_strings(["ACGT"], 3)
    for k in (1, 33):
        with pytest.raises(RuntimeError):
            oracle.build_graph(rs.packed, rs.offsets, k)
    with pytest.raises(RuntimeError):
        oracle.build_graph(rs.packed, np.array([4, 0], dtype=np.uint64), 3)


# --------------------------------------------------------------------------
# the sketch used to size tables (HyperLogLog of the vertex keys)
# --------------------------------------------------------------------------

def test_sketch_depends_only_on_the_distinct_keys():
    rs = synth.ragged_reads(300, 150, 21, 901)
    reads = [rs.read_ascii(r) for r in range(rs.n_reads)]
    twice = synth.from_strings(reads + reads[::-1], 21, lead=3)
    assert np.array_equal(oracle.sketch(rs.packed, rs.offsets, 21),
                          oracle.sketch(twice.packed, twice.offsets, 21))


def test_sketch_of_a_single_vertex():
    rs = synth.from_strings(["A" * 60, "A" * 25], 21)  # every vertex is A^20
    regs = oracle.sketch(rs.packed, rs.offsets, 21)
    assert np.count_nonzero(regs) == 1 and 1 <= regs.max() <= 55
    assert oracle.sketch(synth.from_strings(["ACG"], 21).packed,
                         synth.from_strings(["ACG"], 21).offsets, 21).max() == 0


@pytest.mark.parametrize("n,seed", [(40, 1), (600, 2), (6000, 3)])
def test_sketch_estimate_within_the_hyperloglog_error(n, seed):
    rs = synth.ragged_reads(n, 200, 25, 950 + seed)
    D = oracle.build_graph(rs.packed, rs.offsets, 25).n_vertices
    est = oracle.hll_estimate(oracle.sketch(rs.packed, rs.offsets, 25))
    # standard error 1.04 / sqrt(1024) = 3.25 %; four of them
    assert abs(est - D) <= 0.13 * D, (est, D)
