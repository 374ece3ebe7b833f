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
    for k in (1, 65):  # keys of up to 63 bases (k <= 64)
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


# --------------------------------------------------------------------------
# the capacity predictor's network (FP64 reference)
# --------------------------------------------------------------------------

from oracle import mlp  # noqa: E402


def _mlp_case(seed: int, batch: int, scale: float = 1.0):
    rng = np.random.default_rng(seed)
    blocks = {"W1": rng.uniform(-1, 1, (mlp.HID, mlp.IN)) * np.sqrt(6 / mlp.IN) * scale,
              "b1": rng.normal(0, 0.1, mlp.HID), "W2": rng.uniform(-1, 1, (mlp.HID, mlp.HID))
              * np.sqrt(6 / mlp.HID), "b2": rng.normal(0, 0.1, mlp.HID),
              "w3": rng.uniform(-1, 1, mlp.HID) * np.sqrt(6 / mlp.HID), "b3": 0.3}
    x = rng.integers(0, 25, (batch, mlp.IN)) / 64.0
    t = rng.normal(12.0, 2.0, batch)
    return mlp.pack(blocks), x, t


def test_mlp_layout_round_trips():
    p, _, _ = _mlp_case(1, 1)
    assert p.size == mlp.N_PARAMS == 69825
    assert np.array_equal(mlp.pack(mlp.unpack(p)), p)


def test_mlp_single_path_closed_form():
    # one unit per layer: y = w3 * relu(W2 * relu(W1 x0 + b1) + b2) + b3
    q = {n: np.zeros_like(a) for n, a in mlp.unpack(np.zeros(mlp.N_PARAMS)).items()}
    q["W1"][5, 7], q["b1"][5], q["W2"][9, 5], q["b2"][9], q["w3"][9], q["b3"] = 2, -1, 3, 0.5, 4, 0.25
    x = np.zeros((3, mlp.IN))
    x[:, 7] = [0.0, 0.75, 2.0]
    y, _ = mlp.forward(mlp.pack(q), x)
    expect = [4 * max(0.0, 3 * max(0.0, 2 * v - 1) + 0.5) + 0.25 for v in (0.0, 0.75, 2.0)]
    assert np.allclose(y, expect, rtol=0, atol=1e-12)


def test_mlp_zero_weights_gradient_is_the_bias_residual():
    p = np.zeros(mlp.N_PARAMS)
    p[-1] = 1.5
    x = np.random.default_rng(2).random((5, mlp.IN))
    t = np.array([1.0, 2.0, 3.0, 4.0, 5.0])
    l, g = mlp.loss_and_grads(p, x, t)
    assert l == pytest.approx(0.5 * np.mean((1.5 - t) ** 2))
    assert g[-1] == pytest.approx(np.mean(1.5 - t))
    assert not np.any(g[:-1])


@pytest.mark.parametrize("seed", [3, 4])
def test_mlp_gradients_match_finite_differences(seed):
    p, x, t = _mlp_case(seed, 7)
    _, g = mlp.loss_and_grads(p, x, t)
    rng = np.random.default_rng(seed)
    # indices from every block (W1, b1, W2, b2, w3, b3)
    bounds = np.cumsum([0, mlp.HID * mlp.IN, mlp.HID, mlp.HID * mlp.HID, mlp.HID, mlp.HID, 1])
    idx = np.concatenate([rng.integers(bounds[i], bounds[i + 1], 12) for i in range(6)])
    h = 1e-6
    for i in idx:
        e = np.zeros_like(p)
        e[i] = h
        fd = (mlp.loss(p + e, x, t) - mlp.loss(p - e, x, t)) / (2 * h)
        assert fd == pytest.approx(g[i], rel=1e-5, abs=1e-7), i


def test_adam_first_step_moves_each_parameter_by_lr():
    # m_hat = g and v_hat = g^2 after one step, so the move is lr * g / (|g| + eps)
    g = np.array([3.0, -0.5, 0.0, 1e-3])
    p1, m, v = mlp.adam_step(np.ones(4), g, np.zeros(4), np.zeros(4), 1, 0.01)
    assert np.allclose(p1, 1 - 0.01 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)
    # a constant gradient keeps m_hat / sqrt(v_hat) = sign(g) at every step
    p, m, v = np.zeros(1), np.zeros(1), np.zeros(1)
    for s in range(1, 6):
        p, m, v = mlp.adam_step(p, np.array([2.0]), m, v, s, 0.1)
    assert p[0] == pytest.approx(-0.5, rel=1e-8)


def test_abs_forward_bounds_the_network():
    p, x, _ = _mlp_case(5, 9)
    y, _ = mlp.forward(p, x)
    assert np.all(np.abs(y) <= mlp.abs_forward(p, x) + 1e-12)


# --------------------------------------------------------------------------
# the first flag, normalization and contigs (Section "Normalization of
# graph", Section "Finding contigs", Alg. 5)
# --------------------------------------------------------------------------

from oracle import contigs as oc  # noqa: E402


def load_contig_cases():
    cases, cur = [], None
    with open(os.path.join(GOLDEN, "contigs_k4.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            if line.startswith("case "):
                _, read, k = line.split()
                cur = (read, int(k), [])
                cases.append(cur)
            else:
                cur[2].append(line)
    return cases


def graph_of(reads, k):
    rs = synth.from_strings(reads, k)
    return oracle.build_graph(rs.packed, rs.offsets, k)


@pytest.mark.parametrize("case", range(3))
def test_contigs_of_hand_worked_graphs(case):
    read, k, expect = load_contig_cases()[case]
    g = graph_of([read], k)
    assert oc.find_contigs(g.keys, g.counts, k) == expect
    assert oc.find_contigs(g.keys, g.counts, k, g.first) == expect


def test_fig1_has_no_first_vertex():
    g = graph_of(["ACGACGACGC"], 4)
    assert not g.first.any()
    g = graph_of(["GGACGTACGTA"], 4)
    assert [oc.decode(key, 3) for key in g.keys[g.first.astype(bool)]] == ["GGA"]


@pytest.mark.parametrize("k,seed", [(3, 1), (5, 2), (21, 3)])
def test_first_flag_is_zero_in_degree(k, seed):
    # the paper sets first on a vertex created as a left vertex and clears it
    # whenever the vertex is a right vertex: whatever the order, it ends up
    # set exactly on vertices that are no k-mer's suffix
    rs = synth.ragged_reads(400, 60, k, 3100 + seed)
    reads = [rs.read_ascii(r) for r in range(rs.n_reads)]
    suffixes = {r[j + 1:j + k] for r in reads for j in range(len(r) - k + 1)}
    g = oracle.build_graph(rs.packed, rs.offsets, k, strings=True)
    for s, f in zip(g.strings, g.first):
        assert bool(f) == (s not in suffixes)
    assert np.array_equal(oc.first_flags(g.keys, g.counts, k), g.first)


def test_tiled_error_free_genome_is_one_contig():
    # error-free reads tiling a random genome with no repeated 20-mer: the
    # graph is one path from the genome's first 20-mer, which is one contig
    # spelling the genome
    codes = synth.random_genome(5000, 77)
    genome = synth.codes_to_ascii(codes)
    k = 21
    assert len({genome[i:i + k - 1] for i in range(len(genome) - k + 2)}) == len(genome) - k + 2
    reads = [genome[s:s + 100] for s in range(0, len(genome) - 100 + 1, 37)] + [genome[-100:]]
    g = graph_of(reads, k)
    assert oc.find_contigs(g.keys, g.counts, k) == [genome]
    assert g.first.sum() == 1


@pytest.mark.parametrize("k,seed", [(4, 5), (7, 6), (15, 7)])
def test_contig_walk_invariants(k, seed):
    rs = synth.ragged_reads(300, 80, k, 3200 + seed)
    g = oracle.build_graph(rs.packed, rs.offsets, k, strings=True)
    cnt = {s: c for s, c in zip(g.strings, g.counts)}
    first = {s: bool(f) for s, f in zip(g.strings, g.first)}

    def outs(v):
        return [b for i, b in enumerate("ACGT") if cnt[v][i] > 0]

    starts = [(v, b) for v in sorted(cnt) if first[v] or len(outs(v)) != 1 for b in outs(v)]
    got = oc.find_contigs(g.keys, g.counts, k)
    assert len(got) == len(starts)
    for c, (v, b) in zip(got, starts):
        assert c[:k] == v + b                       # one contig per start edge, in order
        vs = [c[i:i + k - 1] for i in range(len(c) - k + 2)]
        for i in range(len(vs) - 1):                # a walk along edges
            assert c[i + k - 1] in outs(vs[i])
        for i in range(1, len(vs) - 1):             # interior: one exit, not repeated
            assert len(outs(vs[i])) == 1 and vs[i] not in vs[:i]
        last = vs[-1]                               # the end: a branch, a dead end or a repeat
        assert len(outs(last)) != 1 or last in vs[:-1]


def test_normalization_rounds_to_nearest():
    # floor(c / 2.5 + 0.5) worked by hand for c = 0..10
    c = np.arange(11, dtype=np.uint32).reshape(-1, 1)
    assert oc.normalize(c, 2.5).ravel().tolist() == [0, 0, 1, 1, 2, 2, 2, 3, 3, 4, 4]
    # the 10 kb workload: 1000 reads x (100 - 21 + 1) / 10000 = 8
    rs = synth.workload_10kb()
    assert oc.divisor(rs.n_edges(), 10_000) == 8.0
    big = np.array([[2 ** 32 - 1, 7, 0, 1]], dtype=np.uint32)
    assert oc.normalize(big, 0.5).tolist() == [[2 ** 32 - 1, 14, 0, 2]]


def test_normalization_removes_errors_and_keeps_the_genome():
    # 30x error-free tiling plus a few reads with one substitution each: the
    # normalized graph has only the genome's edges, which spell one contig
    codes = synth.random_genome(3000, 91)
    genome = synth.codes_to_ascii(codes)
    k = 25
    reads = []
    for rep in range(30):
        reads += [genome[s:s + 150] for s in range(rep, len(genome) - 150 + 1, 30)]
    reads.append(genome[-150:])
    reads.append(genome[:150])
    bad = list(genome[500:650])
    bad[70] = "A" if bad[70] != "A" else "C"
    reads.append("".join(bad))
    rs = synth.from_strings(reads, k)
    g = oracle.build_graph(rs.packed, rs.offsets, k)
    norm = oc.normalize(g.counts, oc.divisor(rs.n_edges(), len(genome)))
    assert not np.array_equal(norm > 0, g.counts > 0)  # the error's k-mers are gone
    got = oc.find_contigs(g.keys, norm, k)
    # the genome minus its thinly covered ends, in one piece
    assert len(got) == 1 and got[0] in genome and len(got[0]) > len(genome) - 150


# --------------------------------------------------------------------------
# k > 32 (the paper's default k = 51): 128-bit keys
# --------------------------------------------------------------------------

@pytest.mark.parametrize("k", [33, 40, 51, 64])
def test_wide_k_matches_brute_force(k):
    rs = synth.ragged_reads(40, 2 * k, k, 600 + k, lead=k % 4)
    reads = [rs.read_ascii(r) for r in range(rs.n_reads)]
    g = oracle.build_graph(rs.packed, rs.offsets, k, strings=True)
    assert g.as_dict() == brute_force(reads, k)


@pytest.mark.parametrize("k", [33, 51, 64])
def test_wide_keys_encode_the_strings_in_order(k):
    rs = synth.ragged_reads(60, 150, k, 700 + k)
    g = oracle.build_graph(rs.packed, rs.offsets, k, strings=True)
    assert g.keys.shape == (g.n_vertices, 2)
    assert [oracle.decode_key(x, k) for x in g.keys] == g.strings
    as_int = [(int(h) << 64) | int(lo) for h, lo in g.keys]
    assert all(a < b for a, b in zip(as_int[:-1], as_int[1:]))
    assert max(as_int) < (1 << (2 * (k - 1)))  # 126 bits at most: the high word is never all ones
    # the same vertices as a narrow build would have, by string (no truncation)
    ln = rs.lengths()
    assert int(g.counts.astype(np.int64).sum()) == int(np.maximum(ln - k + 1, 0).sum())


def test_paper_default_k51_single_read():
    # one random 400-base read (no repeated 50-mer): a path of 351 vertices
    read = synth.codes_to_ascii(synth.random_genome(400, 51))
    rs = synth.from_strings([read], 51)
    g = oracle.build_graph(rs.packed, rs.offsets, 51, strings=True)
    assert sorted(read[j:j + 50] for j in range(351)) == g.strings
    out = {s: int(c.sum()) for s, c in zip(g.strings, g.counts)}
    assert out[read[-50:]] == 0 and sum(out.values()) == 350
