"""Seeded synthetic read sets for the A-Bruijn graph build.

This module only *makes inputs*: genomes, reads sampled from them, and the
2-bit packed stream the library consumes.  It holds none of the method's
arithmetic (no k-mer, vertex, hash or count logic) and imports nothing else
from this package, so the CUDA path and the CPU oracle can both be fed from it
without sharing any code with each other.

Randomness is counter-based: every draw is ``SplitMix64(key + (i + 1) * GAMMA)``
for a per-purpose ``key`` derived from the seed, i.e. the output function of
Steele, Lea and Flood's SplitMix64 (OOPSLA 2014) evaluated at counter ``i``.
Any slice of any stream can therefore be regenerated independently, on any
machine, bit for bit.

Input format (the one the library reads):

* ``packed``: ``uint8``, four bases per byte, reads concatenated with no
  padding.  Base ``i`` of the stream sits in bits ``[2*(i%4), 2*(i%4)+1]`` of
  byte ``i // 4`` (least-significant pair first).  Codes are A=0, C=1, G=2,
  T=3.
* ``offsets``: ``uint64[n_reads + 1]`` in bases; read ``r`` is
  ``[offsets[r], offsets[r+1])`` of the stream.

Workload shapes follow the paper's experiments (Section "Data preparation":
reads sampled uniformly from a genome at a fixed coverage) with the sizes of
the five benchmark workloads: 10 kb error-free (k=21), 5 Mbp at 50x with 1 %
substitutions (k=31), 100 Mbp with 5 % repeats at 30x and 0.5 % substitutions
(k=31), and many small samples for the batched build.
"""

from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

GAMMA = 0x9E3779B97F4A7C15
_M1 = 0xBF58476D1CE4E5B9
_M2 = 0x94D049BB133111EB
_U = np.uint64
BASES = "ACGT"

# stream identifiers (one per purpose so that draws never overlap)
S_GENOME, S_START, S_ERRPOS, S_ERRVAL, S_LEN, S_FAMILY, S_COPYPOS, S_MUTPOS, \
    S_MUTVAL, S_SEGMENT, S_SAMPLE, S_ARRIVAL = range(1, 13)


def splitmix64(z: np.ndarray) -> np.ndarray:
    """SplitMix64 output function applied elementwise to uint64 states."""
    z = np.asarray(z, dtype=_U)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> _U(30))) * _U(_M1)
        z = (z ^ (z >> _U(27))) * _U(_M2)
        return z ^ (z >> _U(31))


def _stream_key(seed: int, stream: int) -> np.uint64:
    with np.errstate(over="ignore"):
        s = _U(seed & 0xFFFFFFFFFFFFFFFF) * _U(GAMMA) + _U(stream)
    return splitmix64(np.array([s], dtype=_U))[0]


def draws(seed: int, stream: int, n: int, start: int = 0) -> np.ndarray:
    """``n`` uint64 draws ``start .. start+n-1`` of stream ``stream``."""
    key = _stream_key(seed, stream)
    i = np.arange(start + 1, start + n + 1, dtype=_U)
    with np.errstate(over="ignore"):
        return splitmix64(key + i * _U(GAMMA))


def uniform_below(u: np.ndarray, m: int) -> np.ndarray:
    """floor(u * m / 2**64) for uint64 ``u`` and ``1 <= m < 2**63``: the high
    word of the exact 128-bit product, assembled from 32-bit partial products."""
    if not 1 <= m < (1 << 63):
        raise ValueError("m out of range")
    u = np.asarray(u, dtype=_U)
    lo32 = _U(0xFFFFFFFF)
    s32 = _U(32)
    m_lo, m_hi = _U(m & 0xFFFFFFFF), _U(m >> 32)
    u_lo, u_hi = u & lo32, u >> s32
    with np.errstate(over="ignore"):
        a = u_lo * m_lo
        b = u_hi * m_lo
        c = u_lo * m_hi
        d = u_hi * m_hi
        mid = (a >> s32) + (b & lo32) + (c & lo32)
        return (d + (b >> s32) + (c >> s32) + (mid >> s32)).astype(np.int64)


def uniform01(u: np.ndarray) -> np.ndarray:
    """53-bit uniform doubles in [0, 1)."""
    return (np.asarray(u, dtype=_U) >> _U(11)).astype(np.float64) * (1.0 / (1 << 53))


# ----------------------------------------------------------------------------
# sequences
# ----------------------------------------------------------------------------

def ascii_to_codes(s: str) -> np.ndarray:
    lut = np.full(256, 255, dtype=np.uint8)
    for i, c in enumerate(BASES):
        lut[ord(c)] = i
    c = lut[np.frombuffer(s.encode("ascii"), dtype=np.uint8)]
    if (c == 255).any():
        raise ValueError("sequence contains a symbol outside ACGT")
    return c


def codes_to_ascii(c: np.ndarray) -> str:
    return np.frombuffer(b"ACGT", dtype=np.uint8)[np.asarray(c, dtype=np.int64)].tobytes().decode()


def random_genome(length: int, seed: int) -> np.ndarray:
    """i.i.d. uniform ACGT codes; 32 bases are cut from each 64-bit draw."""
    nw = (length + 31) // 32
    w = draws(seed, S_GENOME, nw)
    shifts = (np.arange(32, dtype=_U) * _U(2))
    codes = ((w[:, None] >> shifts[None, :]) & _U(3)).astype(np.uint8).reshape(-1)
    return codes[:length].copy()


def repeat_genome(length: int, seed: int, repeat_fraction: float = 0.05,
                  segment: int = 1000, cmin: int = 2, cmax: int = 50,
                  copy_mutation_rate: float = 0.001) -> tuple[np.ndarray, dict]:
    """Uniform genome in which ``repeat_fraction`` of the sequence is made of
    ``segment``-bp repeat copies.

    Families have a copy number drawn log-uniformly from ``[cmin, cmax]``
    (rounded) until the repeat budget is used; each copy is the family's
    segment with ``round(copy_mutation_rate * segment)`` substitutions, and the
    copies go to distinct, random, segment-aligned positions.
    """
    g = random_genome(length, seed)
    nblocks = length // segment
    ncopies = int(round(repeat_fraction * length / segment))
    ncopies = min(ncopies, nblocks)
    # copy numbers, log-uniform in [cmin, cmax]
    fam_sizes: list[int] = []
    j = 0
    while sum(fam_sizes) < ncopies:
        u = uniform01(draws(seed, S_FAMILY, 1, start=j))[0]
        c = int(round(math.exp(math.log(cmin) + u * (math.log(cmax) - math.log(cmin)))))
        fam_sizes.append(max(cmin, min(cmax, c)))
        j += 1
    fam_sizes[-1] -= sum(fam_sizes) - ncopies
    if fam_sizes[-1] < 1:
        fam_sizes.pop()
    # distinct aligned positions: sort blocks by a random key
    perm = np.argsort(draws(seed, S_COPYPOS, nblocks), kind="stable")[:ncopies]
    nmut = int(round(copy_mutation_rate * segment))
    copy_id = 0
    for f, c in enumerate(fam_sizes):
        seg_codes = random_genome(segment, seed * 1000003 + 7919 * (f + 1) + S_SEGMENT)
        for _ in range(c):
            cp = seg_codes.copy()
            if nmut:
                mp = uniform_below(draws(seed, S_MUTPOS, nmut, start=copy_id * nmut), segment)
                mv = 1 + uniform_below(draws(seed, S_MUTVAL, nmut, start=copy_id * nmut), 3)
                cp[mp] = (cp[mp] + mv) & 3
            b = int(perm[copy_id])
            g[b * segment:(b + 1) * segment] = cp
            copy_id += 1
    return g, {"families": len(fam_sizes), "copies": ncopies, "segment": segment}


def pack_codes(codes: np.ndarray) -> np.ndarray:
    """Pack a code stream (values 0..3) four per byte, least-significant first."""
    c = np.asarray(codes, dtype=np.uint8)
    n = c.size
    pad = (-n) % 4
    if pad:
        c = np.concatenate([c, np.zeros(pad, dtype=np.uint8)])
    c = c.reshape(-1, 4)
    return (c[:, 0] | (c[:, 1] << 2) | (c[:, 2] << 4) | (c[:, 3] << 6)).astype(np.uint8)


# ----------------------------------------------------------------------------
# read sets
# ----------------------------------------------------------------------------

@dataclass
class ReadSet:
    """A packed read set plus the parameters it was made with."""

    name: str
    k: int
    packed: np.ndarray          # uint8
    offsets: np.ndarray         # uint64[n_reads + 1]
    meta: dict = field(default_factory=dict)
    codes: np.ndarray | None = None   # kept for small sets only (tests)

    @property
    def n_reads(self) -> int:
        return int(self.offsets.size - 1)

    @property
    def total_bases(self) -> int:
        return int(self.offsets[-1] - self.offsets[0])

    def lengths(self) -> np.ndarray:
        return np.diff(self.offsets.astype(np.int64))

    def n_edges(self) -> int:
        """Number of length-k substrings over all reads, sum(max(0, len-k+1))."""
        ln = self.lengths()
        return int(np.maximum(ln - self.k + 1, 0).sum())

    def read_ascii(self, r: int) -> str:
        if self.codes is None:
            raise ValueError("codes not kept for this read set")
        a, b = int(self.offsets[r] - self.offsets[0]), int(self.offsets[r + 1] - self.offsets[0])
        return codes_to_ascii(self.codes[a:b])


def from_strings(reads: list[str], k: int, name: str = "strings", lead: int = 0) -> ReadSet:
    """Read set from ASCII strings; ``lead`` bases of padding precede read 0
    (so that ``offsets[0] = lead`` exercises a non-zero first offset)."""
    parts = [np.zeros(lead, dtype=np.uint8)] + [ascii_to_codes(r) for r in reads]
    codes = np.concatenate(parts) if parts else np.zeros(0, dtype=np.uint8)
    lens = np.array([len(r) for r in reads], dtype=np.uint64)
    offsets = np.concatenate([[0], np.cumsum(lens)]).astype(np.uint64) + np.uint64(lead)
    return ReadSet(name, k, pack_codes(codes), offsets, {"lead": lead}, codes[lead:].copy())


def sample_reads(genome: np.ndarray, n_reads: int, read_len: int, error_rate: float,
                 seed: int, k: int, name: str, keep_codes: bool = False,
                 chunk_reads: int = 1 << 20) -> ReadSet:
    """Forward-strand reads of one length at uniform start positions in
    ``[0, G - read_len]``, with substitution errors.

    Errors: ``E = round(error_rate * total_bases)`` positions drawn uniformly
    (with replacement) over the read stream; each adds 1, 2 or 3 (uniform)
    to the base code modulo 4, so a substituted base is one of the other
    three, uniformly.
    """
    G = genome.size
    if read_len > G:
        raise ValueError("read longer than genome")
    total = n_reads * read_len
    starts = uniform_below(draws(seed, S_START, n_reads), G - read_len + 1)
    E = int(round(error_rate * total))
    if E:
        epos = uniform_below(draws(seed, S_ERRPOS, E), total)
        eval_ = (1 + uniform_below(draws(seed, S_ERRVAL, E), 3)).astype(np.uint8)
        order = np.argsort(epos, kind="stable")
        epos, eval_ = epos[order], eval_[order]
    else:
        epos = np.zeros(0, dtype=np.int64)
        eval_ = np.zeros(0, dtype=np.uint8)
    win = np.lib.stride_tricks.sliding_window_view(genome, read_len)
    cr = max(4, (chunk_reads // 4) * 4)
    packed_parts = []
    codes_parts = [] if keep_codes else None
    for r0 in range(0, n_reads, cr):
        r1 = min(n_reads, r0 + cr)
        c = win[starts[r0:r1]].reshape(-1).copy()
        b0, b1 = r0 * read_len, r1 * read_len
        lo, hi = np.searchsorted(epos, b0), np.searchsorted(epos, b1)
        if hi > lo:
            np.add.at(c, epos[lo:hi] - b0, eval_[lo:hi])
            c &= 3
        packed_parts.append(pack_codes(c))
        if keep_codes:
            codes_parts.append(c)
    packed = np.concatenate(packed_parts) if packed_parts else np.zeros(0, np.uint8)
    offsets = (np.arange(n_reads + 1, dtype=np.uint64) * np.uint64(read_len))
    meta = {"genome_len": int(G), "read_len": read_len, "error_rate": error_rate,
            "n_errors": E, "seed": seed}
    return ReadSet(name, k, packed, offsets, meta,
                   np.concatenate(codes_parts) if keep_codes and codes_parts else None)


def ragged_reads(n_reads: int, max_len: int, k: int, seed: int, lead: int = 0,
                 name: str = "ragged") -> ReadSet:
    """Reads of uniform random length in ``[0, max_len]`` with i.i.d. bases;
    includes empty reads and reads shorter than ``k``."""
    lens = uniform_below(draws(seed, S_LEN, n_reads), max_len + 1).astype(np.uint64)
    total = int(lens.sum())
    codes = random_genome(total + lead, seed ^ 0x5EED)
    offsets = (np.concatenate([[0], np.cumsum(lens)]).astype(np.uint64) + np.uint64(lead))
    return ReadSet(name, k, pack_codes(codes), offsets, {"max_len": max_len, "seed": seed},
                   codes[lead:].copy())


# ----------------------------------------------------------------------------
# the benchmark workloads
# ----------------------------------------------------------------------------

def fig1_example() -> ReadSet:
    """The paper's worked example (Fig. 1): the single read ACGACGACGC, k=4."""
    return from_strings(["ACGACGACGC"], 4, name="fig1")


def workload_10kb(seed: int = 1) -> ReadSet:
    """10 kb uniform genome, 1,000 error-free reads of 100 bp, k=21."""
    g = random_genome(10_000, seed)
    rs = sample_reads(g, 1000, 100, 0.0, seed, 21, "10kb_k21", keep_codes=True)
    rs.meta["genome"] = g
    return rs


def workload_5mbp(seed: int = 2) -> ReadSet:
    """5 Mbp uniform genome, 150 bp reads at 50x (1,666,667 reads), 1 % errors, k=31."""
    g = random_genome(5_000_000, seed)
    n = int(round(50 * 5_000_000 / 150))
    return sample_reads(g, n, 150, 0.01, seed, 31, "5mbp_50x_k31")


def workload_2mbp(seed: int = 6) -> ReadSet:
    """The 100 Mbp workload's reads at a fiftieth of its size, for profiling
    one kernel at a time: a 2 Mbp uniform genome, 150 bp reads at 30x
    (400,000 reads), 0.5 % errors, k=31 (a 0.46 GB table at 1.5x)."""
    g = random_genome(2_000_000, seed)
    return sample_reads(g, 400_000, 150, 0.005, seed, 31, "2mbp_30x_k31")


def workload_100mbp(seed: int = 3) -> ReadSet:
    """100 Mbp genome with 5 % 1-kb repeats (2-50 copies, 0.1 % mutations per
    copy), 150 bp reads at 30x (20,000,000 reads), 0.5 % errors, k=31."""
    g, info = repeat_genome(100_000_000, seed)
    rs = sample_reads(g, 20_000_000, 150, 0.005, seed, 31, "100mbp_30x_k31")
    rs.meta.update(info)
    return rs


def batch_sample(i: int, seed: int = 4, gmin: float = 5e4, gmax: float = 2e6,
                 cov_lo: float = 10.0, cov_hi: float = 60.0, read_len: int = 150,
                 error_rate: float = 0.005, ks=(21, 31)) -> ReadSet:
    """Sample ``i`` of the batched-build distribution: genome size log-uniform
    in ``[gmin, gmax]``, coverage uniform in ``[cov_lo, cov_hi]``, k drawn
    from ``ks``.  Each sample is a function of (seed, i) alone."""
    u = uniform01(draws(seed, S_SAMPLE, 3, start=3 * i))
    G = int(round(math.exp(math.log(gmin) + u[0] * (math.log(gmax) - math.log(gmin)))))
    cov = cov_lo + u[1] * (cov_hi - cov_lo)
    k = ks[min(len(ks) - 1, int(u[2] * len(ks)))]
    n = max(1, int(round(cov * G / read_len)))
    s = seed * 100_003 + i
    g = random_genome(G, s)
    rs = sample_reads(g, n, read_len, error_rate, s, k, f"sample{i}")
    rs.meta.update({"coverage": cov})
    return rs


def batch_sample_arrays(job: tuple) -> tuple:
    """(i, seed[, kwargs]) -> (i, k, packed, offsets, edges) of :func:`batch_sample`:
    a picklable form for worker processes."""
    i, seed = job[0], job[1]
    rs = batch_sample(i, seed, **(job[2] if len(job) > 2 else {}))
    return i, rs.k, rs.packed, rs.offsets, rs.n_edges()


def batch_samples(n_samples: int = 256, seed: int = 4, **kw) -> list[ReadSet]:
    """Samples 0 .. n_samples-1 of :func:`batch_sample`."""
    return [batch_sample(i, seed, **kw) for i in range(n_samples)]


def poisson_arrivals(n: int, rate: float, seed: int) -> np.ndarray:
    """Arrival times (seconds) of ``n`` requests of a Poisson process with the
    given rate: cumulative sums of exponential gaps -ln(1 - u) / rate."""
    u = uniform01(draws(seed, S_ARRIVAL, n))
    return np.cumsum(-np.log1p(-u) / rate)


WORKLOADS = {
    "fig1": fig1_example,
    "10kb_k21": workload_10kb,
    "5mbp_50x_k31": workload_5mbp,
    "2mbp_30x_k31": workload_2mbp,
    "100mbp_30x_k31": workload_100mbp,
}
