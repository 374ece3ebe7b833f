"""Normalization and contigs on a built graph -- TEST INFRASTRUCTURE ONLY.

Plain Python over the oracle's sorted graph (``oracle.Graph``: keys, counters
and the ``first`` flags that the C builder sets while it inserts).

* :func:`divisor` and :func:`normalize` -- Section "Normalization of graph":
  every counter is divided by the number of k-mer duplicates, reads x
  (read length - k + 1) / genome size.  Readings: with reads of uneven length
  the numerator is the total number of k-mers (edges); the quotient is
  rounded to the nearest integer, halves up -- floor(count / divisor + 0.5)
  in IEEE double -- because the counters stay integers and an error k-mer
  seen once must fall to 0 while a genomic one seen about ``divisor`` times
  stays 1.
* :func:`first_flags` -- the flag of Section "Finding contigs": set when no
  edge of the graph points to the vertex.  The paper maintains it while
  inserting (set on a vertex created as a left vertex, cleared whenever the
  vertex is a right vertex), which on a built graph leaves it set exactly on
  vertices with no incoming edge; the C builder keeps it that way and the
  tests check the two agree.  Reading: after normalization has zeroed some
  counters, "an edge points to the vertex" means a nonzero counter does, so
  the flag is taken from the counters as they are when contigs are found.
* :func:`find_contigs` -- Section "Finding contigs", Alg. 5 findContigs and
  its makePath.  A vertex starts contigs when its first flag is set or when
  it does not have exactly one outgoing edge (onlyOnePath is false); it
  starts one contig per outgoing edge.  A contig follows edges while the
  vertex it reaches has exactly one outgoing edge.  Readings: an outgoing
  edge is a label with a nonzero counter; a vertex with no outgoing edge
  starts no contig (a contig holds at least one edge); the walk also stops
  on reaching a vertex it has already visited, keeping the edge into it (the
  paper's walk would not end on a cycle of single-exit vertices); contigs are
  listed by (start vertex key, label) so that the result is one list.

Pins in ``tests/test_oracle.py``: the Fig. 1 example derived by hand, a
hand-derived cycle example, an error-free tiling whose one contig re-spells
the genome, the first flag against brute-force in-degrees, and walk
invariants checked on random sets.
"""

from __future__ import annotations

import numpy as np

LETTERS = "ACGT"


def divisor(n_edges: int, genome_size: int) -> float:
    """The number of k-mer duplicates: total k-mers of the reads over the
    genome size (reads x (read length - k + 1) / genome size for reads of
    one length)."""
    return float(n_edges) / float(genome_size)


def normalize(counts: np.ndarray, div: float) -> np.ndarray:
    """floor(count / div + 0.5) for every counter, capped at 2^32 - 1."""
    q = np.floor(counts.astype(np.float64) / float(div) + 0.5)
    return np.minimum(q, float(2 ** 32 - 1)).astype(np.uint32)


def decode(key: int, m: int) -> str:
    return "".join(LETTERS[(int(key) >> (2 * (m - 1 - j))) & 3] for j in range(m))


def first_flags(keys: np.ndarray, counts: np.ndarray, k: int) -> np.ndarray:
    """1 where no nonzero counter of any vertex leads to the vertex."""
    mask = (1 << (2 * (k - 1))) - 1
    index = {int(key): i for i, key in enumerate(keys)}
    first = np.ones(len(keys), dtype=np.uint8)
    for i, key in enumerate(keys):
        for b in range(4):
            if counts[i][b] > 0:
                first[index[((int(key) << 2) | b) & mask]] = 0
    return first


def find_contigs(keys: np.ndarray, counts: np.ndarray, k: int,
                 first: np.ndarray | None = None) -> list[str]:
    """Contigs of a graph given as sorted keys and counters [D][4]; the first
    flags are taken from the counters unless given."""
    m = k - 1
    mask = (1 << (2 * m)) - 1
    if first is None:
        first = first_flags(keys, counts, k)
    index = {int(key): i for i, key in enumerate(keys)}
    out_labels = [[b for b in range(4) if counts[i][b] > 0] for i in range(len(keys))]

    def only_one_path(i: int) -> bool:
        return len(out_labels[i]) == 1

    contigs = []
    for i, key in enumerate(keys):                       # findContigs over the table
        if not (first[i] or not only_one_path(i)):
            continue
        for b in out_labels[i]:                          # makePath: one contig per edge
            seq = [decode(key, m), LETTERS[b]]
            visited = {i}
            t = index[((int(key) << 2) | b) & mask]
            while t not in visited and only_one_path(t):
                visited.add(t)
                c = out_labels[t][0]
                seq.append(LETTERS[c])
                t = index[((int(keys[t]) << 2) | c) & mask]
            contigs.append("".join(seq))
    return contigs
