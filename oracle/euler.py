"""Eulerian path over an A-Bruijn graph -- TEST INFRASTRUCTURE ONLY.

The paper states that the assembly output is an Eulerian path over the graph,
each edge being used as many times as its counter says (Section "Background",
Fig. 1 caption).  It gives no algorithm for it, so this is Hierholzer's
algorithm over the multigraph whose edge v -> u (u = v without its first
base, plus label b) has multiplicity ``counts[v][b]``.

Readings taken: the path starts at the vertex with out-degree minus
in-degree equal to +1, or, when every vertex is balanced (an Eulerian
circuit), at the smallest key with an out-edge; among several unused edges
the lowest label (A < C < G < T) is taken first, which makes the result
deterministic.  ``None`` is returned when no Eulerian path exists (unbalanced
degrees, or edges not all reachable).
"""

from __future__ import annotations

import numpy as np


def eulerian_path(keys: np.ndarray, counts: np.ndarray, k: int) -> list[int] | None:
    m = k - 1
    mask = (1 << (2 * m)) - 1
    rem = {int(v): [int(x) for x in c] for v, c in zip(keys, counts)}
    indeg: dict[int, int] = {v: 0 for v in rem}
    n_edges = 0
    for v, c in rem.items():
        for b in range(4):
            if c[b]:
                u = ((v << 2) | b) & mask
                if u not in indeg:
                    return None  # an edge points at a vertex that does not exist
                indeg[u] += c[b]
                n_edges += c[b]
    if n_edges == 0:
        return []
    start = None
    plus = minus = 0
    for v in sorted(rem):
        d = sum(rem[v]) - indeg[v]
        if d == 1:
            plus += 1
            start = v
        elif d == -1:
            minus += 1
        elif d != 0:
            return None
    if plus > 1 or minus > 1 or plus != minus:
        return None
    if start is None:
        start = min(v for v in rem if sum(rem[v]) > 0)
    stack = [start]
    path: list[int] = []
    while stack:
        v = stack[-1]
        c = rem[v]
        for b in range(4):
            if c[b]:
                c[b] -= 1
                stack.append(((v << 2) | b) & mask)
                break
        else:
            path.append(stack.pop())
    path.reverse()
    if len(path) != n_edges + 1:
        return None  # some edges are not reachable from the start
    return path


def spell(path: list[int], k: int) -> str:
    """The string a vertex path spells: the first vertex, then the last base
    of every following vertex."""
    if not path:
        return ""
    m = k - 1
    first = "".join("ACGT"[(path[0] >> (2 * (m - 1 - j))) & 3] for j in range(m))
    return first + "".join("ACGT"[v & 3] for v in path[1:])
