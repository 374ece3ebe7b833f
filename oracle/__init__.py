"""CPU oracle for the A-Bruijn graph build -- TEST INFRASTRUCTURE ONLY.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of the
benchmark may import this package.  The CUDA library never does, and the two
share no code: this package reads the same packed input and computes the
graph its own way (ASCII strings, a chained FNV-1a hash table, ``qsort``).

* :func:`build_graph` -- the plain C builder (``dbg_oracle.c``), following
  Section "Background" and Alg. 2-4 of the paper; see that file's header for
  the readings of the paper it takes.
* :func:`eulerian_path` / :func:`spell` -- Hierholzer's algorithm over the
  multigraph, backing the paper's statement that the assembly output is an
  Eulerian path over the graph (Section "Background").
* ``oracle.contigs`` -- normalization (Section "Normalization of graph") and
  contigs (Section "Finding contigs", Alg. 5), with the first flag that the C
  builder keeps while inserting (``Graph.first``).
* ``oracle.mlp`` -- the FP64 reference of the capacity predictor's network.

Every function here is pinned by ``tests/test_oracle.py`` against values that
do not come from the oracle itself (the Fig. 1 worked example, brute force,
the k=2 closed form, invariants).
"""

from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dbg_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc into ``oracle/liboracle.so``."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-pthread",
                               "-Wall", "-Wextra", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = ctypes.CDLL(_LIB)
    P, U64, I = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int
    lib.oracle_build.argtypes = [P, P, U64, I, U64, U64, I, ctypes.POINTER(P)]
    lib.oracle_build.restype = I
    lib.oracle_num_vertices.argtypes = [P]
    lib.oracle_num_vertices.restype = U64
    lib.oracle_export_sorted.argtypes = [P, P, P, U64]
    lib.oracle_export_sorted.restype = I
    lib.oracle_export_strings.argtypes = [P, P, U64]
    lib.oracle_export_strings.restype = I
    lib.oracle_free.argtypes = [P]
    lib.oracle_free.restype = None
    lib.oracle_shard_of_keys.argtypes = [P, U64, I, U64, P]
    lib.oracle_shard_of_keys.restype = None
    lib.oracle_sketch.argtypes = [P, P, U64, I, P]
    lib.oracle_sketch.restype = I
    lib.oracle_export_sorted_wide.argtypes = [P, P, P, U64]
    lib.oracle_export_sorted_wide.restype = I
    lib.oracle_export_first.argtypes = [P, P, U64]
    lib.oracle_export_first.restype = I
    _lib = lib
    return lib


@dataclass
class Graph:
    """Sorted vertices: ``keys`` (uint64, A=0 C=1 G=2 T=3, first base most
    significant; for k > 32 a [D, 2] array of the 128-bit key's high and low
    words) and ``counts`` (uint32 [D, 4], columns A, C, G, T)."""

    k: int
    keys: np.ndarray
    counts: np.ndarray
    strings: list[str] | None = None
    first: np.ndarray | None = None  # uint8 [D]: no edge points to the vertex

    @property
    def n_vertices(self) -> int:
        return int(self.keys.shape[0])

    def as_dict(self) -> dict:
        if self.strings is None:
            raise ValueError("strings were not requested")
        return {s: tuple(int(x) for x in c) for s, c in zip(self.strings, self.counts)}


def build_graph(packed: np.ndarray, offsets: np.ndarray, k: int, *, shard_mod: int = 1,
                shard_id: int = 0, threads: int = 1, strings: bool = False) -> Graph:
    """Build the A-Bruijn graph of a packed read set (optionally one shard of it)."""
    lib = _load()
    packed = np.ascontiguousarray(packed, dtype=np.uint8)
    offsets = np.ascontiguousarray(offsets, dtype=np.uint64)
    n_reads = offsets.size - 1
    g = ctypes.c_void_p()
    st = lib.oracle_build(packed.ctypes.data if packed.size else None,
                          offsets.ctypes.data, n_reads, k, shard_mod, shard_id, threads,
                          ctypes.byref(g))
    if st != 0:
        raise RuntimeError(f"oracle_build failed with status {st}")
    try:
        n = int(lib.oracle_num_vertices(g))
        counts = np.empty((n, 4), dtype=np.uint32)
        if k > 32:
            keys = np.empty((n, 2), dtype=np.uint64)
            st = lib.oracle_export_sorted_wide(g, keys.ctypes.data, counts.ctypes.data, n)
        else:
            keys = np.empty(n, dtype=np.uint64)
            st = lib.oracle_export_sorted(g, keys.ctypes.data, counts.ctypes.data, n)
        if st != 0:
            raise RuntimeError(f"oracle_export_sorted failed with status {st}")
        first = np.empty(n, dtype=np.uint8)
        st = lib.oracle_export_first(g, first.ctypes.data if n else None, n) if n else 0
        if st != 0:
            raise RuntimeError(f"oracle_export_first failed with status {st}")
        strs = None
        if strings:
            m = k - 1
            buf = ctypes.create_string_buffer(max(1, n * m))
            st = lib.oracle_export_strings(g, buf, n)
            if st != 0:
                raise RuntimeError(f"oracle_export_strings failed with status {st}")
            raw = buf.raw[: n * m].decode("ascii")
            strs = [raw[i * m:(i + 1) * m] for i in range(n)]
    finally:
        lib.oracle_free(g)
    return Graph(k, keys, counts, strs, first)


def shard_of_keys(keys: np.ndarray, k: int, shard_mod: int) -> np.ndarray:
    """The oracle shard of each encoded key (for filtering another builder's output)."""
    lib = _load()
    keys = np.ascontiguousarray(keys, dtype=np.uint64)
    out = np.empty(keys.size, dtype=np.uint64)
    if keys.size:
        lib.oracle_shard_of_keys(keys.ctypes.data, keys.size, k, shard_mod, out.ctypes.data)
    return out


def sketch(packed: np.ndarray, offsets: np.ndarray, k: int) -> np.ndarray:
    """HyperLogLog registers (uint32[1024]) of the vertex keys of a read set."""
    lib = _load()
    packed = np.ascontiguousarray(packed, dtype=np.uint8)
    offsets = np.ascontiguousarray(offsets, dtype=np.uint64)
    regs = np.zeros(1024, dtype=np.uint32)
    st = lib.oracle_sketch(packed.ctypes.data if packed.size else None, offsets.ctypes.data,
                           offsets.size - 1, k, regs.ctypes.data)
    if st != 0:
        raise RuntimeError(f"oracle_sketch failed with status {st}")
    return regs


def hll_estimate(regs: np.ndarray) -> float:
    """HyperLogLog estimate (Flajolet et al. 2007): alpha_m m^2 / sum 2^-M_j,
    with linear counting m ln(m/V) when the raw estimate is at most 2.5 m and
    V registers are zero."""
    m = float(regs.size)
    alpha = 0.7213 / (1.0 + 1.079 / m)
    raw = alpha * m * m / float(np.sum(np.ldexp(1.0, -regs.astype(np.int64))))
    zeros = int(np.count_nonzero(regs == 0))
    if raw <= 2.5 * m and zeros > 0:
        return m * float(np.log(m / zeros))
    return raw


def decode_key(key, k: int) -> str:
    """The (k-1)-mer of a key (an int, or a (high, low) word pair for k > 32)."""
    m = k - 1
    if not isinstance(key, int) and np.ndim(key) == 1:
        key = (int(key[0]) << 64) | int(key[1])
    return "".join("ACGT"[(int(key) >> (2 * (m - 1 - j))) & 3] for j in range(m))


from .euler import eulerian_path, spell  # noqa: E402,F401
