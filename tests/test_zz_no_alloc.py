"""dbg_export_sorted_noalloc: the sorted export for callers that cannot
allocate device memory while they run (for example a serving loop held to a
memory budget that another component accounts for).  It must return exactly
what dbg_export_sorted returns, call after call, although every call reuses
the same fixed scratch array inside the library."""

import ctypes
import os

import numpy as np
import pytest

from gpu_util import capacity_for, gpu_graph
from paper_2401_02756_gb300 import build, dbg, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    build.build()
    return dbg.load()


def export_noalloc(lib, g, max_n):
    """Call the no-alloc entry point through the C ABI into device buffers."""
    import torch
    keys = torch.full((max(max_n, 1),), -1, dtype=torch.int64, device="cuda")
    counts = torch.full((max(max_n, 1), 4), -1, dtype=torch.int32, device="cuda")
    n = ctypes.c_uint64()
    st = lib.dbg_export_sorted_noalloc(g.handle, keys.data_ptr(), counts.data_ptr(), max_n,
                                       ctypes.byref(n), None)
    D = int(n.value)
    return (st, D, keys[:D].cpu().numpy().view(np.uint64),
            counts[:D].cpu().numpy().view(np.uint32))


def test_noalloc_export_equals_regular_export_on_consecutive_calls(lib):
    sets = [synth.ragged_reads(2000, 300, 21, 515, lead=1), synth.ragged_reads(1500, 250, 31, 616)]
    graphs = [gpu_graph(rs) for rs in sets]
    # two graphs of different size, then the first again: the shared scratch
    # holds the previous call's contents each time
    for g in (graphs[0], graphs[1], graphs[0]):
        ref_keys, ref_counts = g.export()
        assert 0 < ref_keys.size <= dbg.NOALLOC_EXPORT_MAX_VERTICES
        st, D, keys, counts = export_noalloc(lib, g, ref_keys.size)
        assert st == dbg.OK, dbg.STATUS_NAMES.get(st, st)
        assert D == ref_keys.size
        assert np.array_equal(keys, ref_keys)
        assert np.array_equal(counts, ref_counts)
    for g in graphs:
        g.close()


def test_noalloc_export_refuses_a_graph_over_its_limit(lib):
    rs = synth.sample_reads(synth.random_genome(2_000_000, 99), 6000, 150, 0.0, 99, 31, "big")
    g = gpu_graph(rs)
    D, _ = g.stats()
    assert D > dbg.NOALLOC_EXPORT_MAX_VERTICES
    st, n, _, _ = export_noalloc(lib, g, D)
    assert st == dbg.ERR_NOALLOC_LIMIT and n == D
    keys, _ = g.export()  # the regular export is unaffected
    assert keys.size == D
    g.close()


def test_noalloc_export_size_query_and_empty_graph(lib):
    rs = synth.ragged_reads(300, 120, 15, 717)
    g = gpu_graph(rs)
    ref_keys, _ = g.export()
    st, n, _, _ = export_noalloc(lib, g, 3)
    assert st == dbg.ERR_BUFFER_TOO_SMALL and n == ref_keys.size
    g.close()
    empty = dbg.Graph(21, capacity_for(rs))
    st, n, _, _ = export_noalloc(lib, empty, 10)
    assert st == dbg.OK and n == 0
    empty.close()


def test_noalloc_export_refuses_wide_keys(lib):
    rs = synth.ragged_reads(200, 150, 51, 818)
    g = gpu_graph(rs)
    st, _, _, _ = export_noalloc(lib, g, 100_000)
    assert st == dbg.ERR_INVALID_ARG
    g.close()


_NO_ALLOC_CHILD = r"""
import ctypes, sys
import numpy as np
import torch
sys.path.insert(0, sys.argv[1])
sys.path.insert(0, sys.argv[1] + "/tests")
from gpu_util import gpu_graph
from paper_2401_02756_gb300 import dbg, synth
lib = dbg.load()
rs = synth.sample_reads(synth.random_genome(1_000_000, 5), 4000, 150, 0.0, 5, 31, "x")
g = gpu_graph(rs)
D, _ = g.stats()
keys = torch.empty(D, dtype=torch.int64, device="cuda")
counts = torch.empty((D, 4), dtype=torch.int32, device="cuda")
n = ctypes.c_uint64()
def call():
    st = lib.dbg_export_sorted_noalloc(g.handle, keys.data_ptr(), counts.data_ptr(), D,
                                       ctypes.byref(n), None)
    assert st == dbg.OK, st
call()  # the first call on the device looks up the scratch array's address
torch.cuda.synchronize()
free0 = torch.cuda.mem_get_info()[0]
for _ in range(4):
    call()
torch.cuda.synchronize()
free1 = torch.cuda.mem_get_info()[0]
print(D, free0, free1)
"""


def test_noalloc_export_allocates_nothing(lib):
    # in a fresh process (no pool memory cached by an earlier regular export):
    # repeated calls on a graph whose regular export would take more than the
    # fixed scratch's 16 MiB leave the device's free memory exactly as it was
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "-c", _NO_ALLOC_CHILD, root], capture_output=True,
                       text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    D, free0, free1 = map(int, r.stdout.split()[-3:])
    assert 48 * D > (16 << 20) and D <= dbg.NOALLOC_EXPORT_MAX_VERTICES
    assert free1 == free0
