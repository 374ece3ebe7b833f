"""Helpers shared by the GPU tests: move a read set to the device, build
its graph through the C ABI, build it with the oracle, compare."""

import numpy as np

import oracle
from paper_2401_02756_gb300 import dbg


def to_device(rs, pad: int = 16, shift: int = 0):
    """Device copies of a read set: (packed uint8, offsets int64).  ``shift``
    places the stream ``shift`` bytes into a larger buffer (a pointer that is
    not 16-byte aligned); the returned packed tensor starts at that byte."""
    import torch
    buf = torch.zeros(rs.packed.size + pad + shift, dtype=torch.uint8)
    buf[shift:shift + rs.packed.size] = torch.from_numpy(rs.packed)
    dev = buf.cuda()
    packed = dev[shift:]
    offsets = torch.from_numpy(rs.offsets.view(np.int64).copy()).cuda()
    return packed, offsets


def capacity_for(rs, factor: float = 2.0) -> int:
    ln = rs.lengths()
    ub = int(np.maximum(ln - rs.k + 2, 0).sum())
    return max(64, int(ub * factor) + 16)


def gpu_graph(rs, capacity=None, tuning=None, max_probes=0, shift=0):
    g = dbg.Graph(rs.k, capacity or capacity_for(rs), max_probes=max_probes)
    if tuning:
        g.set_tuning(**tuning)
    packed, offsets = to_device(rs, shift=shift)
    g.insert(packed, offsets)
    return g


def gpu_export(rs, **kw):
    g = gpu_graph(rs, **kw)
    st = g.status()
    assert st == dbg.OK, dbg.STATUS_NAMES.get(st, st)
    keys, counts = g.export()
    g.close()
    return keys, counts


def oracle_export(rs, **kw):
    o = oracle.build_graph(rs.packed, rs.offsets, rs.k, **kw)
    return o.keys, o.counts


def assert_same_graph(got, exp):
    gk, gc = got
    ek, ec = exp
    assert gk.dtype == np.uint64 and gc.dtype == np.uint32
    assert gk.shape == ek.shape, (gk.shape, ek.shape)
    if gk.size:
        bad = np.flatnonzero(gk != ek)
        assert bad.size == 0, f"first key mismatch at {bad[0]}: {gk[bad[0]]} vs {ek[bad[0]]}"
        badc = np.flatnonzero((gc != ec).any(axis=1))
        assert badc.size == 0, f"first counter mismatch at {badc[0]}: {gc[badc[0]]} vs {ec[badc[0]]}"
