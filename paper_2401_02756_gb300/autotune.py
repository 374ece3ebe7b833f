"""Autotuner for the insert's launch shape.

The built graph never depends on ``dbg_tuning`` (the parity tests assert
it); only the speed does.  :func:`tune` times candidate settings on the
caller's own read set and table -- each trial rebuilds the graph from empty
(``dbg_build_reads``) and is timed with CUDA events on the build's stream --
and leaves the fastest setting on the graph.  :func:`tune_batch` does the
same for a batched build (``dbg_build_batch``) of many graphs, whose binned
chains take their shape from the first graph's setting.

Candidates cover the insert path (direct or binned); the direct kernel's
block size, read-tile size and warp aggregation; the binned path's table
region (the tiles per region of the tiled apply and the split's fan-out), the
scatter's read tile, the split's block size and the apply mode (tiled or
streaming); and the streaming apply's probe slots per thread (its probe
window), chunk length and CTAs per SM.  The probe bound ``max_probes`` is not
a candidate: it decides when an insert gives up, never how fast it runs.
"""

from __future__ import annotations

import itertools
import statistics

from . import dbg


def _tiled(region_log2: int, scatter_reads: int, split_threads: int) -> dict:
    return dict(insert_path=2, apply_mode=2, region_log2=region_log2, scatter_reads=scatter_reads,
                split_threads=split_threads)


def candidates(k: int, binned: bool) -> list[dict]:
    """The settings tried for a graph of k-mer length ``k``."""
    out = [dict(insert_path=1, block_threads=b, tile_reads=tr, warp_aggregate=a)
           for b, tr, a in itertools.product((128, 256), (64, 0), (0, 1))]
    if binned and k <= 31:
        # the tiled apply: regions (0: its default of 2^21 slots) with the
        # split's block size, and the scatter's read tile
        out += [_tiled(r, 0, 0) for r in (0, 20, 22)]
        out += [_tiled(0, sr, 0) for sr in (256, 512)]
        out += [_tiled(r, 0, 1024) for r in (0, 22)]
        # the streaming apply's launch shapes
        out += [dict(insert_path=2, apply_mode=1, apply_unroll=u, apply_chunk=m, apply_ctas=c,
                     region_log2=r)
                for u, m, c, r in itertools.product((2, 4), (4, 8, 16), (0, 3), (0, 20))]
    return out


def batch_candidates() -> list[dict]:
    """The settings tried for a batched build: the binned chains' shapes --
    region sizes with the split's block size, the scatter's read tile."""
    return ([_tiled(0, 0, 0)] + [_tiled(r, 0, st) for r in (18, 19, 20) for st in (0, 512)] +
            [_tiled(r, sr, 0) for r in (0, 19) for sr in (256, 512)] + [_tiled(0, 0, 1024)])


def time_setting(graph: "dbg.Graph", packed, offsets, setting: dict, reps: int = 2,
                 stream=None) -> float:
    """Mean milliseconds of one build of the reads under ``setting``
    (``float('inf')`` if the build fails under it)."""
    import torch
    graph.set_tuning(**setting)
    s = stream or torch.cuda.current_stream()
    times = []
    for i in range(reps + 1):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(s)
        graph.build(packed, offsets, stream=s)
        b.record(s)
        s.synchronize()
        if i > 0:  # the first run is a warm-up (allocations, caches)
            times.append(a.elapsed_time(b))
    if graph.status(s) != dbg.OK:
        return float("inf")
    return statistics.mean(times)


def tune(graph: "dbg.Graph", packed, offsets, reps: int = 2, stream=None,
         settings: list[dict] | None = None) -> tuple[dict, list[tuple[dict, float]]]:
    """Try the candidate settings, keep the fastest on ``graph`` and return it
    with every (setting, ms) measured.  The graph is left empty."""
    info = graph.info()
    binned = info["table_bytes"] >= (64 << 20)
    trials = []
    for setting in settings or candidates(graph.k, binned):
        trials.append((setting, time_setting(graph, packed, offsets, setting, reps, stream)))
    best = min(trials, key=lambda t: t[1])[0]
    graph.set_tuning(**best)
    graph.reset(stream)
    return best, trials


def tune_batch(items, reps: int = 2, stream=None, settings: list[dict] | None = None):
    """Try settings for a batched build of ``items`` (``(graph, packed,
    offsets)`` as for ``dbg.build_batch``), each applied to every graph; keep
    the fastest on every graph and return it with every (setting, ms).  The
    graphs are left holding their graphs (the last build)."""
    import torch
    s = stream or torch.cuda.current_stream()
    graphs = [g for g, _, _ in items]
    trials = []
    for setting in settings or batch_candidates():
        for g in graphs:
            g.set_tuning(**setting)
        times = []
        for i in range(reps + 1):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(s)
            dbg.build_batch(items, stream=s)
            b.record(s)
            s.synchronize()
            if i > 0:
                times.append(a.elapsed_time(b))
        ok = all(g.status(s) == dbg.OK for g in graphs)
        trials.append((setting, statistics.mean(times) if ok else float("inf")))
    best = min(trials, key=lambda t: t[1])[0]
    for g in graphs:
        g.set_tuning(**best)
    return best, trials
