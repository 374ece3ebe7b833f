"""Autotuner for the insert's launch shape.

The built graph never depends on ``dbg_tuning`` (the parity tests assert
it); only the speed does.  :func:`tune` times candidate settings on the
caller's own read set and table -- each trial empties the table, inserts the
reads, and is timed with CUDA events on the insert's stream -- and leaves the
fastest setting on the graph.  Candidates cover the insert path (direct or
binned), the direct kernel's block size, tile size and warp aggregation, the
binned path's region size and apply mode (tiled or streaming), and the
streaming apply's probe slots per thread, chunk length and CTAs per SM.
"""

from __future__ import annotations

import itertools
import statistics

from . import dbg


def candidates(k: int, binned: bool) -> list[dict]:
    """The settings tried for a graph of k-mer length ``k``."""
    out = [dict(insert_path=1, block_threads=b, tile_reads=tr, warp_aggregate=a)
           for b, tr, a in itertools.product((128, 256), (64, 0), (0, 1))]
    if binned and k <= 31:
        # the tiled apply over region sizes (0: its default of 2^21 slots)
        out += [dict(insert_path=2, apply_mode=2, region_log2=r) for r in (0, 20, 22)]
        # the streaming apply's launch shapes
        out += [dict(insert_path=2, apply_mode=1, apply_unroll=u, apply_chunk=m, apply_ctas=c,
                     region_log2=r)
                for u, m, c, r in itertools.product((2, 4), (4, 8, 16), (0, 3), (0, 20))]
    return out


def time_setting(graph: "dbg.Graph", packed, offsets, setting: dict, reps: int = 2,
                 stream=None) -> float:
    """Mean milliseconds of one insert of the reads into the emptied graph."""
    import torch
    graph.set_tuning(**setting)
    s = stream or torch.cuda.current_stream()
    times = []
    for i in range(reps + 1):
        graph.reset(s)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(s)
        graph.insert(packed, offsets, stream=s)
        b.record(s)
        s.synchronize()
        if i > 0:  # the first run is a warm-up (allocations, caches)
            times.append(a.elapsed_time(b))
    st = graph.status(s)
    if st != dbg.OK:
        raise dbg.DbgError(st, f"insert under {setting}")
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
