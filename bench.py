#!/usr/bin/env python
"""Benchmark: A-Bruijn graph build throughput (edges inserted per second) on GB300.

One step = one complete graph build of the workload into a pre-allocated
table: K2 (empty the table) then K1 (insert every k-mer of every read), with
the reads already resident in HBM.  ``value`` is edges/s over K timed steps
(whole job, max over ranks; N > 1 runs independent replicas).  ``e2e`` is
the same build through the host-buffer entry point (pinned host reads copied
in chunks inside the timed region, graph statistics read back each step).
The ``roofline`` object rates the insert kernel alone: algorithmic bytes per
launch (64 B per vertex touch -- one 32-byte sector read and written -- plus
the packed reads and offsets) over its CUDA-event duration, against the
measured HBM copy bandwidth.  ``cpu_baseline`` times the CPU oracle on a
bounded sample of the same reads.

``--impl reference`` times the CPU oracle itself (the only reference there
is) on bounded samples of the same workload.
"""

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "edges inserted/s on 1 GB300 + % atomic/HBM roofline; batch p50/p99 latency"
FALLBACK_HBM_GBS = 6800.0
SECTOR_RMW_BYTES = 64  # one 32-byte sector read + written per vertex touch


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="100mbp_30x_k31",
                    help="100mbp_30x_k31 | 5mbp_50x_k31 | 2mbp_30x_k31 | 10kb_k21 | batch256 | "
                         "serve | sizing64 (--profile-case only)")
    ap.add_argument("--requests", type=int, default=400, help="serve: number of requests")
    ap.add_argument("--rate", type=float, default=200.0, help="serve: arrivals per second")
    ap.add_argument("--budget-gb", type=float, default=150.0, help="serve: device memory budget")
    ap.add_argument("--downstream", action="store_true",
                    help="also time normalization and contigs on the built table")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batch", action="store_true",
                    help="leave the batched-build sub-object out of the default line")
    ap.add_argument("--no-serve", action="store_true",
                    help="leave the request-loop sub-object out of the default line")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-probe", action="store_true")
    ap.add_argument("--tuning", default="",
                    help="insert launch shape, e.g. apply_unroll=4,insert_path=2 (graph unchanged)")
    ap.add_argument("--profile-case", action="store_true",
                    help="only build the workload's graph warmup + steps times (a small case "
                         "for ncu) and print a summary line")
    ap.add_argument("--profile-export", action="store_true",
                    help="with --profile-case: also export the graph twice into device buffers")
    ap.add_argument("--agg-study", action="store_true",
                    help="time the direct insert with and without warp aggregation and exit")
    ap.add_argument("--probe-sweep", action="store_true",
                    help="print the random-sector probe rate over buffer sizes and exit")
    ap.add_argument("--window-sweep", action="store_true",
                    help="print only the sliding-window probe rates and exit")
    return ap.parse_args()


# ---------------------------------------------------------------------------
# helpers
# ---------------------------------------------------------------------------

def workload_distinct(name):
    """Distinct vertices of a workload as recorded by the oracle, if known."""
    p = os.path.join(ROOT, "tests", "golden", "workload_digests.json")
    if os.path.exists(p):
        d = json.load(open(p)).get(name)
        if d:
            return int(d["n_vertices"])
    return None


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return FALLBACK_HBM_GBS, "fallback"


def kernel_source_digest():
    """Digest of the insert kernels' code: their sources without line
    comments and blank lines (a comment edit keeps recorded profiles valid)."""
    h = hashlib.sha256()
    for f in ("dbg_insert.cu", "dbg_binned.cu", "dbg_binned.cuh", "dbg_tiles.cuh", "dbg_internal.cuh",
              "dbg_tma.cuh"):
        for line in open(os.path.join(ROOT, "paper_2401_02756_gb300", "csrc", f), encoding="utf-8"):
            code = line.split("//", 1)[0].rstrip()
            if code:
                h.update(code.encode() + b"\n")
    return h.hexdigest()[:16]


def recorded_traffic(workload, kernel):
    """DRAM bytes per launch of `kernel` from a committed ncu summary, if it
    was taken on the current kernel source."""
    p = os.path.join(ROOT, "profiles", "insert_traffic.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p))
    e = d.get(workload, {}).get(kernel)
    if not e or e.get("kernel_source_digest") != kernel_source_digest():
        return None
    return e.get("dram_bytes_per_launch")


class ClockSampler:
    """nvidia-smi clock and throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = str(gpu_index)
        self.rows = []
        self.proc = None
        self.th = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", self.idx], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                text=True)
        except (FileNotFoundError, OSError):
            self.proc = None
            return
        self.th = threading.Thread(target=self._read, daemon=True)
        self.th.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.3)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in self.rows:
            for n, v in zip(names, r[5:9]):
                if v.lower() in ("active", "1"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(self.rows)}


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def time_oracle_sample(rs, seconds_target, threads, seed_reads=20_000):
    """Time the oracle (as it stands) on a prefix of the reads sized to take
    about ``seconds_target`` seconds; returns (edges/s, sample description)."""
    import oracle
    from paper_2401_02756_gb300 import synth

    def prefix(n):
        n = min(n, rs.n_reads)
        nb = int((int(rs.offsets[n]) + 3) // 4)
        return synth.ReadSet(rs.name, rs.k, rs.packed[:nb], rs.offsets[:n + 1].copy())

    cal = prefix(seed_reads)
    t = time.perf_counter()
    oracle.build_graph(cal.packed, cal.offsets, cal.k, threads=threads)
    dt = max(time.perf_counter() - t, 1e-3)
    n = int(min(rs.n_reads, max(seed_reads, seed_reads * seconds_target / dt)))
    smp = prefix(n)
    t = time.perf_counter()
    oracle.build_graph(smp.packed, smp.offsets, smp.k, threads=threads)
    dt = time.perf_counter() - t
    return smp.n_edges() / dt, dt, n, f"first {n} of {rs.n_reads} reads ({smp.n_edges()} edges), {dt:.1f} s"


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------

def path_roofline(edges, touches, in_bytes, insert_s, peak_gbs, probe, binned=False):
    """The whole insert against the two ceilings of a hash-table build: HBM
    (every vertex touch a 32-byte sector read and written, plus the input)
    and the measured random-sector atomic rate on a table-sized buffer.  The
    roofline is the lower of the two for the direct insert, which touches the
    table at random.  The binned insert does not, so the atomic rate is no
    ceiling for it: it is then reported as the direct path's ceiling only,
    and the roofline is the HBM one."""
    edge_bytes = (touches * SECTOR_RMW_BYTES + in_bytes) / edges
    hbm = peak_gbs * 1e9 / edge_bytes
    achieved = edges / insert_s
    out = {"unit": "edges/s", "achieved": achieved, "bytes_per_edge": edge_bytes,
           "hbm_ceiling": hbm, "frac_of_hbm_ceiling": achieved / hbm,
           "atomic_ceiling": None, "frac_of_atomic_ceiling": None}
    if probe:
        atomic = probe["load_red_touches_per_s"] * edges / touches
        if binned:
            out.update(atomic_ceiling=None, frac_of_atomic_ceiling=None,
                       direct_path_atomic_ceiling=atomic,
                       over_direct_path_atomic_ceiling=achieved / atomic,
                       roofline=hbm, frac_of_roofline=achieved / hbm)
        else:
            out.update(atomic_ceiling=atomic, frac_of_atomic_ceiling=achieved / atomic,
                       roofline=min(hbm, atomic), frac_of_roofline=achieved / min(hbm, atomic))
    else:
        out.update(roofline=hbm, frac_of_roofline=achieved / hbm)
    return out


def workload_config(name, rs, D, d_source, capacity, tuning, world):
    """The benchmark's ``config`` object, the same for both arms."""
    return {"workload": name, "genome_bp": rs.meta.get("genome_len"),
            "n_reads": rs.n_reads, "read_len": rs.meta.get("read_len"), "k": rs.k,
            "error_rate": rs.meta.get("error_rate"), "edges": rs.n_edges(),
            "distinct_vertices": D, "distinct_source": d_source,
            "capacity_slots": capacity, "table_gb": capacity * 32 / 1e9 if capacity else None,
            "l2": "table and reads larger than L2 (no flush needed)",
            "tuning": tuning or "default",
            "parallelism": f"replicas x{world}"}


def job_throughput(local_ms: float, units_per_rank: float, world: int, dist=None,
                   device=None) -> tuple[float, float]:
    """Whole-job throughput of `world` replicas: the units every rank
    processed over the slowest rank's time (max over ranks).  Returns
    (units per second, the max time in ms)."""
    if dist is not None:
        import torch
        t = torch.tensor([float(local_ms)], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        local_ms = float(t.item())
    return units_per_rank * world / (local_ms / 1e3), local_ms


def run_ours(args):
    import torch

    from paper_2401_02756_gb300 import build as _build
    from paper_2401_02756_gb300 import dbg, synth

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.cuda.current_device()

    if rank == 0:
        _build.build()
    if dist:
        dist.barrier()
    dbg.load()

    rs = synth.WORKLOADS[args.workload]()
    edges = rs.n_edges()
    touches = int(np.maximum(rs.lengths() - rs.k + 2, 0).sum())
    packed = torch.from_numpy(np.concatenate([rs.packed, np.zeros(16, np.uint8)])).to(dev)
    offsets = torch.from_numpy(rs.offsets.view(np.int64).copy()).to(dev)

    D = workload_distinct(args.workload)
    d_source = "oracle (recorded)"
    if D is None:  # size the table from a pilot build in a generous table
        d_source = "pilot build"
        pilot = dbg.Graph(rs.k, int(touches * 1.05) + 1024)
        pilot.insert(packed, offsets)
        D, _ = pilot.stats()
        pilot.close()
    capacity = int(math.ceil(1.5 * D))
    g = dbg.Graph(rs.k, capacity)
    tuning = {kv.split("=")[0]: int(kv.split("=")[1]) for kv in args.tuning.split(",") if kv}
    if tuning:
        g.set_tuning(**tuning)
    stream = torch.cuda.current_stream()

    for _ in range(args.warmup):
        g.build(packed, offsets, stream=stream)
    torch.cuda.synchronize()
    st = g.status()
    if st != dbg.OK:
        raise RuntimeError(f"warm-up build failed: {dbg.STATUS_NAMES.get(st, st)}")
    nv, ne = g.stats()
    if ne != edges or nv != D:
        raise RuntimeError(f"graph check failed: {nv} vertices / {ne} edges, expected {D} / {edges}")

    K = args.steps
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(K)]
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    g.enable_kernel_timing(K)  # per-kernel CUDA events inside each insert call, same stream
    clocks = ClockSampler(dev)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.25)
    t0.record(stream)
    for i in range(K):
        # one step: the whole graph built from empty (dbg_build_reads: the
        # table's emptying is folded into the insert's tiled apply)
        ev[i][0].record(stream)
        g.build(packed, offsets, stream=stream)
        ev[i][1].record(stream)
    t1.record(stream)
    torch.cuda.synchronize()
    clock_info = clocks.stop()
    if dist:
        dist.barrier()
    total_ms = t0.elapsed_time(t1)
    step_ms = [a.elapsed_time(b) for a, b in ev]
    k1_ms = step_ms  # the build is the insert (with the emptying folded in)
    kt = g.kernel_times(K)
    g.enable_kernel_timing(0)
    bin_counters = g.binned_counters()  # the last timed call's (after the timed region)
    st = g.status()
    if st != dbg.OK:
        raise RuntimeError(f"timed build failed: {dbg.STATUS_NAMES.get(st, st)}")

    value, total_ms = job_throughput(total_ms, edges * K, world, dist, dev)
    k1_mean_s = statistics.mean(k1_ms) / 1e3
    in_bytes = rs.packed.nbytes + rs.offsets.nbytes
    # algorithmic bytes per launch of each kernel
    names = dbg.Graph.KERNELS
    kernels = {}
    for j, name in enumerate(names):
        col = [float(x) for x in kt[:, j] if x >= 0]
        if col:
            kernels[name] = {"ms": statistics.mean(col), "launches_per_step": 1}
    tiled = "bin_split" in kernels
    if tiled:  # bucket sizing: total + buckets; split: units (tile buckets) + tile scatter
        kernels["bin_count"]["launches_per_step"] = 2
        kernels["bin_split"]["launches_per_step"] = 2
        # the fall-back span: the gated emptying pass and the gated direct
        # insert (both return at once when the binned kernels did the work)
        kernels["direct_fallback"]["launches_per_step"] = 2
    kernel_bytes = {
        "direct": touches * SECTOR_RMW_BYTES + in_bytes,
        # (the direct path's build empties the table first: 32 B per slot,
        # a kernel outside the timer's list)
        # tiled: the read offsets only (bucket sizing); streaming: the count pass reads the input
        "bin_count": (rs.offsets.nbytes if tiled else in_bytes),
        "bin_scan": 0,
        "bin_scatter": in_bytes + 8 * touches,
        # the second partition: every event read and written once
        "bin_split": 16 * touches,
        # tiled, building from empty: events read once, every table slot
        # written once (never read); streaming: events read once, one sector
        # read-modify-write per vertex
        "bin_apply": 8 * touches + (32 * capacity if tiled else SECTOR_RMW_BYTES * D),
        "bin_deferred": 0,
        "direct_fallback": 0,
    }
    launched = sum(1 for j in range(len(names)) if (kt[:, j] >= 0).any())
    # the whole step against HBM: the algorithmic bytes of every kernel it
    # launched over the step's mean time
    step_alg = sum(kernel_bytes[n] for n in kernels)  # (each entry: bytes per step)
    insert_roofline = {"alg_bytes": step_alg, "achieved": step_alg / k1_mean_s / 1e9,
                       "frac": step_alg / k1_mean_s / 1e9 / measured_peaks()[0]}
    dom = max(kernels, key=lambda n: kernels[n]["ms"])
    dom_s = kernels[dom]["ms"] / 1e3
    alg_bytes = kernel_bytes[dom]
    peak, peak_kind = measured_peaks()
    achieved = alg_bytes / dom_s / 1e9
    traffic = recorded_traffic(args.workload, dom)
    for name in kernels:
        b = kernel_bytes[name]
        kernels[name]["alg_gb"] = b / 1e9
        kernels[name]["gbs"] = b / (kernels[name]["ms"] / 1e3) / 1e9 if b else None

    # measured random-sector ceiling (K5) over a buffer the size of the table
    probe = None
    if not args.no_probe:
        buf = torch.empty(capacity * 32, dtype=torch.uint8, device=dev)
        buf.zero_()
        for _ in range(2):
            dbg.probe_random_sectors(buf, capacity, touches, 7, 1, stream)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ms = []
        for mode in (0, 1):
            a.record(stream)
            dbg.probe_random_sectors(buf, capacity, touches, 11 + mode, mode, stream)
            b.record(stream)
            torch.cuda.synchronize()
            ms.append(a.elapsed_time(b))
        del buf
        probe = {"touches": touches, "red_only_ms": round(ms[0], 3), "load_red_ms": round(ms[1], 3),
                 "load_red_touches_per_s": touches / (ms[1] / 1e3),
                 "load_red_gbs_equiv": touches * SECTOR_RMW_BYTES / (ms[1] / 1e3) / 1e9,
                 "insert_rate_over_probe_rate": (ms[1] / 1e3) / k1_mean_s}

    # end to end through the host-buffer entry point
    e2e = None
    if not args.no_e2e:
        pk_h = torch.from_numpy(rs.packed).pin_memory()
        of_h = torch.from_numpy(rs.offsets.view(np.int64)).pin_memory()
        g.build_host(pk_h, of_h, stream=stream)
        g.stats(stream)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        a = time.perf_counter()
        for _ in range(K):
            g.build_host(pk_h, of_h, stream=stream)
            nv_e, ne_e = g.stats(stream)  # device -> host read of the result
        torch.cuda.synchronize()
        e2e_s = time.perf_counter() - a
        if dist:
            t = torch.tensor([e2e_s], device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            e2e_s = float(t.item())
        if ne_e != edges:
            raise RuntimeError("end-to-end build lost edges")
        e2e = {"value": edges * K * world / e2e_s, "unit": "edges/s",
               "h2d_bytes_per_step": int(rs.packed.nbytes + rs.offsets.nbytes),
               "d2h_bytes_per_step": 2 * 8 + 4}

    # the sorted export (not part of a step) into preallocated device buffers:
    # one warm-up, then the median of three (the vertex count for the buffers
    # comes from g.stats(), outside the timed calls)
    ea, eb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    keys_d = torch.empty(D, dtype=torch.int64, device=dev)
    counts_d = torch.empty((D, 4), dtype=torch.int32, device=dev)
    ex_ms = []
    for i in range(4):
        ea.record(stream)
        n_exp = g.export_into(keys_d, counts_d, stream)
        eb.record(stream)
        torch.cuda.synchronize()
        if i:
            ex_ms.append(ea.elapsed_time(eb))
    export_ms = statistics.median(ex_ms)
    if n_exp != D:
        raise RuntimeError("export size mismatch")
    del keys_d, counts_d

    # the paper's downstream passes on the resident table: normalization
    # (divisor = edges / genome size) and contigs (Alg. 5), each timed once
    downstream = None
    if args.downstream:
        import ctypes
        L = dbg.load()
        div = edges / float(rs.meta.get("genome_len") or 1)
        ea.record(stream)
        g.normalize(div, stream)
        eb.record(stream)
        torch.cuda.synchronize()
        norm_ms = ea.elapsed_time(eb)
        nc, nb = ctypes.c_uint64(), ctypes.c_uint64()
        t_c = time.perf_counter()
        st_c = L.dbg_find_contigs(g.handle, None, 0, None, 0, ctypes.byref(nc), ctypes.byref(nb),
                                  stream.cuda_stream)
        contig_s = time.perf_counter() - t_c
        if st_c not in (dbg.OK, dbg.ERR_BUFFER_TOO_SMALL):
            raise RuntimeError(f"contigs failed: {dbg.STATUS_NAMES.get(st_c, st_c)}")
        downstream = {"divisor": div, "normalize_ms": norm_ms,
                      "contigs_ms_size_pass": contig_s * 1e3, "contigs": int(nc.value),
                      "contig_bases": int(nb.value),
                      "note": "contig time is the first (sizing) call: marks, starts, sort, "
                              "walk lengths, scan; the second call repeats it and writes"}
    g.close()
    del packed, offsets
    torch.cuda.empty_cache()

    # the batched form and the request loop, each with its own clock record
    # (bounded: a few passes each; --workload batch256 / serve run them alone)
    batch = serve = None
    if rank == 0 and world == 1 and not args.no_batch:
        ck = ClockSampler(dev)
        ck.start()
        batch = measure_batch(steps=3, warmup=2)
        batch["clocks"] = ck.stop()
        torch.cuda.empty_cache()
    if rank == 0 and world == 1 and not args.no_serve:
        ck = ClockSampler(dev)
        ck.start()
        serve = measure_serve(400, 200.0, 150.0, steps=2, overload_rate=2000.0)
        serve["clocks"] = ck.stop()
        torch.cuda.empty_cache()

    serve_big = None
    if rank == 0 and world == 1 and not args.no_serve:
        ck = ClockSampler(dev)
        ck.start()
        serve_big = measure_serve_big(rs)
        serve_big["clocks"] = ck.stop()
        torch.cuda.empty_cache()

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cores = host_cores()
        v, dt, _, desc = time_oracle_sample(rs, 15.0, cores)
        v1, _, _, desc1 = time_oracle_sample(rs, 8.0, 1, seed_reads=5_000)
        cpu = {"value": v, "unit": "edges/s", "cores": cores, "kind": "oracle",
               "sample": desc + f", {cores} threads (hash-sharded vertices, every thread scans every read)",
               "single_thread": {"value": v1, "unit": "edges/s", "cores": 1, "sample": desc1}}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "edges/s", "n_gpus": world, "steps": K,
            "warmup": args.warmup, "ms_per_step": total_ms / K, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": workload_config(args.workload, rs, D, d_source, capacity, tuning, world),
            "insert_only_edges_per_s": edges / k1_mean_s,
            "insert_ms": {"mean": statistics.mean(k1_ms), "min": min(k1_ms), "max": max(k1_ms)},
            "insert_path": ("direct" if "bin_apply" not in kernels else
                            "binned" if bin_counters["binned"] else "binned, fell back to direct"),
            "binned_counters": bin_counters,
            "kernels": kernels,
            "reset": "folded into the build (dbg_build_reads): the tiled apply writes every "
                     "table tile from an EMPTY tile in shared memory",
            "export_ms": export_ms,
            "export_note": "dbg_export_sorted into device buffers (compaction that counts the "
                           "vertices, radix sort of (32-bit key prefix, slot) pairs inside the "
                           "output buffers, gather, runs of equal prefixes put in order); median "
                           "of 3 after a warm-up",
            "downstream": downstream,
            "step_ms_p50": float(np.percentile(step_ms, 50)),
            "step_ms_p99": float(np.percentile(step_ms, 99)),
            "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak,
                         "unit": "GB/s", "frac": achieved / peak, "traffic": traffic,
                         "peak_source": f"{peak_kind} HBM copy bandwidth",
                         "alg_bytes_per_launch": alg_bytes,
                         "scope": "frac: the dominant kernel alone (its algorithmic bytes over "
                                  "its mean CUDA-event time); insert: every kernel of the step",
                         "insert": insert_roofline},
            "random_sector_probe": probe,
            "path_roofline": path_roofline(edges, touches, in_bytes, k1_mean_s, peak, probe,
                                           binned="bin_apply" in kernels),
            "cpu_baseline": cpu, "e2e": e2e, "clocks": clock_info,
            "batch256": batch, "serve_poisson200": serve, "serve_100mbp_poisson1": serve_big,
            "gpu_launches": sum(v["launches_per_step"] for v in kernels.values()) * K,
            "kernel_source_digest": kernel_source_digest(),
        }
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


# ---------------------------------------------------------------------------
# reference arm: the CPU oracle
# ---------------------------------------------------------------------------

def run_reference(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    from paper_2401_02756_gb300 import synth

    oracle.build()
    rs = synth.WORKLOADS[args.workload]()
    D = workload_distinct(args.workload)
    cores = host_cores()
    # about 100 s of oracle work in all (measured steps run ~1.5x the
    # calibration's estimate: a larger sample holds more distinct vertices)
    per_step = max(2.0, min(15.0, 100.0 / max(1, args.steps + args.warmup)))
    # size one step's sample from a calibration run
    _, _, n, _ = time_oracle_sample(rs, per_step, cores)
    nb = int((int(rs.offsets[n]) + 3) // 4)
    smp = synth.ReadSet(rs.name, rs.k, rs.packed[:nb], rs.offsets[:n + 1].copy())
    for _ in range(args.warmup):
        oracle.build_graph(smp.packed, smp.offsets, smp.k, threads=cores)
    times = []
    for _ in range(args.steps):
        t = time.perf_counter()
        oracle.build_graph(smp.packed, smp.offsets, smp.k, threads=cores)
        times.append(time.perf_counter() - t)
    value = smp.n_edges() / statistics.mean(times)
    sample = (f"first {n} of {rs.n_reads} reads ({smp.n_edges()} edges) per step, "
              f"{cores} threads")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "edges/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": statistics.mean(times) * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": workload_config(args.workload, rs, D, "oracle (recorded)",
                                  int(math.ceil(1.5 * D)) if D else None, None, world),
        "cpu_baseline": {"value": value, "unit": "edges/s", "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "edges/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def gen_batch_samples(n, seed):
    """Samples 0 .. n-1 of the batched-build distribution, made by worker
    processes (spawned: safe after CUDA is initialised)."""
    import multiprocessing as mp

    from paper_2401_02756_gb300 import synth
    with mp.get_context("spawn").Pool(max(1, min(16, (os.cpu_count() or 2) - 1))) as pool:
        made = pool.map(synth.batch_sample_arrays, [(i, seed) for i in range(n)], chunksize=2)
    return [synth.ReadSet(f"sample{i}", k, packed, offsets) for i, k, packed, offsets, _ in made]


def measure_batch(steps, warmup, n_samples=256, seed=4):
    """256 independent samples of uneven size, sized by the capacity predictor
    (sketch of every sample, one batched network forward), then built three
    ways into the same tables: one plain dbg_insert_reads per sample, one
    dbg_insert_batch call, and a CUDA graph holding that call, replayed.  The
    exact builder then judges the predictor: its error against each sample's
    distinct-vertex count.  Returns the measurements as a dict."""
    import torch

    from paper_2401_02756_gb300 import build as _build
    from paper_2401_02756_gb300 import dbg
    from paper_2401_02756_gb300.predictor import REG_STRIDE, CapacityPredictor
    _build.build()
    dbg.load()
    torch.cuda.set_device(0)
    t_gen = time.perf_counter()
    samples = gen_batch_samples(n_samples, seed)
    t_gen = time.perf_counter() - t_gen
    stream = torch.cuda.current_stream()
    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731
    dev_in, edges = [], 0
    for rs in samples:
        pk = torch.from_numpy(np.concatenate([rs.packed, np.zeros(16, np.uint8)])).cuda()
        of = torch.from_numpy(rs.offsets.view(np.int64).copy()).cuda()
        dev_in.append((pk, of))
        edges += rs.n_edges()

    # sizing: sketches and one batched forward, timed
    pred = CapacityPredictor()
    regs = torch.zeros(len(samples), REG_STRIDE, dtype=torch.int32, device="cuda")

    sketch_items = [(rs.k, pk, of, regs[i]) for i, (rs, (pk, of)) in enumerate(zip(samples, dev_in))]

    def size_all():
        dbg.sketch_batch(sketch_items, stream=stream)
        return pred.log_vertices(regs, len(samples), stream=stream)

    size_ms = []
    for i in range(warmup + steps):
        a, b = ev(), ev()
        a.record(stream)
        size_all()
        b.record(stream)
        torch.cuda.synchronize()
        if i >= warmup:
            size_ms.append(a.elapsed_time(b))
    preds = pred.predict_registers(regs, len(samples))
    graphs = [dbg.Graph(rs.k, pred.capacity(p)) for rs, p in zip(samples, preds)]
    positions = [int(np.maximum(rs.lengths() - rs.k + 2, 0).sum()) for rs in samples]
    for pos, g in zip(positions, graphs):
        # every graph asks for event room for all its vertex positions (high-
        # coverage samples exceed the default of 4.25 per slot): its share of
        # the library's buffers for a batched build, and for a plain build its
        # own buffer when its table takes the binned path
        g.reserve_events(pos)
    items = [(g, pk, of) for g, (pk, of) in zip(graphs, dev_in)]

    # a step builds every graph from empty: the batched form with one
    # dbg_build_batch call (binned chains for the large tables, shared direct
    # launches for the small ones), the plain form with one dbg_build_reads
    # per sample
    def batched():
        dbg.build_batch(items, stream)

    def plain():
        for g, (pk, of) in zip(graphs, dev_in):
            g.build(pk, of, stream=stream)

    def capture():
        batched()  # grows the library's buffers before the capture
        torch.cuda.synchronize()
        cap_stream = torch.cuda.Stream()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=cap_stream):
            dbg.build_batch(items, cap_stream)
        torch.cuda.synchronize()
        return graph

    def timed(fn):
        for _ in range(warmup):
            fn()
        ms = []
        for _ in range(steps):
            a, b = ev(), ev()
            a.record(stream)
            fn()
            b.record(stream)
            torch.cuda.synchronize()
            ms.append(a.elapsed_time(b))
        for g in graphs:
            if g.status() != dbg.OK:
                raise RuntimeError("batch: build failed")
        return ms

    # the binned chains' shape, picked by the autotuner on this batch (untimed)
    from paper_2401_02756_gb300 import autotune
    best, trials = autotune.tune_batch(items, reps=1, stream=stream)
    results = {}
    cg = capture()
    results["batched_graph"] = timed(cg.replay)
    results["batched"] = timed(batched)
    results["per_sample"] = timed(plain)  # every graph with the batch's tuning
    for g in graphs:  # every graph with the library's own choice of path and shape
        g.set_tuning()
    results["per_sample_default"] = timed(plain)
    for g in graphs:
        g.set_tuning(**best)
    D = np.array([g.stats()[0] for g in graphs], dtype=np.float64)
    # the same batch with the single-table choice of path: tables under
    # 256 MiB on the direct insert (shared launches), the others in chains
    for g in graphs:
        if g.info()["table_bytes"] < (256 << 20):
            g.set_tuning(insert_path=1)
        else:
            g.set_tuning(**best)
    cg_mixed = capture()
    results["batched_graph_small_direct"] = timed(cg_mixed.replay)
    for g in graphs:
        g.set_tuning(**best)
    del cg, cg_mixed

    # without a predictor, plain per-sample launches need the sizes another
    # way: a pilot build of each sample in a table of all its vertex
    # positions (one table per k, emptied between samples; the emptying is
    # not timed), then the vertex count
    touches = [int(np.maximum(rs.lengths() - rs.k + 2, 0).sum()) for rs in samples]
    pilots = {}
    for rs, t in zip(samples, touches):
        pilots[rs.k] = max(pilots.get(rs.k, 0), t)
    pilots = {k: dbg.Graph(k, n + 64) for k, n in pilots.items()}
    pilot_ms = 0.0
    for rs, (pk, of) in zip(samples, dev_in):
        p = pilots[rs.k]
        p.reset(stream)
        a, b = ev(), ev()
        a.record(stream)
        p.insert(pk, of, stream=stream)
        p.stats(stream)
        b.record(stream)
        torch.cuda.synchronize()
        pilot_ms += a.elapsed_time(b)
    for p in pilots.values():
        p.close()
    mlp = np.array([p.mlp for p in preds])
    hll = np.array([p.hll for p in preds])
    for g in graphs:
        g.close()
    gm = statistics.mean(results["batched_graph"])
    bm = statistics.mean(results["batched"])
    # the plain builds' baseline: the faster of the two tunings
    pm_tuned = statistics.mean(results["per_sample"])
    pm_default = statistics.mean(results["per_sample_default"])
    pm = min(pm_tuned, pm_default)
    sm = statistics.mean(size_ms)

    def err(est):
        e = np.abs(est / D - 1.0)
        return {"mean": float(e.mean()), "p99": float(np.quantile(e, 0.99)),
                "max": float(e.max())}

    return {
        "edges_per_s": edges / (gm / 1e3), "ms_per_batch": gm, "steps": steps, "warmup": warmup,
        "config": {"workload": "batch256", "samples": len(samples), "edges": edges,
                   "k": sorted({rs.k for rs in samples}), "generation_s": t_gen,
                   "sizing": "capacity predictor (margin x 1.5 x predicted vertices)",
                   "l2": "tables emptied between steps; 256 tables total "
                         f"{sum(pred.capacity(p) for p in preds) * 32 / 1e9:.1f} GB > L2"},
        "tuning": best, "tuning_trials_ms": [[t, ms] for t, ms in trials],
        "small_direct_edges_per_s":
            edges / (statistics.mean(results["batched_graph_small_direct"]) / 1e3),
        "step": "every graph built from empty (dbg_build_batch replayed from a CUDA graph: "
                "binned chains of up to 128 tables; plain: one dbg_build_reads per sample)",
        "batched_edges_per_s": edges / (bm / 1e3),
        "per_sample_edges_per_s": edges / (pm / 1e3),
        "per_sample_note": "the faster of: every plain build with the batch's tuning "
                           f"({edges / (pm_tuned / 1e3):.3e} edges/s), with the library's "
                           f"default choice of path per graph ({edges / (pm_default / 1e3):.3e})",
        "graph_over_per_sample": pm / gm,
        "batched_over_per_sample": pm / bm,
        "sizing_ms": sm,
        "batched_predicted_edges_per_s": edges / ((gm + sm) / 1e3),
        # sizing counted on the batched side only: the plain builds get their sizes free
        "batched_predicted_over_per_sample": pm / (gm + sm),
        "pilot_sizing_ms": pilot_ms,
        "per_sample_with_pilot_sizing_edges_per_s": edges / ((pm + pilot_ms) / 1e3),
        "batched_predicted_over_per_sample_with_pilot_sizing": (pm + pilot_ms) / (gm + sm),
        "batch_ms_p50": float(np.percentile(results["batched_graph"], 50)),
        "batch_ms_p99": float(np.percentile(results["batched_graph"], 99)),
        "predictor_error": {"network": err(mlp), "hyperloglog": err(hll),
                            "tables_overflowed": 0},
    }


def run_batch(args):
    clocks = ClockSampler(0)
    clocks.start()
    b = measure_batch(args.steps, args.warmup)
    clock_info = clocks.stop()
    line = {"metric": METRIC, "value": b["edges_per_s"], "unit": "edges/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": b["ms_per_batch"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
            "data": "synthetic", "config": b["config"], "clocks": clock_info}
    line.update({k: v for k, v in b.items() if k not in ("config", "steps", "warmup")})
    print(json.dumps(line), flush=True)



def measure_serve(n, rate, budget_gb, steps, seed=31, overload_rate=None):
    """The request loop: Poisson arrivals of build requests drawn from the
    batched-build size distribution, served by the continuous-batching loop
    and, for comparison, one at a time with plain calls.  A step is one
    closed-loop pass (every request present at the start) and gives the
    throughput; one realtime pass of each server at ``rate`` gives the
    latencies, and (if given) one more pass of the server at
    ``overload_rate``, where requests arrive faster than one at a time could
    serve them, shows the batching under load.  Returns a dict."""
    import multiprocessing as mp

    import torch

    from paper_2401_02756_gb300 import build as _build
    from paper_2401_02756_gb300 import dbg, synth
    from paper_2401_02756_gb300.predictor import CapacityPredictor
    from paper_2401_02756_gb300.serve import BuildServer, Request, sequential
    t_gen = time.perf_counter()
    with mp.get_context("spawn").Pool(max(1, min(16, (os.cpu_count() or 2) - 1))) as pool:
        made = pool.map(synth.batch_sample_arrays, [(i, seed) for i in range(n)], chunksize=2)
    t_gen = time.perf_counter() - t_gen
    _build.build()
    dbg.load()
    torch.cuda.set_device(0)
    arrivals = synth.poisson_arrivals(n, rate, seed)
    reqs = []
    for (i, k, packed, offsets, e), t in zip(made, arrivals):
        pp = torch.empty(packed.size, dtype=torch.uint8, pin_memory=True)
        pp.numpy()[:] = packed
        po = torch.empty(offsets.size, dtype=torch.int64, pin_memory=True)
        po.numpy()[:] = offsets.view(np.int64)
        reqs.append(Request(i, k, pp.numpy(), po.numpy().view(np.uint64), float(t), e))
    edges = sum(r.edges for r in reqs)
    pred = CapacityPredictor()
    # the chains' shape for this request mix, picked by the autotuner on a
    # batched build of the first 64 requests (untimed)
    from paper_2401_02756_gb300 import autotune
    trial = []
    for r in reqs[:64]:
        pk = torch.from_numpy(np.concatenate([r.packed, np.zeros(16, np.uint8)])).cuda()
        of = torch.from_numpy(r.offsets.view(np.int64).copy()).cuda()
        g = dbg.Graph(r.k, pred.capacity(pred.predict(r.k, pk, of)))
        ln = np.diff(r.offsets.astype(np.int64))
        g.reserve_events(int(np.maximum(ln - r.k + 2, 0).sum()))
        trial.append((g, pk, of))
    tuning, _ = autotune.tune_batch(trial, reps=1)
    for g, _, _ in trial:
        g.close()
    del trial
    torch.cuda.empty_cache()
    srv = BuildServer(pred, budget_bytes=budget_gb * 1e9, tuning=tuning)
    warm = reqs[:min(16, n)]
    srv.run(warm, realtime=False)
    sequential(warm, pred, realtime=False)
    torch.cuda.synchronize()

    closed, closed_seq = [], []
    for _ in range(steps):
        closed.append(srv.run(reqs, realtime=False).summary())
    for _ in range(max(1, min(steps, 2))):
        closed_seq.append(sequential(reqs, pred, realtime=False).summary())
    live = srv.run(reqs, realtime=True).summary()
    live_seq = sequential(reqs, pred, realtime=True).summary()
    over = None
    if overload_rate:
        fast = [Request(r.rid, r.k, r.packed, r.offsets, float(t), r.edges)
                for r, t in zip(reqs, synth.poisson_arrivals(n, overload_rate, seed + 1))]
        over = srv.run(fast, realtime=True).summary()
        over["arrival_rate_per_s"] = overload_rate
    thr = statistics.mean(c["edges_per_s"] for c in closed)
    thr_seq = statistics.mean(c["edges_per_s"] for c in closed_seq)
    return {
        "edges_per_s": thr, "ms_per_pass": statistics.mean(c["wall_s"] for c in closed) * 1e3,
        "config": {"workload": f"serve_poisson{rate:g}", "requests": n, "edges": edges,
                   "arrival_rate_per_s": rate, "budget_gb": budget_gb,
                   "sizes": "batched-build distribution (genome 50 kb-2 Mbp, 10-60x, k 21/31)",
                   "generation_s": t_gen, "answer": "sorted graph exported to host memory",
                   "tuning": tuning},
        "latency_ms_p50": live["latency_ms_p50"], "latency_ms_p99": live["latency_ms_p99"],
        "build_latency_ms_p50": live["build_latency_ms_p50"],
        "build_latency_ms_p99": live["build_latency_ms_p99"],
        "mean_batch": live["mean_batch"], "peak_bytes": live["peak_bytes"],
        "realtime": live, "closed_loop": closed[-1], "overload": over,
        "sequential": {"edges_per_s": thr_seq, "latency_ms_p50": live_seq["latency_ms_p50"],
                       "latency_ms_p99": live_seq["latency_ms_p99"], "realtime": live_seq},
        "server_over_sequential": thr / thr_seq,
    }


def measure_serve_big(rs, n=6, rate=1.0, budget_gb=150.0, seed=33):
    """The request loop on requests the size of the 100 Mbp workload (2.4e9
    edges each, all the same reads) arriving at a low Poisson rate: each
    request's table is far beyond what the capacity network was trained on,
    so HyperLogLog sizes it; the binned chain builds it; the answer is its
    sorted graph (422 M vertices) in host memory.  Beside it, the same
    requests served one at a time with plain calls.  Returns a dict."""
    import torch

    from paper_2401_02756_gb300 import synth
    from paper_2401_02756_gb300.predictor import CapacityPredictor
    from paper_2401_02756_gb300.serve import BuildServer, Request, sequential
    pp = torch.empty(rs.packed.size, dtype=torch.uint8, pin_memory=True)
    pp.numpy()[:] = rs.packed
    po = torch.empty(rs.offsets.size, dtype=torch.int64, pin_memory=True)
    po.numpy()[:] = rs.offsets.view(np.int64)
    packed, offsets = pp.numpy(), po.numpy().view(np.uint64)
    arrivals = synth.poisson_arrivals(n, rate, seed)
    reqs = [Request(i, rs.k, packed, offsets, float(t), rs.n_edges()) for i, t in enumerate(arrivals)]
    pred = CapacityPredictor()
    D = workload_distinct(rs.name) or 0
    srv = BuildServer(pred, budget_bytes=budget_gb * 1e9, max_batch=4)
    srv.reserve_host_rows(int(D * 1.1))  # every worker's pinned output, before the run
    srv.run(reqs[:1], realtime=False)    # the library's chain buffers grown once
    live = srv.run(reqs, realtime=True).summary()
    from paper_2401_02756_gb300.serve import _Exporter
    ex = _Exporter(torch.device("cuda"))
    ex.buffers(int(D * 1.1))
    sequential(reqs[:1], pred, realtime=False, exporter=ex)  # its own buffers grown once
    seq = sequential(reqs[:2], pred, realtime=False, exporter=ex).summary()
    return {"config": {"workload": f"serve_100mbp_poisson{rate:g}", "requests": n,
                       "warm": "pinned outputs and the library's buffers sized before the run",
                       "edges_per_request": rs.n_edges(), "arrival_rate_per_s": rate,
                       "budget_gb": budget_gb,
                       "sizing": "HyperLogLog (beyond the network's training range)",
                       "answer": "sorted graph exported to host memory"},
            "latency_ms_p50": live["latency_ms_p50"], "latency_ms_p99": live["latency_ms_p99"],
            "build_latency_ms_p50": live["build_latency_ms_p50"],
            "build_latency_ms_p99": live["build_latency_ms_p99"],
            "mean_batch": live["mean_batch"], "peak_bytes": live["peak_bytes"],
            "allocator_peak_bytes": live["allocator_peak_bytes"], "realtime": live,
            "sequential_one_at_a_time_ms": seq["wall_s"] * 1e3 / 2}


def run_serve(args):
    clocks = ClockSampler(0)
    clocks.start()
    sv = measure_serve(args.requests, args.rate, args.budget_gb, args.steps,
                       overload_rate=10 * args.rate)
    clock_info = clocks.stop()
    line = {"metric": METRIC, "value": sv["edges_per_s"], "unit": "edges/s", "n_gpus": 1,
            "steps": args.steps, "warmup": 1, "ms_per_step": sv["ms_per_pass"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
            "data": "synthetic", "config": sv["config"], "clocks": clock_info}
    line.update({k: v for k, v in sv.items() if k not in ("config", "edges_per_s", "ms_per_pass")})
    print(json.dumps(line), flush=True)


def run_profile_case(args):
    """Build the workload's graph (dbg_build_reads, the benchmark's step)
    warmup + steps times with the given tuning, check it, print one line:
    the command profilers run (one kernel at a time, on a small workload)."""
    import torch

    from paper_2401_02756_gb300 import build as _build
    from paper_2401_02756_gb300 import dbg, synth
    _build.build()
    dbg.load()
    torch.cuda.set_device(0)
    if args.workload == "batch256":
        return run_profile_batch(args)
    if args.workload == "sizing64":
        return run_profile_sizing(args)
    rs = synth.WORKLOADS[args.workload]()
    packed = torch.from_numpy(np.concatenate([rs.packed, np.zeros(16, np.uint8)])).cuda()
    offsets = torch.from_numpy(rs.offsets.view(np.int64).copy()).cuda()
    touches = int(np.maximum(rs.lengths() - rs.k + 2, 0).sum())
    D = workload_distinct(args.workload)
    if D is None:
        pilot = dbg.Graph(rs.k, int(touches * 1.05) + 1024)
        pilot.insert(packed, offsets)
        D, _ = pilot.stats()
        pilot.close()
    g = dbg.Graph(rs.k, int(math.ceil(1.5 * D)))
    tuning = {kv.split("=")[0]: int(kv.split("=")[1]) for kv in args.tuning.split(",") if kv}
    if tuning:
        g.set_tuning(**tuning)
    for _ in range(args.warmup + args.steps):
        g.build(packed, offsets)
    torch.cuda.synchronize()
    nv, ne = g.stats()
    if g.status() != dbg.OK or nv != D or ne != rs.n_edges():
        raise RuntimeError("profile case: wrong graph")
    if args.profile_export:
        keys = torch.empty(nv, dtype=torch.int64, device="cuda")
        counts = torch.empty((nv, 4), dtype=torch.int32, device="cuda")
        for _ in range(2):
            if g.export_into(keys, counts) != nv:
                raise RuntimeError("profile case: export size")
        del keys, counts
    print(json.dumps({"workload": args.workload, "tuning": tuning or "default", "builds":
                      args.warmup + args.steps, "vertices": nv, "edges": ne, "touches": touches,
                      "table_slots": g.info()["n_slots"], "binned": g.binned_counters()}),
          flush=True)
    g.close()


def run_profile_batch(args):
    """The batched workload's sizing (sketches, one network forward) and its
    batched build (dbg_build_batch), warmup + steps times, with the
    benchmark's chain shape (2^19-slot regions); one summary line."""
    import torch

    from paper_2401_02756_gb300 import dbg
    from paper_2401_02756_gb300.predictor import REG_STRIDE, CapacityPredictor
    samples = gen_batch_samples(256, 4)
    dev = [(torch.from_numpy(np.concatenate([rs.packed, np.zeros(16, np.uint8)])).cuda(),
            torch.from_numpy(rs.offsets.view(np.int64).copy()).cuda()) for rs in samples]
    pred = CapacityPredictor()
    regs = torch.zeros(len(samples), REG_STRIDE, dtype=torch.int32, device="cuda")
    sk = [(rs.k, pk, of, regs[i]) for i, (rs, (pk, of)) in enumerate(zip(samples, dev))]
    dbg.sketch_batch(sk)
    graphs = [dbg.Graph(rs.k, pred.capacity(p))
              for rs, p in zip(samples, pred.predict_registers(regs, len(samples)))]
    for rs, g in zip(samples, graphs):
        g.reserve_events(int(np.maximum(rs.lengths() - rs.k + 2, 0).sum()))
        g.set_tuning(insert_path=2, apply_mode=2, region_log2=19)
    items = [(g, pk, of) for g, (pk, of) in zip(graphs, dev)]
    for _ in range(args.warmup + args.steps):
        dbg.sketch_batch(sk)
        pred.log_vertices(regs, len(samples))
        dbg.build_batch(items)
    torch.cuda.synchronize()
    if any(g.status() != dbg.OK for g in graphs):
        raise RuntimeError("profile case: a batched build failed")
    print(json.dumps({"workload": "batch256", "builds": args.warmup + args.steps,
                      "graphs": len(graphs), "vertices": sum(g.stats()[0] for g in graphs)}),
          flush=True)
    for g in graphs:
        g.close()


def run_profile_sizing(args, n_samples=64):
    """The batched workload's sizing alone on its first 64 samples (about
    1.1e9 vertex positions, 0.3 GB of packed bases: larger than L2, small on
    the device): dbg_sketch_batch and one network forward, warmup + steps
    times; one summary line."""
    import torch

    from paper_2401_02756_gb300 import dbg
    from paper_2401_02756_gb300.predictor import REG_STRIDE, CapacityPredictor
    samples = gen_batch_samples(n_samples, 4)
    dev = [(torch.from_numpy(np.concatenate([rs.packed, np.zeros(16, np.uint8)])).cuda(),
            torch.from_numpy(rs.offsets.view(np.int64).copy()).cuda()) for rs in samples]
    pred = CapacityPredictor()
    regs = torch.zeros(len(samples), REG_STRIDE, dtype=torch.int32, device="cuda")
    sk = [(rs.k, pk, of, regs[i]) for i, (rs, (pk, of)) in enumerate(zip(samples, dev))]
    for _ in range(args.warmup + args.steps):
        dbg.sketch_batch(sk)
        pred.log_vertices(regs, len(samples))
    preds = pred.predict_registers(regs, len(samples))
    print(json.dumps({"workload": "sizing64", "sizings": args.warmup + args.steps,
                      "samples": len(samples),
                      "positions": int(sum(np.maximum(rs.lengths() - rs.k + 2, 0).sum()
                                           for rs in samples)),
                      "predicted_vertices": float(sum(p.mlp for p in preds))}), flush=True)


def microsatellite_reads(n_per_period=20000, read_len=150, seed=5):
    """Low-complexity reads: a random unit of 1..6 bases repeated over the
    whole read (microsatellites), n_per_period reads per unit length -- every
    warp of the direct insert then sees the same few keys many times."""
    from paper_2401_02756_gb300 import synth
    reads = []
    for period in range(1, 7):
        u = synth.draws(seed, 90 + period, n_per_period * period)
        units = (u % 4).astype(np.uint8).reshape(n_per_period, period)
        for unit in units:
            reads.append(synth.codes_to_ascii(np.resize(unit, read_len)))
    return synth.from_strings(reads, 31, "microsatellites")


def run_agg_study(args):
    """The direct insert (insert_path = 1) with warp aggregation off and on
    (__match_any_sync on the key, then on (slot, label)): the 100 Mbp
    workload, where a warp's 32 positions are 32 consecutive k-mers of one
    read (distinct keys), and microsatellite reads, where they repeat.  One
    JSON line per (workload, setting): mean build ms over the steps."""
    import torch

    from paper_2401_02756_gb300 import build as _build
    from paper_2401_02756_gb300 import dbg, synth
    _build.build()
    dbg.load()
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    for name in ("100mbp_30x_k31", "microsatellites"):
        rs = synth.WORKLOADS[name]() if name in synth.WORKLOADS else microsatellite_reads()
        packed = torch.from_numpy(np.concatenate([rs.packed, np.zeros(16, np.uint8)])).cuda()
        offsets = torch.from_numpy(rs.offsets.view(np.int64).copy()).cuda()
        touches = int(np.maximum(rs.lengths() - rs.k + 2, 0).sum())
        D = workload_distinct(name)
        cap = int(math.ceil(1.5 * D)) if D else max(1024, touches // 4)
        g = dbg.Graph(rs.k, cap)
        ref = None
        for agg in (0, 1):
            g.set_tuning(insert_path=1, warp_aggregate=agg)
            for _ in range(args.warmup):
                g.build(packed, offsets, stream=stream)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for _ in range(args.steps):
                g.build(packed, offsets, stream=stream)
            b.record(stream)
            torch.cuda.synchronize()
            st = g.stats()
            ref = ref or st
            if g.status() != dbg.OK or st != ref:
                raise RuntimeError(f"{name}: build differs with warp_aggregate={agg}")
            ms = a.elapsed_time(b) / args.steps
            print(json.dumps({"workload": name, "warp_aggregate": agg, "build_ms": ms,
                              "edges": rs.n_edges(), "edges_per_s": rs.n_edges() / (ms / 1e3),
                              "distinct_vertices": st[0], "table_slots": cap}), flush=True)
        g.close()
        del packed, offsets
        torch.cuda.empty_cache()


def run_probe_sweep(window_only=False):
    """Random 32-byte-sector probe (K5) rate over buffer sizes, one JSON line each."""
    import torch

    from paper_2401_02756_gb300 import build as _build
    from paper_2401_02756_gb300 import dbg
    _build.build()
    dbg.load()
    n_ops = 1 << 30
    sizes = [] if window_only else [1 << 18, 1 << 20, 1 << 21, 1 << 22, 1 << 23, 1 << 24, 1 << 26,
                                    1 << 28, 633846003]
    for n_slots in sizes:
        buf = torch.zeros(n_slots * 32, dtype=torch.uint8, device="cuda")
        for mode in (0, 1, 2):
            dbg.probe_random_sectors(buf, n_slots, 1 << 26, 3, mode, None)
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            dbg.probe_random_sectors(buf, n_slots, n_ops, 5 + mode, mode, None)
            b.record()
            torch.cuda.synchronize()
            ms = a.elapsed_time(b)
            print(json.dumps({"n_slots": n_slots, "MB": n_slots * 32 / 2 ** 20, "mode": mode,
                              "ms": ms, "Gops": n_ops / ms / 1e6}), flush=True)
        del buf
        torch.cuda.empty_cache()
    # a window sliding across a table-sized buffer (the binned apply's pattern)
    n_slots = 633846003
    buf = torch.zeros(n_slots * 32, dtype=torch.uint8, device="cuda")
    n_ops = 2420000000
    for flags in (0, 1):
        for wlog in (15, 17, 19, 20, 21, 23):
            dbg.probe_window(buf, n_slots, 1 << 26, 1 << wlog, 3, flags, None)
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            dbg.probe_window(buf, n_slots, n_ops, 1 << wlog, 9, flags, None)
            b.record()
            torch.cuda.synchronize()
            ms = a.elapsed_time(b)
            print(json.dumps({"n_slots": n_slots, "window_slots": 1 << wlog,
                              "window_MB": (1 << wlog) * 32 / 2 ** 20,
                              "mode": "window" + ("+evict_last" if flags else ""), "ms": ms,
                              "Gops": n_ops / ms / 1e6}), flush=True)


def main():
    args = parse_args()
    if args.probe_sweep or args.window_sweep:
        run_probe_sweep(window_only=args.window_sweep)
    elif args.agg_study:
        run_agg_study(args)
    elif args.profile_case:
        run_profile_case(args)
    elif args.workload == "batch256" and args.impl == "ours":
        run_batch(args)
    elif args.workload == "serve" and args.impl == "ours":
        run_serve(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
