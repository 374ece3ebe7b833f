"""Request loop: build many graphs concurrently under a device-memory budget.

A request is one read set (2-bit packed bases and read offsets in host
memory) and a k; its answer is the sorted graph (the same arrays as
``dbg_export_sorted``).  The loop does continuous batching: requests that
arrive while others are on the GPU are admitted as soon as memory allows,
and every admitted request that is ready joins the next batched insert, so
the work of many requests overlaps on the device.

Stages of one request, each on its own CUDA stream:

1. **ingest** -- its reads are copied to the device and sketched
   (``dbg_sketch_reads``); admission reserves the bytes of its inputs.
   Requests admitted in the same loop iteration are sized together by one
   batched network forward (``dbg_mlp_forward``).
2. **build** -- its table (``table_bytes(capacity)`` for the predicted
   capacity) is reserved against the budget, laid out in memory taken from
   the PyTorch caching allocator (``dbg_create_on``: no cudaMalloc, no
   device synchronisation), and built with every other ready request in one
   ``dbg_build_batch`` call: binned chains that take all of the batch's
   tables in one launch of each binned kernel, each request's event room
   (its vertex positions, counted on the host) reserved towards the
   library's chain buffers.
3. **export** -- a worker thread checks the status, exports the sorted graph
   into pinned host buffers and hands it to the caller's sink, then
   releases the request's memory.  Tables stay device-resident until then.

Overflow is handled exactly: a table whose status reports that it ran out of
room is rebuilt at twice the capacity from the request's resident inputs.

Footprint admitted = packed bytes + offsets bytes + registers + table bytes
+ the export's device buffers (24 bytes a vertex) and the library's sort
scratch (4 bytes a vertex) for the vertices the table is sized for, held
under ``budget_bytes`` together with the buffers the library keeps for the
binned chains (``dbg_scratch_bytes``; they grow to the largest batch and
stay): a batch is cut short when the growth it needs does not fit.  Every
device byte the server uses comes from the PyTorch allocator except the
library's; a report gives both the accounted peak and the allocator's own.
"""

from __future__ import annotations

import math
import queue
import threading
import time
from collections import deque
from dataclasses import dataclass, field

import numpy as np

from . import dbg
from .predictor import REG_STRIDE, CapacityPredictor, Prediction


@dataclass
class Request:
    rid: int
    k: int
    packed: np.ndarray          # uint8, 2-bit packed bases (host; pinned for speed)
    offsets: np.ndarray         # uint64 [n_reads + 1]
    arrival: float = 0.0        # seconds after the start of the run
    edges: int = 0

    @property
    def n_reads(self) -> int:
        return int(self.offsets.size - 1)

    def input_bytes(self) -> int:
        return _round(self.packed.size + 16) + _round(self.offsets.size * 8) + REG_STRIDE * 4


@dataclass
class Timing:
    rid: int
    arrival: float
    admitted: float = math.nan   # inputs admitted
    built: float = math.nan      # build finished (first seen by the export worker)
    done: float = math.nan       # export in host memory, handed to the sink
    capacity: int = 0
    vertices: int = 0
    edges: int = 0
    rebuilds: int = 0


@dataclass
class Report:
    timings: list = field(default_factory=list)
    wall: float = 0.0
    peak_bytes: int = 0          # the largest footprint the budget accounting held
    allocator_peak_bytes: int = 0  # what the PyTorch allocator held for the run, at most
    batches: int = 0
    batch_sizes: list = field(default_factory=list)

    def latencies(self, end: str = "done") -> np.ndarray:
        return np.array([getattr(t, end) - t.arrival for t in self.timings])

    def summary(self) -> dict:
        lat = self.latencies() * 1e3
        blt = self.latencies("built") * 1e3
        edges = sum(t.edges for t in self.timings)
        return {"requests": len(self.timings), "edges": int(edges),
                "wall_s": self.wall, "edges_per_s": edges / self.wall if self.wall else None,
                "latency_ms_p50": float(np.percentile(lat, 50)),
                "latency_ms_p99": float(np.percentile(lat, 99)),
                "build_latency_ms_p50": float(np.percentile(blt, 50)),
                "build_latency_ms_p99": float(np.percentile(blt, 99)),
                "peak_bytes": int(self.peak_bytes),
                "allocator_peak_bytes": int(self.allocator_peak_bytes),
                "batches": self.batches,
                "mean_batch": float(np.mean(self.batch_sizes)) if self.batch_sizes else 0.0,
                "rebuilds": int(sum(t.rebuilds for t in self.timings))}


def _round(n: int) -> int:
    return (int(n) + 511) // 512 * 512


EXPORT_BYTES_PER_VERTEX = 8 + 16 + 4  # device keys and counters, and the sort's index scratch
EXPORT_BYTES_FIXED = 8 << 20          # the sort's histograms, at most (checked per export)


def chain_events(positions: int) -> int:
    """Events a binned chain reserves for a read set of ``positions`` vertex
    positions (dbg_reserve_events: the positions plus its bucket margin)."""
    return positions + positions // 16 + 65536 + 256 * 2048


def chain_scratch_bytes(events: int) -> int:
    """Device bytes of the library's chain buffers for ``events`` events, a
    little over: the first event buffer (8 bytes each), the second (1.125
    times as large plus 2^20 events) and about 48 MB of bookkeeping."""
    return int((8 * events + 8 * (events + events // 8 + (1 << 20)) + (48 << 20)) * 1.03)


def table_footprint(capacity: int, expected_vertices: float) -> int:
    """Device bytes a request's table accounts for from its build to the end
    of its export: the table, and the export's device buffers for the
    vertices it is expected to hold."""
    return (_round(dbg.table_bytes(capacity)) +
            _round(expected_vertices * EXPORT_BYTES_PER_VERTEX + EXPORT_BYTES_FIXED))


class _Job:
    """A request in flight: its device inputs, table and timing."""

    __slots__ = ("req", "timing", "packed", "offsets", "regs", "reserved", "table_bytes",
                 "export_bytes", "capacity", "graph", "mem", "ingest_ev", "positions")

    def __init__(self, req: Request, timing: Timing):
        self.req, self.timing = req, timing
        self.packed = self.offsets = self.regs = self.graph = self.mem = self.ingest_ev = None
        self.reserved = self.table_bytes = self.export_bytes = 0
        self.capacity = 0
        ln = np.diff(req.offsets.astype(np.int64))
        self.positions = int(np.maximum(ln - req.k + 2, 0).sum())


class _Exporter:
    """An export worker's stream and its pinned host output buffers."""

    def __init__(self, device):
        import torch
        self.stream = torch.cuda.Stream(device)
        self.rows = 0
        self.keys = self.counts = None

    def buffers(self, rows: int):
        """(keys uint64 [>= rows], counts uint32 [>= rows, 4]), pinned, reused."""
        import torch
        if rows > self.rows:
            rows = max(rows, 2 * self.rows)
            self.keys_t = torch.empty(rows, dtype=torch.int64, pin_memory=True)
            self.counts_t = torch.empty((rows, 4), dtype=torch.int32, pin_memory=True)
            self.keys = self.keys_t.numpy().view(np.uint64)
            self.counts = self.counts_t.numpy().view(np.uint32)
            self.rows = rows
        return self.keys, self.counts

    @staticmethod
    def scratch_need(graph, n: int) -> int:
        """Device bytes of the export's sort scratch for ``n`` vertices."""
        return dbg.export_scratch_bytes(graph.k, max(1, n), graph.info()["n_slots"])

    def export(self, graph, n: int, s):
        """The sorted graph of ``n`` vertices in pinned host memory: exported
        into device buffers on ``s`` (dbg_export_sorted_with: every byte from
        the PyTorch allocator, none from the library's pool), then copied;
        views [:n] are returned."""
        import torch
        keys, counts = self.buffers(max(1, n))
        if n == 0:
            return keys[:0], counts[:0]
        with torch.cuda.stream(s):
            kd = torch.empty(n, dtype=torch.int64, device=s.device)
            cd = torch.empty((n, 4), dtype=torch.int32, device=s.device)
            scratch = torch.empty(self.scratch_need(graph, n), dtype=torch.uint8, device=s.device)
        if graph.export_with(kd, cd, scratch, s) != n:
            raise RuntimeError("export: vertex count changed")
        with torch.cuda.stream(s):
            self.keys_t[:n].copy_(kd, non_blocking=True)
            self.counts_t[:n].copy_(cd, non_blocking=True)
        s.synchronize()
        return keys[:n], counts[:n]


class BuildServer:
    """Continuous-batching graph builds under a device-memory budget."""

    def __init__(self, predictor: CapacityPredictor | None = None, budget_bytes: float = 150e9,
                 headroom: float = 1.5, max_batch: int = 128, export_workers: int = 4,
                 device="cuda", tuning: dict | None = None):
        import torch
        self.device = torch.device(device)
        self.tuning = dict(tuning or {})  # every table's launch shape (autotune.tune_batch)
        self._lib = 0  # bytes accounted for the library's chain buffers
        self.predictor = predictor or CapacityPredictor(device=device)
        self.budget = int(budget_bytes)
        self.headroom = headroom
        self.max_batch = max_batch
        self.s_ingest = torch.cuda.Stream(self.device)
        self.s_build = torch.cuda.Stream(self.device)
        # one stream and one growable pinned output buffer per export worker
        self._exporters = [_Exporter(self.device) for _ in range(max(1, export_workers))]
        self._lock = threading.Lock()
        self._used = 0
        self._peak = 0

    def reserve_host_rows(self, rows: int) -> None:
        """Size every export worker's pinned output buffers for graphs of
        ``rows`` vertices now (pinning host memory takes time: better before
        requests arrive than on their path)."""
        for ex in self._exporters:
            ex.buffers(rows)

    # -- memory accounting ------------------------------------------------------
    def _reserve(self, n: int, force: bool = False) -> bool:
        with self._lock:
            if self._used + n > self.budget and not force:
                return False
            self._used += n
            self._peak = max(self._peak, self._used)
            return True

    def _release(self, n: int) -> None:
        with self._lock:
            self._used -= n

    # -- stages -----------------------------------------------------------------
    def _ingest(self, jobs: list[_Job], now: float):
        """Copy inputs, sketch them and size them in one batched forward (ingest stream)."""
        import torch
        s = self.s_ingest
        with torch.cuda.stream(s):
            regs = torch.empty(len(jobs), REG_STRIDE, dtype=torch.int32, device=self.device)
            for i, j in enumerate(jobs):
                r = j.req
                j.packed = torch.empty(r.packed.size + 16, dtype=torch.uint8, device=self.device)
                j.packed[:r.packed.size].copy_(torch.from_numpy(r.packed), non_blocking=True)
                j.offsets = torch.from_numpy(r.offsets.view(np.int64)).to(self.device,
                                                                           non_blocking=True)
                dbg.sketch(r.k, j.packed, j.offsets, registers=regs[i], stream=s)
                j.timing.admitted = now
            y = self.predictor.log_vertices(regs, len(jobs), stream=s)
            y_host = torch.empty(len(jobs), dtype=torch.float32, pin_memory=True)
            regs_host = torch.empty(regs.shape, dtype=torch.int32, pin_memory=True)
            y_host.copy_(y, non_blocking=True)
            regs_host.copy_(regs, non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(s)
        for j in jobs:
            j.regs = regs
            j.ingest_ev = ev
        return jobs, (y_host, regs_host), ev

    def _size(self, jobs, out) -> None:
        y_host, regs_host = out[0].numpy(), out[1].numpy()
        for i, j in enumerate(jobs):
            if int(regs_host[i, -1]) != dbg.OK:
                raise dbg.DbgError(int(regs_host[i, -1]), f"sketch of request {j.req.rid}")
            p = Prediction(math.exp(float(y_host[i])),
                           dbg.sketch_estimate(regs_host[i, :dbg.SKETCH_REGISTERS].view(np.uint32)))
            j.capacity = self.predictor.capacity(p, self.headroom)

    def _make_table(self, j: _Job, capacity: int, s, force: bool = False,
                    lib_extra: int = 0, direct: bool = False) -> bool:
        """Reserve and lay out a table for the job, initialised on stream ``s``;
        False if it does not fit in the budget (unless ``force``).  The
        reservation covers the export's buffers too (``table_footprint``),
        for as many vertices as the table was sized for, and ``lib_extra``
        bytes of growth of the library's chain buffers."""
        import torch
        # (the prediction times its margin: the most vertices it allows for)
        nbytes = table_footprint(capacity, capacity / self.headroom)
        if not self._reserve(nbytes + lib_extra, force):
            return False
        with self._lock:
            self._lib += lib_extra
        j.reserved += nbytes
        j.table_bytes = nbytes
        j.export_bytes = nbytes - _round(dbg.table_bytes(capacity))
        with torch.cuda.stream(s):
            j.mem = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        j.graph = dbg.Graph(j.req.k, capacity, memory=j.mem, stream=s)
        if direct:  # the batch's chain buffers would not fit the budget
            j.graph.set_tuning(insert_path=1)
        else:
            if self.tuning:
                j.graph.set_tuning(**self.tuning)
            j.graph.reserve_events(j.positions)  # (its share of the chain buffers: no allocation)
        j.capacity = j.timing.capacity = capacity
        return True

    def _sync_library_bytes(self) -> None:
        """Account what the library really holds (its buffers grew to a batch's
        chain: taken even past the budget; the report's peak shows it)."""
        held = dbg.scratch_bytes()
        with self._lock:
            if held > self._lib:
                self._used += held - self._lib
                self._lib = held
                self._peak = max(self._peak, self._used)

    def _launch(self, batch: list[_Job]) -> object:
        import torch
        s = self.s_build
        seen = set()
        for j in batch:
            if id(j.ingest_ev) not in seen:
                s.wait_event(j.ingest_ev)
                seen.add(id(j.ingest_ev))
        # every table is new: a build (the binned chains' apply then writes each
        # table tile by tile without reading it)
        dbg.build_batch([(j.graph, j.packed, j.offsets) for j in batch], stream=s)
        ev = torch.cuda.Event()
        ev.record(s)
        return ev

    def _finish(self, j: _Job, t0: float, sink, ex: "_Exporter") -> None:
        """Export worker: check, rebuild on overflow, export, hand over, release."""
        s = ex.stream
        while True:
            st = j.graph.status(s)
            if st == dbg.OK:
                break
            if st not in (dbg.ERR_CAPACITY, dbg.ERR_NEEDS_GROW):
                raise dbg.DbgError(st, f"request {j.req.rid}")
            # exact fallback: a fresh table at twice the size, built from the
            # resident inputs.  Only the export workers release memory, so the
            # rebuild cannot wait for room: it takes it even past the budget
            # (the report's peak shows it).
            j.graph.close()
            j.mem = None
            self._release(j.table_bytes)
            j.reserved -= j.table_bytes
            j.timing.rebuilds += 1
            self._make_table(j, 2 * j.capacity, s, force=True)
            j.graph.set_tuning(insert_path=1)  # (alone: the direct insert, no chain buffers)
            j.graph.build(j.packed, j.offsets, stream=s)
        # the sorted export: into device buffers from the allocator (the sort
        # then runs inside them, with 4 bytes a vertex of library scratch),
        # accounted against the budget while they live, then to pinned host
        # memory.  Only the export workers release memory, so this takes its
        # room even past the budget rather than wait (the peak shows it).
        nv, ne = j.graph.stats(s)
        # (reserved with the table for the expected vertex count; more
        # vertices than that take the difference, past the budget if need be)
        xb = max(0, _round(nv * 24 + ex.scratch_need(j.graph, nv)) - j.export_bytes)
        self._reserve(xb, force=True)
        try:
            keys, counts = ex.export(j.graph, nv, s)
        finally:
            self._release(xb)
        j.timing.vertices, j.timing.edges = nv, ne
        j.timing.done = time.perf_counter() - t0
        if sink is not None:
            sink(j.req, keys, counts)
        for t in (j.mem, j.packed, j.offsets, j.regs):
            if t is not None:
                t.record_stream(s)
        j.graph.close()
        j.graph = j.mem = j.packed = j.offsets = j.regs = None
        self._release(j.reserved)
        j.reserved = 0

    # -- the loop ---------------------------------------------------------------
    def run(self, requests: list[Request], sink=None, realtime: bool = True) -> Report:
        """Serve ``requests`` (arrival times in seconds from now when
        ``realtime``, else all at once) and return their timings.  ``sink(req,
        keys, counts)`` receives each sorted graph (host arrays, valid during
        the call only)."""
        import torch
        reqs = sorted(requests, key=lambda r: r.arrival)
        n = len(reqs)
        timings = {r.rid: Timing(r.rid, r.arrival if realtime else 0.0) for r in reqs}
        report = Report()
        # the library's buffers count against the budget; more of them than
        # a third of it (left by earlier work in this process) are given back
        # first (dbg_release_scratch synchronises the device)
        if dbg.scratch_bytes() > self.budget / 3:
            dbg.release_scratch()
            with self._lock:
                self._used -= self._lib
                self._lib = 0
        self._sync_library_bytes()
        with self._lock:
            self._peak = self._used  # the peak of this run only
        torch.cuda.reset_peak_memory_stats(self.device)
        alloc0 = torch.cuda.memory_allocated(self.device)
        done_q: queue.Queue = queue.Queue()
        work_q: queue.Queue = queue.Queue()
        errors: list = []
        t0 = time.perf_counter()

        def worker(ex):
            while True:
                j = work_q.get()
                if j is None:
                    return
                try:
                    self._finish(j, t0, sink, ex)
                except Exception as e:  # surfaced to the caller below
                    errors.append(e)
                done_q.put(j)

        threads = [threading.Thread(target=worker, args=(ex,), daemon=True)
                   for ex in self._exporters]
        for th in threads:
            th.start()
        building: deque = deque()   # (batch, event) in launch order
        nxt = 0
        pending: deque = deque()
        ingesting: deque = deque()   # (jobs, pinned predictions, event)
        sized: deque = deque()
        finished = in_flight = 0
        try:
            while finished < n and not errors:
                now = time.perf_counter() - t0
                while nxt < n and (not realtime or reqs[nxt].arrival <= now):
                    pending.append(_Job(reqs[nxt], timings[reqs[nxt].rid]))
                    nxt += 1
                # 1. admit inputs while they fit, and only while no sized request
                #    waits for table memory (inputs must not starve tables)
                admit = []
                while pending and not sized and len(admit) < self.max_batch:
                    j = pending[0]
                    nb = j.req.input_bytes()
                    # a request alone on an idle server is always admitted
                    idle = in_flight == 0 and not ingesting and not admit
                    if not self._reserve(nb, idle):
                        break
                    j.reserved += nb
                    admit.append(pending.popleft())
                if admit:
                    ingesting.append(self._ingest(admit, now))
                # 2. size what finished ingesting
                while ingesting and ingesting[0][2].query():
                    jobs, out, _ = ingesting.popleft()
                    self._size(jobs, out)
                    sized.extend(jobs)
                # 3. tables for sized jobs while memory allows (with the growth
                #    of the library's chain buffers the batch needs), then one
                #    batched insert
                batch = []
                events = 0
                direct = None  # the batch's first request decides: chains or direct
                while sized and len(batch) < self.max_batch:
                    j = sized[0]
                    # with nothing in flight no memory will come back: the
                    # head request then takes its table past the budget
                    force = in_flight == 0 and not batch
                    ev = events + chain_events(j.positions)
                    extra = max(0, chain_scratch_bytes(ev) - self._lib)
                    if direct is None:
                        # chain buffers that do not fit now, or would keep more
                        # than a third of the budget: the direct insert
                        need = table_footprint(j.capacity, j.capacity / self.headroom)
                        direct = extra > 0 and (self._used + need + extra > self.budget or
                                                self._lib + extra > self.budget / 3)
                    if direct:
                        extra = 0
                    if not self._make_table(j, j.capacity, self.s_build, force, extra, direct):
                        break
                    events = ev
                    batch.append(sized.popleft())
                if batch:
                    in_flight += len(batch)
                    building.append((batch, self._launch(batch)))
                    self._sync_library_bytes()
                    report.batches += 1
                    report.batch_sizes.append(len(batch))
                # 4. builds that completed go to the export workers
                progressed = bool(admit or batch)
                while building and building[0][1].query():
                    done_batch, _ = building.popleft()
                    t_built = time.perf_counter() - t0
                    for j in done_batch:
                        j.timing.built = t_built
                        work_q.put(j)
                    progressed = True
                # 5. collect finished requests
                while True:
                    try:
                        done_q.get_nowait()
                    except queue.Empty:
                        break
                    finished += 1
                    in_flight -= 1
                    progressed = True
                if not progressed:
                    if nxt < n and not pending and not ingesting and not sized:
                        wait = reqs[nxt].arrival - (time.perf_counter() - t0)
                        time.sleep(min(max(wait, 0.0), 0.002))
                    else:
                        time.sleep(0.0002)
        finally:
            for th in threads:
                work_q.put(None)
            for th in threads:
                th.join()
        if errors:
            raise errors[0]
        report.wall = time.perf_counter() - t0
        report.timings = [timings[r.rid] for r in reqs]
        report.peak_bytes = self._peak
        report.allocator_peak_bytes = torch.cuda.max_memory_allocated(self.device) - alloc0
        return report


def sequential(requests: list[Request], predictor: CapacityPredictor, sink=None,
               realtime: bool = True, headroom: float = 1.5, exporter=None) -> Report:
    """The same requests served one at a time with plain calls: for each, in
    arrival order, copy its reads to the device, sketch and size it, create a
    table, insert, export (into the same kind of reused pinned buffer as the
    server's; ``exporter`` keeps it across calls), destroy (first come, first
    served)."""
    import torch
    reqs = sorted(requests, key=lambda r: r.arrival)
    report = Report()
    s = torch.cuda.current_stream()
    ex = exporter or _Exporter(torch.device("cuda"))
    t0 = time.perf_counter()
    for r in reqs:
        if realtime:
            wait = r.arrival - (time.perf_counter() - t0)
            if wait > 0:
                time.sleep(wait)
        t = Timing(r.rid, r.arrival if realtime else 0.0)
        t.admitted = time.perf_counter() - t0
        packed = torch.empty(r.packed.size + 16, dtype=torch.uint8, device="cuda")
        packed[:r.packed.size].copy_(torch.from_numpy(r.packed))
        offsets = torch.from_numpy(r.offsets.view(np.int64)).cuda()
        pred = predictor.predict(r.k, packed, offsets)
        g = dbg.Graph(r.k, predictor.capacity(pred, headroom))
        g.build(packed, offsets)
        while g.status() != dbg.OK:  # exact fallback, as in the server
            cap = 2 * g.info()["n_slots"]
            g.close()
            g = dbg.Graph(r.k, cap)
            g.build(packed, offsets)
            t.rebuilds += 1
        s.synchronize()
        t.built = time.perf_counter() - t0
        t.capacity = g.info()["n_slots"]
        t.vertices, t.edges = g.stats()
        keys, counts = ex.export(g, t.vertices, s)
        g.close()
        t.done = time.perf_counter() - t0
        if sink is not None:
            sink(r, keys, counts)
        report.timings.append(t)
    report.wall = time.perf_counter() - t0
    return report


