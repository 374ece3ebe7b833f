"""Thin ctypes binding of ``libdbg.so`` (the C ABI in ``include/dbg.h``).

Argument marshalling only: every step of the graph build runs in the
library's CUDA kernels.  Device buffers are passed as PyTorch CUDA tensors
(or anything with ``data_ptr()``), host buffers as numpy arrays, and streams
as ``torch.cuda.Stream`` objects or raw ``cudaStream_t`` integers
(``None`` = PyTorch's current stream).  The library must have been built
(``paper_2401_02756_gb300.build.build()``); there is no fallback.
"""

from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libdbg.so")

(OK, ERR_INVALID_ARG, ERR_OOM, ERR_CAPACITY, ERR_CUDA, ERR_BUFFER_TOO_SMALL, ERR_BAD_OFFSETS,
 ERR_NOALLOC_LIMIT, ERR_NEEDS_GROW, ERR_TIMEOUT) = range(10)
STATUS_NAMES = {0: "DBG_OK", 1: "DBG_ERR_INVALID_ARG", 2: "DBG_ERR_OOM", 3: "DBG_ERR_CAPACITY",
                4: "DBG_ERR_CUDA", 5: "DBG_ERR_BUFFER_TOO_SMALL", 6: "DBG_ERR_BAD_OFFSETS",
                7: "DBG_ERR_NOALLOC_LIMIT", 8: "DBG_ERR_NEEDS_GROW", 9: "DBG_ERR_TIMEOUT"}
NOALLOC_EXPORT_MAX_VERTICES = 1 << 19

EXPORTED = [
    "dbg_create", "dbg_create_ex", "dbg_table_bytes", "dbg_create_on", "dbg_destroy", "dbg_reset", "dbg_set_tuning", "dbg_get_info",
    "dbg_reserve_events", "dbg_enable_kernel_timing", "dbg_kernel_times", "dbg_binned_counters",
    "dbg_set_spill",
    "dbg_grow",
    "dbg_insert_reads", "dbg_insert_reads_host", "dbg_build_reads", "dbg_build_reads_host",
    "dbg_insert_batch", "dbg_build_batch", "dbg_release_scratch", "dbg_scratch_bytes",
    "dbg_get_status", "dbg_stats",
    "dbg_export_sorted", "dbg_export_sorted_noalloc", "dbg_export_scratch_bytes",
    "dbg_export_sorted_with", "dbg_normalize", "dbg_find_contigs", "dbg_pack_ascii", "dbg_strerror", "dbg_last_cuda_error",
    "dbg_probe_random_sectors", "dbg_probe_window", "dbg_sketch_reads", "dbg_sketch_batch",
    "dbg_sketch_estimate",
    "dbg_mlp_work_floats", "dbg_mlp_features", "dbg_mlp_init", "dbg_mlp_forward",
    "dbg_mlp_train_step", "dbg_binary_version",
]
MLP_INPUTS, MLP_HIDDEN, MLP_PARAMS = 1024, 64, 69825
SKETCH_REGISTERS = 1024


class DbgError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        msg = f"{what}: {STATUS_NAMES.get(code, code)} ({_strerror(code)})"
        if code == ERR_CUDA:
            msg += f" [{last_cuda_error()}]"
        super().__init__(msg)


class Tuning(ctypes.Structure):
    _fields_ = [("block_threads", ctypes.c_int), ("tile_reads", ctypes.c_int),
                ("grid_ctas", ctypes.c_int), ("warp_aggregate", ctypes.c_int),
                ("insert_path", ctypes.c_int), ("apply_unroll", ctypes.c_int),
                ("apply_chunk", ctypes.c_int), ("apply_ctas", ctypes.c_int),
                ("apply_counters", ctypes.c_int), ("region_log2", ctypes.c_int),
                ("apply_group", ctypes.c_int), ("apply_mode", ctypes.c_int),
                ("scatter_reads", ctypes.c_int), ("split_threads", ctypes.c_int)]


class Info(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int), ("n_slots", ctypes.c_uint64), ("table_bytes", ctypes.c_uint64),
                ("max_probes", ctypes.c_uint32), ("device", ctypes.c_int),
                ("event_capacity", ctypes.c_uint64), ("spill_capacity", ctypes.c_uint64)]


class SketchItem(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int), ("packed", ctypes.c_void_p), ("offsets", ctypes.c_void_p),
                ("n_reads", ctypes.c_uint64), ("registers", ctypes.c_void_p)]


class BatchItem(ctypes.Structure):
    _fields_ = [("graph", ctypes.c_void_p), ("packed", ctypes.c_void_p),
                ("offsets", ctypes.c_void_p), ("n_reads", ctypes.c_uint64)]


_lib = None


def load() -> ctypes.CDLL:
    """Load ``libdbg.so``; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is not built: call paper_2401_02756_gb300.build.build() "
                           "(needs nvcc); there is no CPU fallback")
    L = ctypes.CDLL(LIB_PATH)
    P, U64, U32, I = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int
    sig = {
        "dbg_create": (I, [I, U64, ctypes.POINTER(P)]),
        "dbg_create_ex": (I, [I, U64, U32, ctypes.POINTER(P)]),
        "dbg_table_bytes": (U64, [U64]),
        "dbg_create_on": (I, [I, U64, U32, P, U64, P, ctypes.POINTER(P)]),
        "dbg_destroy": (None, [P]),
        "dbg_reset": (I, [P, P]),
        "dbg_set_tuning": (I, [P, ctypes.POINTER(Tuning)]),
        "dbg_get_info": (I, [P, ctypes.POINTER(Info)]),
        "dbg_reserve_events": (I, [P, U64]),
        "dbg_set_spill": (I, [P, U64]),
        "dbg_grow": (I, [P, U64, P]),
        "dbg_enable_kernel_timing": (I, [P, I]),
        "dbg_kernel_times": (I, [P, ctypes.POINTER(ctypes.c_float), I, ctypes.POINTER(I)]),
        "dbg_binned_counters": (I, [P, ctypes.POINTER(U64)]),
        "dbg_insert_reads": (I, [P, P, P, U64, P]),
        "dbg_insert_reads_host": (I, [P, P, P, U64, P]),
        "dbg_build_reads": (I, [P, P, P, U64, P]),
        "dbg_build_reads_host": (I, [P, P, P, U64, P]),
        "dbg_insert_batch": (I, [ctypes.POINTER(BatchItem), I, P]),
        "dbg_build_batch": (I, [ctypes.POINTER(BatchItem), I, P]),
        "dbg_release_scratch": (I, []),
        "dbg_scratch_bytes": (U64, []),
        "dbg_get_status": (I, [P, P]),
        "dbg_stats": (I, [P, ctypes.POINTER(U64), ctypes.POINTER(U64), P]),
        "dbg_export_sorted": (I, [P, P, P, U64, ctypes.POINTER(U64), P]),
        "dbg_export_sorted_noalloc": (I, [P, P, P, U64, ctypes.POINTER(U64), P]),
        "dbg_export_scratch_bytes": (U64, [I, U64, U64]),
        "dbg_export_sorted_with": (I, [P, P, P, U64, ctypes.POINTER(U64), P, U64, P]),
        "dbg_normalize": (I, [P, ctypes.c_double, P]),
        "dbg_find_contigs": (I, [P, P, U64, P, U64, ctypes.POINTER(U64), ctypes.POINTER(U64), P]),
        "dbg_pack_ascii": (I, [ctypes.c_char_p, U64, P, I, ctypes.POINTER(U64)]),
        "dbg_strerror": (ctypes.c_char_p, [I]),
        "dbg_last_cuda_error": (ctypes.c_char_p, []),
        "dbg_binary_version": (I, [ctypes.POINTER(I)]),
        "dbg_probe_random_sectors": (I, [P, U64, U64, U64, I, P]),
        "dbg_probe_window": (I, [P, U64, U64, U64, U64, I, P]),
        "dbg_sketch_reads": (I, [I, P, P, U64, P, P]),
        "dbg_sketch_estimate": (ctypes.c_double, [P]),
        "dbg_sketch_batch": (I, [P, I, P]),
        "dbg_mlp_work_floats": (U64, [I]),
        "dbg_mlp_features": (I, [P, ctypes.c_int64, I, P, P]),
        "dbg_mlp_init": (I, [P, U64, P]),
        "dbg_mlp_forward": (I, [P, P, I, P, P, P]),
        "dbg_mlp_train_step": (I, [P, P, P, P, I, ctypes.c_float, P, P, I, P, P, P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def _strerror(code: int) -> str:
    try:
        return load().dbg_strerror(code).decode()
    except Exception:  # pragma: no cover - only when the library is missing
        return "?"


def last_cuda_error() -> str:
    return load().dbg_last_cuda_error().decode()


def _check(code: int, what: str) -> None:
    if code != OK:
        raise DbgError(code, what)


def _stream(stream) -> int | None:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream or None
    if isinstance(stream, int):
        return stream or None
    return getattr(stream, "cuda_stream", None) or None


def _dptr(x) -> int:
    """Device pointer of a CUDA tensor (or an int)."""
    if isinstance(x, int):
        return x
    if hasattr(x, "is_cuda") and not x.is_cuda:
        raise ValueError("expected a CUDA tensor")
    return int(x.data_ptr())


def _hptr(a: np.ndarray) -> int:
    if not isinstance(a, np.ndarray):
        a = np.asarray(a)
    if not a.flags["C_CONTIGUOUS"]:
        raise ValueError("host array must be contiguous")
    return int(a.ctypes.data) if a.size else 0


def _host_view(x, dtype):
    """numpy view of a host buffer (numpy array or CPU tensor, pinned or not)."""
    if hasattr(x, "numpy"):
        return x.numpy().view(dtype)
    return np.ascontiguousarray(x).view(dtype)


class Graph:
    """An A-Bruijn graph under construction, held in device memory."""

    def __init__(self, k: int, capacity: int, max_probes: int = 0, memory=None, stream=None):
        """A table of ``capacity`` slots, allocated by the library, or -- when
        ``memory`` (a CUDA uint8 tensor of at least ``table_bytes(capacity)``
        bytes, 256-byte aligned) is given -- laid out in that memory and
        initialized asynchronously on ``stream``.  The graph keeps a reference
        to ``memory``; a caller that uses the graph on other streams than the
        one ``memory`` was allocated on orders the release itself
        (``Tensor.record_stream``)."""
        L = load()
        h = ctypes.c_void_p()
        self._memory = None
        if memory is None:
            _check(L.dbg_create_ex(int(k), int(capacity), int(max_probes), ctypes.byref(h)),
                   "dbg_create")
        else:
            _check(L.dbg_create_on(int(k), int(capacity), int(max_probes), _dptr(memory),
                                   int(memory.numel() * memory.element_size()), _stream(stream),
                                   ctypes.byref(h)), "dbg_create_on")
            self._memory = memory
        self._h = h
        self.k = int(k)

    # -- lifecycle ----------------------------------------------------------
    @property
    def handle(self) -> int:
        if self._h is None:
            raise ValueError("graph is closed")
        return self._h.value

    def close(self) -> None:
        if getattr(self, "_h", None) is not None:
            load().dbg_destroy(self._h)
            self._h = None
        self._memory = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- configuration ------------------------------------------------------
    def info(self) -> dict:
        inf = Info()
        _check(load().dbg_get_info(self.handle, ctypes.byref(inf)), "dbg_get_info")
        return {"k": inf.k, "n_slots": inf.n_slots, "table_bytes": inf.table_bytes,
                "max_probes": inf.max_probes, "device": inf.device,
                "event_capacity": inf.event_capacity, "spill_capacity": inf.spill_capacity}

    TUNING_FIELDS = ("block_threads", "tile_reads", "grid_ctas", "warp_aggregate", "insert_path",
                     "apply_unroll", "apply_chunk", "apply_ctas", "apply_counters", "region_log2",
                     "apply_group", "apply_mode", "scatter_reads", "split_threads")

    def set_tuning(self, **fields) -> None:
        """Launch shape and path of the insert; fields (all optional, 0 = automatic):
        ``block_threads``, ``tile_reads``, ``grid_ctas``, ``warp_aggregate`` (-1/0/1),
        ``insert_path`` (1 direct, 2 binned), ``apply_unroll`` (2/4/8 probe slots per
        thread), ``apply_chunk`` (4/8/16 events per thread per chunk), ``apply_ctas``
        (CTAs per SM), ``apply_counters`` (1..64), ``region_log2`` (16..26),
        ``apply_group`` (regions per apply launch), ``apply_mode`` (1 streaming, 2 tiled),
        ``scatter_reads`` (the binned scatter's reads per tile, 32..512), ``split_threads``
        (the split's CTA size, 256/512/1024).  The built graph does not depend on any of
        these."""
        unknown = set(fields) - set(self.TUNING_FIELDS)
        if unknown:
            raise ValueError(f"unknown tuning fields {sorted(unknown)}")
        vals = {f: 0 for f in self.TUNING_FIELDS}
        vals["warp_aggregate"] = -1
        vals.update(fields)
        t = Tuning(*[int(vals[f]) for f in self.TUNING_FIELDS])
        _check(load().dbg_set_tuning(self.handle, ctypes.byref(t)), "dbg_set_tuning")

    KERNELS = ("direct", "bin_count", "bin_scan", "bin_scatter", "bin_split", "bin_apply",
               "bin_deferred", "direct_fallback")

    def enable_kernel_timing(self, calls: int) -> None:
        """Record CUDA events around each kernel of the next insert calls (keep ``calls``)."""
        _check(load().dbg_enable_kernel_timing(self.handle, int(calls)), "dbg_enable_kernel_timing")

    def kernel_times(self, max_calls: int = 1024) -> np.ndarray:
        """[calls, len(KERNELS)] kernel durations in ms (-1: not launched), oldest first."""
        K = len(self.KERNELS)
        buf = (ctypes.c_float * (K * max_calls))()
        n = ctypes.c_int()
        _check(load().dbg_kernel_times(self.handle, buf, max_calls, ctypes.byref(n)),
               "dbg_kernel_times")
        return np.frombuffer(buf, dtype=np.float32)[: K * n.value].reshape(n.value, K).copy()

    def binned_counters(self) -> dict:
        """The last binned insert call's diagnostics (synchronizes the device):
        whether the binned kernels did its work, and how many events the
        global pass applied -- those whose probe left their tile (deferred)
        and those that did not fit their tile's bucket (overflow)."""
        out = (ctypes.c_uint64 * 3)()
        _check(load().dbg_binned_counters(self.handle, out), "dbg_binned_counters")
        return {"binned": bool(out[0]), "deferred": int(out[1]), "overflow": int(out[2])}

    def set_spill(self, records: int) -> None:
        """Keep vertices that find no slot in a spill buffer of ``records``
        records (0 removes it); complete the graph with :meth:`grow`."""
        _check(load().dbg_set_spill(self.handle, int(records)), "dbg_set_spill")

    def grow(self, new_capacity: int = 0, stream=None) -> None:
        """Rebuild in a table of ``new_capacity`` slots (0: twice the size) and
        replay the spilled vertices."""
        _check(load().dbg_grow(self.handle, int(new_capacity), _stream(stream)), "dbg_grow")

    def reserve_events(self, events: int = 0) -> None:
        """Size the binned insert's event buffer (0 = default, 4 per slot)."""
        _check(load().dbg_reserve_events(self.handle, int(events)), "dbg_reserve_events")

    # -- build --------------------------------------------------------------
    def reset(self, stream=None) -> None:
        _check(load().dbg_reset(self.handle, _stream(stream)), "dbg_reset")

    def insert(self, packed, offsets, n_reads: int | None = None, stream=None) -> None:
        """Insert reads held in device memory (``packed`` uint8, ``offsets``
        int64/uint64 with n_reads + 1 entries)."""
        if n_reads is None:
            n_reads = int(offsets.numel()) - 1
        _check(load().dbg_insert_reads(self.handle, _dptr(packed) or None, _dptr(offsets) or None,
                                       int(n_reads), _stream(stream)), "dbg_insert_reads")

    def insert_host(self, packed, offsets, stream=None) -> None:
        """Insert reads held in host memory (copied by the library, in chunks)."""
        pk = _host_view(packed, np.uint8)
        of = _host_view(offsets, np.uint64)
        _check(load().dbg_insert_reads_host(self.handle, _hptr(pk) or None, _hptr(of) or None,
                                            int(of.size) - 1, _stream(stream)),
               "dbg_insert_reads_host")

    def build(self, packed, offsets, n_reads: int | None = None, stream=None) -> None:
        """Discard the graph and build it from reads in device memory (one
        stream-ordered call: dbg_reset + dbg_insert_reads)."""
        if n_reads is None:
            n_reads = int(offsets.numel()) - 1
        _check(load().dbg_build_reads(self.handle, _dptr(packed) or None, _dptr(offsets) or None,
                                      int(n_reads), _stream(stream)), "dbg_build_reads")

    def build_host(self, packed, offsets, stream=None) -> None:
        """dbg_build_reads with reads in host memory."""
        pk = _host_view(packed, np.uint8)
        of = _host_view(offsets, np.uint64)
        _check(load().dbg_build_reads_host(self.handle, _hptr(pk) or None, _hptr(of) or None,
                                           int(of.size) - 1, _stream(stream)),
               "dbg_build_reads_host")

    # -- results ------------------------------------------------------------
    def status(self, stream=None) -> int:
        return int(load().dbg_get_status(self.handle, _stream(stream)))

    def stats(self, stream=None) -> tuple[int, int]:
        nv, ne = ctypes.c_uint64(), ctypes.c_uint64()
        _check(load().dbg_stats(self.handle, ctypes.byref(nv), ctypes.byref(ne), _stream(stream)),
               "dbg_stats")
        return int(nv.value), int(ne.value)

    def export(self, stream=None, out=None) -> tuple[np.ndarray, np.ndarray]:
        """Sorted vertices: keys (uint64 [D], or [D, 2] high and low words for
        k > 32) and counters (uint32 [D, 4], A C G T).  ``out`` = (keys,
        counts) host arrays (pinned for speed) of at least D rows makes it one
        call into them; the views [:D] are returned."""
        L = load()
        n = ctypes.c_uint64()
        wide = self.k > 32
        if out is not None:
            keys, counts = out
            st = L.dbg_export_sorted(self.handle, keys.ctypes.data, counts.ctypes.data,
                                     min(keys.shape[0], counts.shape[0]), ctypes.byref(n),
                                     _stream(stream))
            if st == OK:
                return keys[:n.value], counts[:n.value]
            if st != ERR_BUFFER_TOO_SMALL:
                raise DbgError(st, "dbg_export_sorted")
        st = L.dbg_export_sorted(self.handle, None, None, 0, ctypes.byref(n), _stream(stream))
        if st not in (OK, ERR_BUFFER_TOO_SMALL):
            raise DbgError(st, "dbg_export_sorted")
        D = int(n.value)
        keys = np.empty((D, 2) if wide else D, dtype=np.uint64)
        counts = np.empty((D, 4), dtype=np.uint32)
        if D:
            _check(L.dbg_export_sorted(self.handle, keys.ctypes.data, counts.ctypes.data, D,
                                       ctypes.byref(n), _stream(stream)), "dbg_export_sorted")
        return keys, counts

    def normalize(self, divisor: float, stream=None) -> None:
        """Counters := floor(counter / divisor + 0.5) (the paper's normalization)."""
        _check(load().dbg_normalize(self.handle, float(divisor), _stream(stream)),
               "dbg_normalize")

    def contigs(self, stream=None) -> list[str]:
        """The graph's contigs (Alg. 5), ordered by (start vertex, label)."""
        L = load()
        n, b = ctypes.c_uint64(), ctypes.c_uint64()
        st = L.dbg_find_contigs(self.handle, None, 0, None, 0, ctypes.byref(n), ctypes.byref(b),
                                _stream(stream))
        if st not in (OK, ERR_BUFFER_TOO_SMALL):
            raise DbgError(st, "dbg_find_contigs")
        if n.value == 0:
            return []
        bases = np.empty(b.value, dtype=np.uint8)
        offs = np.empty(n.value + 1, dtype=np.uint64)
        _check(L.dbg_find_contigs(self.handle, bases.ctypes.data, bases.size, offs.ctypes.data,
                                  n.value, ctypes.byref(n), ctypes.byref(b), _stream(stream)),
               "dbg_find_contigs")
        raw = bases.tobytes().decode("ascii")
        return [raw[int(offs[i]):int(offs[i + 1])] for i in range(n.value)]

    def export_into(self, keys, counts, stream=None) -> int:
        """One dbg_export_sorted call into caller-owned CUDA tensors (keys
        int64 [>= D] or [>= D, 2], counts int32 [>= D, 4]); returns D.  Raises
        if they hold fewer than D rows."""
        n = ctypes.c_uint64()
        rows = min(int(keys.shape[0]), int(counts.shape[0]))
        _check(load().dbg_export_sorted(self.handle, keys.data_ptr(), counts.data_ptr(), rows,
                                        ctypes.byref(n), _stream(stream)), "dbg_export_sorted")
        return int(n.value)

    def export_with(self, keys, counts, scratch, stream=None) -> int:
        """dbg_export_sorted_with: into caller-owned CUDA tensors (keys int64
        [>= D], counts int32 [>= D, 4], scratch uint8 of at least
        ``export_scratch_bytes(k, D, n_slots)`` bytes); returns D."""
        n = ctypes.c_uint64()
        rows = min(int(keys.shape[0]), int(counts.shape[0]))
        _check(load().dbg_export_sorted_with(self.handle, keys.data_ptr(), counts.data_ptr(), rows,
                                             ctypes.byref(n), scratch.data_ptr(),
                                             int(scratch.numel()), _stream(stream)),
               "dbg_export_sorted_with")
        return int(n.value)

    def export_device(self, stream=None):
        """Sorted vertices as CUDA tensors (int64 keys [D], or [D, 2] for k > 32;
        int32 counters [D, 4])."""
        import torch
        L = load()
        n = ctypes.c_uint64()
        st = L.dbg_export_sorted(self.handle, None, None, 0, ctypes.byref(n), _stream(stream))
        if st not in (OK, ERR_BUFFER_TOO_SMALL):
            raise DbgError(st, "dbg_export_sorted")
        D = int(n.value)
        keys = torch.empty((D, 2) if self.k > 32 else D, dtype=torch.int64, device="cuda")
        counts = torch.empty((D, 4), dtype=torch.int32, device="cuda")
        if D:
            _check(L.dbg_export_sorted(self.handle, keys.data_ptr(), counts.data_ptr(), D,
                                       ctypes.byref(n), _stream(stream)), "dbg_export_sorted")
        return keys, counts


def _batch_items(items):
    arr = (BatchItem * max(1, len(items)))()
    for i, (g, pk, of) in enumerate(items):
        arr[i] = BatchItem(g.handle, _dptr(pk) or None, _dptr(of) or None, int(of.numel()) - 1)
    return arr


def insert_batch(items, stream=None) -> None:
    """``items``: list of ``(graph, packed, offsets)`` with device buffers."""
    _check(load().dbg_insert_batch(_batch_items(items), len(items), _stream(stream)),
           "dbg_insert_batch")


def build_batch(items, stream=None) -> None:
    """dbg_build_batch: every graph emptied, then built from its reads."""
    _check(load().dbg_build_batch(_batch_items(items), len(items), _stream(stream)),
           "dbg_build_batch")


def export_scratch_bytes(k: int, n_vertices: int, n_slots: int) -> int:
    """Bytes of caller scratch dbg_export_sorted_with needs."""
    return int(load().dbg_export_scratch_bytes(int(k), int(n_vertices), int(n_slots)))


def scratch_bytes() -> int:
    """Device bytes the library holds between calls on the current device."""
    return int(load().dbg_scratch_bytes())


def release_scratch() -> None:
    """Give back the batched inserts' buffers and the export's cached memory."""
    _check(load().dbg_release_scratch(), "dbg_release_scratch")


def probe_random_sectors(buf, n_slots: int, n_ops: int, seed: int, mode: int, stream=None) -> None:
    _check(load().dbg_probe_random_sectors(_dptr(buf), int(n_slots), int(n_ops), int(seed),
                                           int(mode), _stream(stream)), "dbg_probe_random_sectors")


def probe_window(buf, n_slots: int, n_ops: int, window_slots: int, seed: int, flags: int = 0,
                 stream=None) -> None:
    _check(load().dbg_probe_window(_dptr(buf), int(n_slots), int(n_ops), int(window_slots),
                                   int(seed), int(flags), _stream(stream)), "dbg_probe_window")


def sketch(k: int, packed, offsets, registers=None, stream=None):
    """HyperLogLog registers of a read set's vertex keys (device tensors in,
    a CUDA int32 tensor of SKETCH_REGISTERS + 1 words out; the last word is
    the status)."""
    import torch
    if registers is None:
        registers = torch.empty(SKETCH_REGISTERS + 1, dtype=torch.int32, device=packed.device)
    _check(load().dbg_sketch_reads(int(k), _dptr(packed) or None, _dptr(offsets) or None,
                                   int(offsets.numel()) - 1, _dptr(registers), _stream(stream)),
           "dbg_sketch_reads")
    return registers


def sketch_batch(items, stream=None) -> None:
    """``items``: list of ``(k, packed, offsets, registers)`` device tensors;
    each ``registers`` holds SKETCH_REGISTERS + 1 int32 words."""
    arr = (SketchItem * max(1, len(items)))()
    for i, (k, pk, of, rg) in enumerate(items):
        arr[i] = SketchItem(int(k), _dptr(pk) or None, _dptr(of) or None, int(of.numel()) - 1,
                            _dptr(rg))
    _check(load().dbg_sketch_batch(arr, len(items), _stream(stream)), "dbg_sketch_batch")


def sketch_estimate(registers) -> float:
    """Distinct-key estimate from registers (host numpy array or CPU tensor)."""
    r = np.ascontiguousarray(_host_view(registers, np.uint32)[:SKETCH_REGISTERS])
    return float(load().dbg_sketch_estimate(r.ctypes.data))


def table_bytes(capacity: int) -> int:
    """Device bytes a table of ``capacity`` slots takes on caller memory."""
    return int(load().dbg_table_bytes(int(capacity)))


def mlp_work_floats(batch: int) -> int:
    """Floats of scratch the network needs for a batch."""
    return int(load().dbg_mlp_work_floats(int(batch)))


def mlp_features(registers, x, batch: int, stride: int | None = None, stream=None):
    """x[b] = registers[b * stride : b * stride + MLP_INPUTS] / 64 (device tensors)."""
    stride = SKETCH_REGISTERS + 1 if stride is None else int(stride)
    _check(load().dbg_mlp_features(_dptr(registers), stride, int(batch), _dptr(x),
                                   _stream(stream)), "dbg_mlp_features")
    return x


def mlp_init(params, seed: int, stream=None):
    """He-uniform weights, zero biases, into a device float32 tensor of MLP_PARAMS."""
    _check(load().dbg_mlp_init(_dptr(params), int(seed), _stream(stream)), "dbg_mlp_init")
    return params


def mlp_forward(params, x, y, work, batch: int | None = None, stream=None):
    """y[b] = network(x[b]) (device float32 tensors; x is batch x MLP_INPUTS)."""
    batch = int(y.numel()) if batch is None else int(batch)
    _check(load().dbg_mlp_forward(_dptr(params), _dptr(x), batch, _dptr(y), _dptr(work),
                                  _stream(stream)), "dbg_mlp_forward")
    return y


def mlp_train_step(params, grads, adam_m, adam_v, step: int, lr: float, x, target, work,
                   loss=None, batch: int | None = None, stream=None):
    """One Adam step on the mean of (y - target)^2 / 2; ``loss`` (a device
    float32 tensor of one element, or None) receives the loss before the step."""
    batch = int(target.numel()) if batch is None else int(batch)
    _check(load().dbg_mlp_train_step(_dptr(params), _dptr(grads), _dptr(adam_m), _dptr(adam_v),
                                     int(step), float(lr), _dptr(x), _dptr(target), batch,
                                     _dptr(work), _dptr(loss) if loss is not None else None,
                                     _stream(stream)), "dbg_mlp_train_step")


def pack_ascii(seq: str, phase: int = 0) -> np.ndarray:
    """Pack ACGT text with the library's host helper (raises on other symbols)."""
    b = seq.encode("ascii")
    out = np.zeros((len(b) + phase + 3) // 4, dtype=np.uint8)
    bad = ctypes.c_uint64()
    st = load().dbg_pack_ascii(b, len(b), out.ctypes.data if out.size else None, phase,
                               ctypes.byref(bad))
    if st != OK:
        raise DbgError(st, f"dbg_pack_ascii (symbol at {bad.value})")
    return out
