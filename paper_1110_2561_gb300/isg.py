"""Python binding of libisg: the C entry points of include/isg.h under the same names.

Argument marshalling only -- every step of the computation runs in libisg's CUDA kernels.
Device buffers are torch CUDA tensors (passed as raw pointers) and streams are torch streams
(passed as cudaStream_t); PyTorch supplies memory and streams, nothing else. If libisg.so has
not been built, every call raises RuntimeError: there is no fallback path.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

ISG_FP64, ISG_FP32 = 0, 1
STATUS = {0: "ISG_OK", 1: "ISG_ERR_INVALID", 2: "ISG_ERR_TOO_LARGE", 3: "ISG_ERR_NOMEM", 4: "ISG_ERR_CUDA",
          5: "ISG_ERR_TIMEOUT", 6: "ISG_ERR_BUSY", 7: "ISG_ERR_NOT_READY", 8: "ISG_ERR_INTERNAL"}


class IsgError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class isg_options(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int32) for n in (
        "struct_size", "max_spins", "inner_bits", "low_bits", "block_threads", "copies", "ctas_per_sm",
        "flush_tasks", "shard_bits", "bin_stride")] + [
        ("shard_lo", ctypes.c_int64), ("shard_hi", ctypes.c_int64),
        ("accumulate", ctypes.c_int32), ("warp_aggregate", ctypes.c_int32),
        ("stride_residue", ctypes.c_int32), ("autotune", ctypes.c_int32),
        ("symmetry", ctypes.c_int32), ("split", ctypes.c_int32), ("lane_model", ctypes.c_int32)]


_lock = threading.Lock()
_lib = None
vp, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
_SIGS = {
    "isg_options_init": (None, [vp]),
    "isg_graph_create": (i32, [i32, i64, vp, vp, vp, ctypes.POINTER(vp)]),
    "isg_graph_destroy": (None, [vp]),
    "isg_graph_bins": (i32, [vp, vp, vp, vp, vp, vp]),
    "isg_graph_size": (i32, [vp, vp, vp]),
    "isg_enumerate": (i32, [vp, vp, vp, i32, vp]),
    "isg_enumerate_split": (i32, [vp, vp, vp, i32, ctypes.c_uint64]),
    "isg_enumerate_split_batch": (i32, [i32, vp, vp, vp, i32]),
    "isg_split_plan": (i32, [vp, ctypes.c_uint64, ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(i32),
                             ctypes.POINTER(i32), ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]),
    "isg_debug_emulate_split": (i32, [vp, ctypes.c_uint64, vp]),
    "isg_thermo": (i32, [vp, i32, vp, i32, vp, i32, vp, i32, vp, i32, vp, vp, vp, vp, vp]),
    "isg_magnetisation": (i32, [vp, i32, vp, i32, vp, i32, vp, i32, vp, i32, vp, vp, vp, vp]),
    "isg_last_error": (ctypes.c_char_p, []),
    "isg_version": (ctypes.c_char_p, []),
    "isg_debug_plan": (i32, [vp, vp, i32, vp]),
    "isg_debug_emulate": (i32, [vp, vp, vp]),
    "isg_debug_lane_banks": (i32, [vp, vp, i32, ctypes.c_uint64, vp, vp]),
    "isg_debug_lane_layout": (i32, [vp, vp, vp]),
    "isg_debug_emulate_planted": (i32, [vp, vp, i32, i32, vp, ctypes.POINTER(ctypes.c_uint32)]),
    "isg_debug_server_inject": (i32, [vp, i32]),
    "isg_debug_server_lane_counts": (i32, [vp, ctypes.POINTER(i64), ctypes.POINTER(i64)]),
    "isg_device_status": (i32, [vp, i32]),
    "isg_rank_shards": (i32, [i32, i32, i32, i32, ctypes.POINTER(i32), ctypes.POINTER(i64), ctypes.POINTER(i64)]),
    "isg_enumerate_rank": (i32, [vp, vp, vp, i32, i32, i32, vp]),
    "isg_debug_emulate_rank": (i32, [vp, i32, i32, vp, vp]),
    "isg_probe_peaks": (i32, [vp, vp, vp, vp, vp]),
    "isg_enumerate_noalloc": (i32, [vp, vp, vp, vp]),
    "isg_autotune": (i32, [vp, vp, vp, vp]),
    "isg_specific_heat_peak": (i32, [vp, i32, vp, ctypes.c_double, ctypes.c_double, ctypes.c_double, i32, vp, vp, vp]),
    "isg_enumerate_batch": (i32, [i32, vp, vp, vp, i32, vp]),
    "isg_batch_create": (i32, [i32, vp, vp, ctypes.POINTER(vp)]),
    "isg_batch_run": (i32, [vp, vp]),
    "isg_batch_table": (i32, [vp, i32, ctypes.POINTER(vp)]),
    "isg_batch_status": (i32, [vp, vp]),
    "isg_batch_destroy": (None, [vp]),
    "isg_server_options_init": (None, [vp]),
    "isg_server_create": (i32, [vp, ctypes.POINTER(vp)]),
    "isg_server_submit": (i32, [vp, vp, ctypes.POINTER(i64)]),
    "isg_server_poll": (i32, [vp, i64, ctypes.POINTER(i32)]),
    "isg_server_wait": (i32, [vp, i64, i64]),
    "isg_server_result": (i32, [vp, i64, vp, vp]),
    "isg_server_cancel": (i32, [vp, i64]),
    "isg_server_stats": (i32, [vp, vp]),
    "isg_server_destroy": (None, [vp]),
}


def library_path() -> str:
    return _build.LIB


def lib():
    """The loaded libisg.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.LIB
            if not os.path.exists(path):
                raise RuntimeError(f"{path} is missing: build it with __graft_entry__.build() "
                                   "(python -m paper_1110_2561_gb300.build); there is no fallback")
            L = ctypes.CDLL(path)
            for name, (res, args) in _SIGS.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def _check(status: int):
    if status != 0:
        raise IsgError(status, lib().isg_last_error().decode())


def _options(**kw) -> isg_options:
    o = isg_options()
    lib().isg_options_init(ctypes.byref(o))
    for k, v in kw.items():
        if v is None:
            continue
        if not hasattr(o, k):
            raise TypeError(f"unknown option {k!r}")
        setattr(o, k, int(v))
    return o


def _stream_handle(stream) -> int:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


class Graph:
    """Owning handle of an isg_graph (freed with isg_graph_destroy)."""

    def __init__(self, ptr: int, n: int):
        self.ptr = ptr
        self.n = n
        self._shape = None

    def __del__(self):
        if getattr(self, "ptr", None) and _lib is not None:
            _lib.isg_graph_destroy(self.ptr)
            self.ptr = None

    @property
    def _as_parameter_(self):
        return ctypes.c_void_p(self.ptr)


def isg_graph_create(n_spins: int, edges) -> Graph:
    """Graph of n_spins spins from rows (i, j, J) (int arrays are copied)."""
    e = np.asarray(edges, dtype=np.int64).reshape(-1, 3)
    i = np.ascontiguousarray(e[:, 0], dtype=np.int32)
    j = np.ascontiguousarray(e[:, 1], dtype=np.int32)
    J = np.ascontiguousarray(e[:, 2], dtype=np.int32)
    out = ctypes.c_void_p()
    _check(lib().isg_graph_create(n_spins, len(i), i.ctypes.data, j.ctypes.data, J.ctypes.data, ctypes.byref(out)))
    return Graph(out.value, n_spins)


def isg_graph_destroy(graph: Graph):
    if graph.ptr:
        lib().isg_graph_destroy(graph.ptr)
        graph.ptr = None


def isg_graph_bins(graph: Graph):
    """(e_min, e_step, n_e, m_min, n_m)."""
    v = [ctypes.c_int32() for _ in range(5)]
    _check(lib().isg_graph_bins(graph, *[ctypes.byref(x) for x in v]))
    return tuple(x.value for x in v)


def isg_graph_size(graph: Graph):
    a, b = ctypes.c_int32(), ctypes.c_int32()
    _check(lib().isg_graph_size(graph, ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


def table_shape(graph: Graph):
    if graph._shape is None:
        _, _, n_e, _, n_m = isg_graph_bins(graph)
        graph._shape = (n_e, n_m)
    return graph._shape


def isg_enumerate(graph: Graph, g_out=None, stream=None, **options):
    """Exact g(E, M) of the graph (Sec. 2-3 of arXiv:1110.2561).

    g_out: a torch int64 CUDA tensor of table_shape(graph) (filled asynchronously on `stream`),
    a numpy int64 array (host; the call synchronises), or None for a new numpy array.
    options: fields of isg_options (inner_bits, low_bits, block_threads, copies, ctas_per_sm,
    flush_tasks, shard_bits, shard_lo, shard_hi, accumulate, max_spins)."""
    shape = table_shape(graph)
    o = _options(**options)
    if g_out is None:
        g_out = np.zeros(shape, dtype=np.int64)
    if isinstance(g_out, np.ndarray):
        if g_out.dtype != np.int64 or not g_out.flags.c_contiguous or g_out.shape != shape:
            raise ValueError(f"g_out must be a C-contiguous int64 array of shape {shape}")
        _check(lib().isg_enumerate(graph, _stream_handle(stream) if stream is not None else None,
                                   g_out.ctypes.data, 0, ctypes.byref(o)))
        return g_out
    _check_tensor(g_out, shape, "int64")
    _check(lib().isg_enumerate(graph, _stream_handle(stream), g_out.data_ptr(), 1, ctypes.byref(o)))
    return g_out


def isg_rank_shards(n_spins: int, rank: int, world_size: int, symmetry: bool = False):
    """(shard_bits, shard_lo, shard_hi): the shards of the configuration space that rank `rank` of
    `world_size` enumerates (see isg_enumerate_rank)."""
    b, lo, hi = ctypes.c_int32(), ctypes.c_int64(), ctypes.c_int64()
    _check(lib().isg_rank_shards(n_spins, rank, world_size, 1 if symmetry else 0, ctypes.byref(b), ctypes.byref(lo),
                                 ctypes.byref(hi)))
    return b.value, lo.value, hi.value


def isg_enumerate_rank(graph: Graph, rank: int, world_size: int, g_out=None, stream=None, **options):
    """Rank `rank`'s share of g (the tables of all ranks sum to the exact table). g_out as for
    isg_enumerate; options as there (symmetry allowed, shard fields not)."""
    shape = table_shape(graph)
    o = _options(**options)
    if g_out is None:
        g_out = np.zeros(shape, dtype=np.int64)
    if isinstance(g_out, np.ndarray):
        if g_out.dtype != np.int64 or not g_out.flags.c_contiguous or g_out.shape != shape:
            raise ValueError(f"g_out must be a C-contiguous int64 array of shape {shape}")
        _check(lib().isg_enumerate_rank(graph, _stream_handle(stream) if stream is not None else None,
                                        g_out.ctypes.data, 0, rank, world_size, ctypes.byref(o)))
        return g_out
    _check_tensor(g_out, shape, "int64")
    _check(lib().isg_enumerate_rank(graph, _stream_handle(stream), g_out.data_ptr(), 1, rank, world_size,
                                    ctypes.byref(o)))
    return g_out


def enumerate_distributed(graph: Graph, g_out, group=None, stream=None, **options):
    """The exact table of one graph enumerated by every rank of a torch.distributed process group:
    isg_enumerate_rank on this rank's share, then one all-reduce (sum) of the int64 table over the
    group. g_out: a torch int64 tensor of table_shape(graph), a CUDA tensor (NCCL reduces it in
    place; a gloo group stages it through host memory) or a CPU tensor (gloo). Returns g_out."""
    import torch
    import torch.distributed as dist
    rank, world = dist.get_rank(group), dist.get_world_size(group)
    if g_out.is_cuda:
        st = stream if stream is not None else torch.cuda.current_stream(g_out.device)
        isg_enumerate_rank(graph, rank, world, g_out, st, **options)
        with torch.cuda.stream(st):             # the collective is ordered after the enumeration
            if dist.get_backend(group) == "nccl":
                dist.all_reduce(g_out, op=dist.ReduceOp.SUM, group=group)
            else:
                host = g_out.cpu()              # waits for the enumeration on st
                dist.all_reduce(host, op=dist.ReduceOp.SUM, group=group)
                g_out.copy_(host)
        return g_out
    if g_out.dtype != torch.int64 or not g_out.is_contiguous() or tuple(g_out.shape) != table_shape(graph):
        raise ValueError(f"g_out must be a contiguous int64 tensor of shape {table_shape(graph)}")
    isg_enumerate_rank(graph, rank, world, g_out.numpy(), **options)
    dist.all_reduce(g_out, op=dist.ReduceOp.SUM, group=group)
    return g_out


def isg_debug_emulate_rank(graph: Graph, rank: int, world_size: int, **options) -> np.ndarray:
    """isg_enumerate_rank's work run on the host by the kernels' walk (small N only)."""
    g = np.zeros(table_shape(graph), dtype=np.int64)
    o = _options(**options)
    _check(lib().isg_debug_emulate_rank(graph, rank, world_size, ctypes.byref(o), g.ctypes.data))
    return g


def isg_device_status(stream=None, clear: bool = True):
    """Raise IsgError (ISG_ERR_INTERNAL) if a kernel self-check of a device-output call on the
    current device failed since the last clear (synchronises `stream`); clear resets the word."""
    _check(lib().isg_device_status(_stream_handle(stream), 1 if clear else 0))


def isg_autotune(graph: Graph, stream=None, **options) -> dict:
    """Timed choice of the planning fields for this graph (cached in the library); returns them."""
    o = _options(**options)
    t = isg_options()
    _check(lib().isg_autotune(graph, _stream_handle(stream), ctypes.byref(o), ctypes.byref(t)))
    return {name: getattr(t, name) for name, _ in t._fields_ if name != "struct_size"}


def isg_enumerate_noalloc(graph: Graph, g_out, stream=None, **options):
    """isg_enumerate into a torch int64 CUDA tensor without any device allocation by the library.

    For callers that cannot allocate device memory (memory owned by another allocator, a fixed
    budget, or a loop that must not enter an allocator): the library's scratch is a 16 KiB array
    of device memory it holds for the life of the process. Calls share that array, so calls whose
    work overlaps on the GPU race: issue them on one stream. The first call on a device sets up
    that device's address of the array; make it before any stream capture."""
    _check_tensor(g_out, table_shape(graph), "int64")
    o = _options(**options)
    _check(lib().isg_enumerate_noalloc(graph, _stream_handle(stream), g_out.data_ptr(), ctypes.byref(o)))
    return g_out


def isg_enumerate_split(graph: Graph, g_out=None, stream=None, boundary: int = 0):
    """The exact g(E, M) by split-and-convolve (a variant of the full enumeration that visits
    2^(|S|-1) * sum 2^|C| configurations; see isg_split_plan). g_out as for isg_enumerate (the table is
    overwritten). boundary: a mask of boundary spins, or 0 for the library's choice."""
    shape = table_shape(graph)
    if g_out is None:
        g_out = np.zeros(shape, dtype=np.int64)
    if isinstance(g_out, np.ndarray):
        if g_out.dtype != np.int64 or not g_out.flags.c_contiguous or g_out.shape != shape:
            raise ValueError(f"g_out must be a C-contiguous int64 array of shape {shape}")
        _check(lib().isg_enumerate_split(graph, _stream_handle(stream) if stream is not None else None,
                                         g_out.ctypes.data, 0, boundary))
        return g_out
    _check_tensor(g_out, shape, "int64")
    _check(lib().isg_enumerate_split(graph, _stream_handle(stream), g_out.data_ptr(), 1, boundary))
    return g_out


def isg_enumerate_split_batch(graphs, g_out=None, stream=None):
    """Exact tables of many graphs in one call, each by split-and-convolve where its plan models
    less work than the full enumeration, else by the batched full enumeration. g_out: None (new numpy tables, synchronous), a list of numpy int64 tables, or a list
    of torch int64 CUDA tensors (enqueued on `stream`)."""
    shapes = [table_shape(g) for g in graphs]
    if g_out is None:
        g_out = [np.zeros(s, dtype=np.int64) for s in shapes]
    on_device = len(g_out) > 0 and not isinstance(g_out[0], np.ndarray)
    ptrs = []
    for t, s in zip(g_out, shapes):
        if on_device:
            _check_tensor(t, s, "int64")
            ptrs.append(t.data_ptr())
        else:
            if t.dtype != np.int64 or not t.flags.c_contiguous or t.shape != s:
                raise ValueError(f"host tables must be C-contiguous int64 arrays of shape {s}")
            ptrs.append(t.ctypes.data)
    arr = (ctypes.c_void_p * len(ptrs))(*ptrs)
    sh = _stream_handle(stream) if (stream is not None or on_device) else None
    _check(lib().isg_enumerate_split_batch(len(graphs), _graph_array(graphs), sh, arr, 1 if on_device else 0))
    return g_out


def isg_split_plan(graph: Graph, boundary: int = 0) -> dict:
    """The boundary set and cost isg_enumerate_split would use (host only)."""
    chosen = ctypes.c_uint64()
    nc, big = ctypes.c_int32(), ctypes.c_int32()
    visits, ratio = ctypes.c_double(), ctypes.c_double()
    _check(lib().isg_split_plan(graph, boundary, ctypes.byref(chosen), ctypes.byref(nc), ctypes.byref(big),
                                ctypes.byref(visits), ctypes.byref(ratio)))
    return {"boundary": chosen.value, "boundary_spins": bin(chosen.value).count("1"), "components": nc.value,
            "largest_component": big.value, "visits": visits.value, "work_ratio": ratio.value}


def isg_debug_emulate_split(graph: Graph, boundary: int = 0) -> np.ndarray:
    """The split kernel's work run on the host with every index checked (small graphs only)."""
    g = np.zeros(table_shape(graph), dtype=np.int64)
    _check(lib().isg_debug_emulate_split(graph, boundary, g.ctypes.data))
    return g


def _graph_array(graphs):
    arr = (ctypes.c_void_p * len(graphs))(*[g.ptr for g in graphs])
    return arr


def isg_enumerate_batch(graphs, g_out=None, stream=None, **options):
    """Tables of many graphs from one persistent launch. g_out: None (new numpy arrays), a list of
    numpy int64 arrays, or a list of torch int64 CUDA tensors, one per graph in its table_shape."""
    shapes = [table_shape(g) for g in graphs]
    if g_out is None:
        g_out = [np.zeros(s, dtype=np.int64) for s in shapes]
    on_device = 0 if isinstance(g_out[0], np.ndarray) else 1
    ptrs = []
    for t, s in zip(g_out, shapes):
        if on_device:
            _check_tensor(t, s, "int64")
            ptrs.append(t.data_ptr())
        else:
            if t.dtype != np.int64 or not t.flags.c_contiguous or t.shape != s:
                raise ValueError(f"host tables must be C-contiguous int64 arrays of shape {s}")
            ptrs.append(t.ctypes.data)
    arr = (ctypes.c_void_p * len(ptrs))(*ptrs)
    o = _options(**options)
    sh = _stream_handle(stream) if (stream is not None or on_device) else None
    _check(lib().isg_enumerate_batch(len(graphs), _graph_array(graphs), sh, arr, on_device, ctypes.byref(o)))
    return g_out


class Batch:
    """Prepared batch (isg_batch_create): device-resident programs and tables, runs replayed from
    a captured CUDA graph."""

    def __init__(self, graphs, **options):
        o = _options(**options)
        out = ctypes.c_void_p()
        _check(lib().isg_batch_create(len(graphs), _graph_array(graphs), ctypes.byref(o), ctypes.byref(out)))
        self.ptr = out.value
        self.shapes = [table_shape(g) for g in graphs]

    def run(self, stream=None):
        _check(lib().isg_batch_run(self.ptr, _stream_handle(stream)))

    def status(self, stream=None):
        _check(lib().isg_batch_status(self.ptr, _stream_handle(stream)))

    def table_ptr(self, k: int) -> int:
        p = ctypes.c_void_p()
        _check(lib().isg_batch_table(self.ptr, k, ctypes.byref(p)))
        return p.value

    def table(self, k: int):
        """Graph k's table as a torch int64 CUDA tensor viewing the batch's memory (no copy)."""
        import torch
        n_e, n_m = self.shapes[k]
        return _tensor_view(self.table_ptr(k), n_e * n_m, torch.int64).view(n_e, n_m)

    def close(self):
        if getattr(self, "ptr", None):
            lib().isg_batch_destroy(self.ptr)
            self.ptr = None

    def __del__(self):
        if _lib is not None:
            self.close()


class isg_server_options(ctypes.Structure):
    _fields_ = [("struct_size", ctypes.c_int32), ("max_spins", ctypes.c_int32), ("max_inflight", ctypes.c_int32),
                ("max_queued", ctypes.c_int32), ("arena_bytes", ctypes.c_int64), ("step_ms", ctypes.c_double),
                ("block_threads", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32),
                ("split_work_ratio", ctypes.c_double), ("symmetry", ctypes.c_int32), ("lane_model", ctypes.c_int32)]


class Server:
    """isg_server_*: a continuously batching request server on the current device.

    options: fields of isg_server_options (max_spins, max_inflight, max_queued, arena_bytes,
    step_ms, block_threads, ctas_per_sm, split_work_ratio, symmetry, lane_model)."""

    def __init__(self, **options):
        o = isg_server_options()
        lib().isg_server_options_init(ctypes.byref(o))
        for k, v in options.items():
            if not hasattr(o, k):
                raise TypeError(f"unknown server option {k!r}")
            setattr(o, k, v)
        out = ctypes.c_void_p()
        _check(lib().isg_server_create(ctypes.byref(o), ctypes.byref(out)))
        self.ptr = out.value
        self.shapes = {}

    def submit(self, graph: Graph) -> int:
        t = ctypes.c_int64()
        _check(lib().isg_server_submit(self.ptr, graph, ctypes.byref(t)))
        self.shapes[t.value] = table_shape(graph)
        return t.value

    def poll(self, ticket: int) -> bool:
        d = ctypes.c_int32()
        _check(lib().isg_server_poll(self.ptr, ticket, ctypes.byref(d)))
        return bool(d.value)

    def wait(self, ticket: int, timeout_ms: int = -1):
        _check(lib().isg_server_wait(self.ptr, ticket, timeout_ms))

    def result(self, ticket: int):
        """(table, times) with times = (queued s, service s, latency s, submitted at s)."""
        g = np.zeros(self.shapes[ticket], dtype=np.int64)
        times = (ctypes.c_double * 4)()
        _check(lib().isg_server_result(self.ptr, ticket, g.ctypes.data, times))
        del self.shapes[ticket]
        return g, tuple(times)

    def cancel(self, ticket: int):
        _check(lib().isg_server_cancel(self.ptr, ticket))
        self.shapes.pop(ticket, None)

    def inject_failure(self, where: int):
        """isg_debug_server_inject: make the next engine step fail on the host (1: before its first
        enqueue, 2: after its launch; 0: cancel)."""
        _check(lib().isg_debug_server_inject(self.ptr, where))

    def lane_counts(self) -> dict:
        """isg_debug_server_lane_counts: requests given lane tables, and enumeration launches for them."""
        req, lau = i64(), i64()
        _check(lib().isg_debug_server_lane_counts(self.ptr, ctypes.byref(req), ctypes.byref(lau)))
        return {"requests": req.value, "launches": lau.value}

    def stats(self) -> dict:
        v = (ctypes.c_double * 8)()
        _check(lib().isg_server_stats(self.ptr, v))
        keys = ("steps", "configs", "device_ms", "queued", "admitted", "rate_est", "uptime_s", "tickets")
        return dict(zip(keys, list(v)))

    def close(self):
        if getattr(self, "ptr", None):
            lib().isg_server_destroy(self.ptr)
            self.ptr = None

    def __del__(self):
        if _lib is not None:
            self.close()


def _tensor_view(ptr: int, numel: int, dtype):
    """A torch CUDA tensor aliasing device memory owned by the library (via __cuda_array_interface__)."""
    import torch

    class _Holder:
        __cuda_array_interface__ = {"shape": (numel,), "typestr": "<i8", "data": (ptr, False), "version": 3,
                                    "strides": None}
    return torch.as_tensor(_Holder(), device="cuda")


_TORCH = {}


def _check_tensor(t, shape, dtype: str):
    if not _TORCH:
        import torch
        _TORCH.update(torch=torch, int64=torch.int64, float64=torch.float64)
    if not (isinstance(t, _TORCH["torch"].Tensor) and t.is_cuda and t.dtype is _TORCH[dtype] and t.is_contiguous()
            and t.shape == shape):
        raise ValueError(f"expected a contiguous {dtype} CUDA tensor of shape {tuple(shape)}")


def _f64(x) -> np.ndarray:
    if isinstance(x, np.ndarray) and x.dtype == np.float64 and x.ndim == 1 and x.flags.c_contiguous:
        return x
    return np.ascontiguousarray(np.atleast_1d(x), dtype=np.float64)


def _grid_call(fn, n_out: int, g, graph: Graph, T, h, precision: int, stream, out):
    T, h = _f64(T), _f64(h)
    shape = table_shape(graph)
    if isinstance(g, np.ndarray):
        g = np.ascontiguousarray(g, dtype=np.int64)
        if g.shape != shape:
            raise ValueError(f"g must have shape {shape}")
        g_ptr, g_dev = g.ctypes.data, 0
    else:
        _check_tensor(g, shape, "int64")
        g_ptr, g_dev = g.data_ptr(), 1
    s = _stream_handle(stream) if (stream is not None or g_dev or out is not None) else None
    if out is None:
        res = [np.zeros((len(T), len(h)), dtype=np.float64) for _ in range(n_out)]
        _check(fn(g_ptr, g_dev, graph, len(T), T.ctypes.data, len(h), h.ctypes.data, precision, s, 0,
                  *[r.ctypes.data for r in res]))
        return tuple(res)
    if len(out) != n_out:
        raise ValueError(f"out must hold {n_out} entries")
    ptrs = []
    oshape = (len(T), len(h))
    for t in out:
        if t is None:
            ptrs.append(None)
        else:
            _check_tensor(t, oshape, "float64")
            ptrs.append(t.data_ptr())
    _check(fn(g_ptr, g_dev, graph, len(T), T.ctypes.data, len(h), h.ctypes.data, precision, s, 1, *ptrs))
    return out


def isg_thermo(g, graph: Graph, T, h, precision: int = ISG_FP64, stream=None, out=None):
    """ln Z, <H>, <M>, C, chi on the grid T x h (Eq. 2 over g).

    g: torch int64 CUDA tensor or numpy int64 array of table_shape(graph). out: None (numpy
    results, the call synchronises) or a tuple of 5 float64 CUDA tensors of shape (len(T), len(h))
    (filled asynchronously; None entries are skipped)."""
    return _grid_call(lib().isg_thermo, 5, g, graph, T, h, precision, stream, out)


def isg_magnetisation(g, graph: Graph, T, h, precision: int = ISG_FP64, stream=None, out=None):
    """<|M|>, <M^2>, <M^4> and Binder's cumulant 1 - <M^4>/(3<M^2>^2) on the grid T x h, with the
    weights of Eq. 2 over g. g and out as for isg_thermo (out: a tuple of 4)."""
    return _grid_call(lib().isg_magnetisation, 4, g, graph, T, h, precision, stream, out)


class PreparedCall:
    """A C entry point with its arguments validated and marshalled once; calling it again costs
    only the C call (for latency-bound loops over small problems). The caller keeps the buffers
    alive and unchanged in shape while the prepared call is in use."""

    def __init__(self, fn, args, keep):
        self._fn, self._args, self._keep = fn, args, keep

    def __call__(self):
        _check(self._fn(*self._args))


def prepare_enumerate(graph: Graph, g_out, stream=None, **options) -> PreparedCall:
    """isg_enumerate into a torch int64 CUDA tensor, prepared once."""
    _check_tensor(g_out, table_shape(graph), "int64")
    o = _options(**options)
    args = (graph.ptr, _stream_handle(stream), g_out.data_ptr(), 1, ctypes.byref(o))
    return PreparedCall(lib().isg_enumerate, args, (graph, g_out, o))


def prepare_thermo(g, graph: Graph, T, h, out, precision: int = ISG_FP64, stream=None) -> PreparedCall:
    """isg_thermo from a device table into five float64 CUDA tensors, prepared once."""
    T, h = _f64(T), _f64(h)
    _check_tensor(g, table_shape(graph), "int64")
    ptrs = []
    for t in out:
        if t is None:
            ptrs.append(None)
        else:
            _check_tensor(t, (len(T), len(h)), "float64")
            ptrs.append(t.data_ptr())
    args = (g.data_ptr(), 1, graph.ptr, len(T), T.ctypes.data, len(h), h.ctypes.data, precision,
            _stream_handle(stream), 1, *ptrs)
    return PreparedCall(lib().isg_thermo, args, (graph, g, T, h, out))


def isg_specific_heat_peak(g, graph: Graph, h: float, T_lo: float, T_hi: float, precision: int = ISG_FP64,
                           stream=None):
    """(T, C) at the maximum of the specific heat C(T) at field h on [T_lo, T_hi]."""
    if isinstance(g, np.ndarray):
        g = np.ascontiguousarray(g, dtype=np.int64)
        if g.shape != table_shape(graph):
            raise ValueError(f"g must have shape {table_shape(graph)}")
        ptr, dev = g.ctypes.data, 0
    else:
        _check_tensor(g, table_shape(graph), "int64")
        ptr, dev = g.data_ptr(), 1
    t, c = ctypes.c_double(), ctypes.c_double()
    sh = _stream_handle(stream) if (stream is not None or dev) else None
    _check(lib().isg_specific_heat_peak(ptr, dev, graph, h, T_lo, T_hi, precision, sh, ctypes.byref(t), ctypes.byref(c)))
    return t.value, c.value


def isg_debug_plan(graph: Graph, sms: int = 0, **options) -> dict:
    out = np.zeros(19, dtype=np.int64)
    o = _options(**options)
    _check(lib().isg_debug_plan(graph, ctypes.byref(o), sms, out.ctypes.data))
    keys = ("small", "q", "b", "tasks", "threads", "copies", "ctas_per_sm", "flush_rounds", "grid", "smem_bytes",
            "G", "n_e_compact", "blob_bytes", "stride", "lane_model", "lane_cost", "lane_cost_index_order",
            "lane_mask", "lane_tables")
    d = dict(zip(keys, (int(x) for x in out)))
    d["lane_cost"] /= 1e6
    d["lane_cost_index_order"] /= 1e6
    return d


def isg_debug_lane_banks(graph: Graph, samples: int = 4096, seed: int = 1, **options):
    """(mean, max) shared-memory wavefronts of sampled warp reductions of the plan (host only)."""
    mean = ctypes.c_double()
    worst = ctypes.c_int32()
    o = _options(**options)
    _check(lib().isg_debug_lane_banks(graph, ctypes.byref(o), samples, seed, ctypes.byref(mean), ctypes.byref(worst)))
    return mean.value, worst.value


def isg_debug_lane_layout(graph: Graph, **options) -> dict:
    """The histogram layout of one copy under the plan (host only): row stride, words per copy,
    sub-tables with their first words and column ranges, each lane's first word and sub-table."""
    out = np.zeros(99, dtype=np.int32)
    o = _options(**options)
    _check(lib().isg_debug_lane_layout(graph, ctypes.byref(o), out.ctypes.data))
    n = int(out[2])
    return {"stride": int(out[0]), "copy_words": int(out[1]), "n_sub": n, "sub_off": out[3:3 + n].copy(),
            "m_lo": out[13:13 + n].copy(), "m_hi": out[23:23 + n].copy(), "lane_word": out[33:65].copy(),
            "lane_sub": out[65:97].copy(), "packed": bool(out[97])}


def isg_debug_emulate(graph: Graph, **options) -> np.ndarray:
    """The enumeration kernels' per-thread walk run on the host (small N only)."""
    g = np.zeros(table_shape(graph), dtype=np.int64)
    o = _options(**options)
    _check(lib().isg_debug_emulate(graph, ctypes.byref(o), g.ctypes.data))
    return g


def isg_debug_emulate_planted(graph: Graph, site: int, delta: int, **options):
    """The host emulation with `delta` added to the field constant of internal site `site` (a
    planted program mistake). Returns (status, word, message, table): the status the library
    reports for the walk's self-check word, the word, isg_last_error's message and the table."""
    g = np.zeros(table_shape(graph), dtype=np.int64)
    o = _options(**options)
    w = ctypes.c_uint32()
    st = lib().isg_debug_emulate_planted(graph, ctypes.byref(o), site, delta, g.ctypes.data, ctypes.byref(w))
    return st, w.value, (isg_last_error() if st else ""), g


def isg_probe_peaks(stream=None) -> dict:
    """Measured lane-op rates (per second, whole GPU) of red.shared (conflict-free, scattered) and ALU."""
    v = [ctypes.c_double() for _ in range(4)]
    _check(lib().isg_probe_peaks(_stream_handle(stream), *[ctypes.byref(x) for x in v]))
    return {"red_conflict_free": v[0].value, "red_scattered": v[1].value, "alu": v[2].value,
            "match_aggregated": v[3].value}


def isg_last_error() -> str:
    return lib().isg_last_error().decode()


def isg_version() -> str:
    return lib().isg_version().decode()
