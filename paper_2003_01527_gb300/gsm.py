"""Python binding of libgsm (include/gsm.h): argument marshalling only.

Every function named ``gsm_*`` here is the C entry point of the same name;
the ``Matcher`` class is a convenience wrapper over them.  All matching work
runs in the library's CUDA kernels; this module never computes a result
itself, and importing it fails loudly when libgsm.so is missing.

PyTorch supplies device memory (the caching allocator, through the library's
alloc/free hooks) and streams (the context runs on the caller's current torch
stream unless told otherwise).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# GSM_DEBUG=1 in the environment: the build with device bounds checks
DEBUG = os.environ.get("GSM_DEBUG", "") not in ("", "0")
LIB_PATH = os.path.join(_HERE, "libgsm_debug.so" if DEBUG else "libgsm.so")

GSM_OK = 0
GSM_PENDING = 1
GSM_ERR_INVALID_ARG = -1
GSM_ERR_INVALID_GRAPH = -2
GSM_ERR_INVALID_QUERY = -3
GSM_ERR_NO_GRAPH = -4
GSM_ERR_OOM = -5
GSM_ERR_BUDGET = -6
GSM_ERR_OVERFLOW = -7
GSM_ERR_TRUNCATED = -8
GSM_ERR_TIMEOUT = -9
GSM_ERR_CUDA = -10
GSM_ERR_TOO_LARGE = -11
GSM_ERR_INTERNAL = -12

GSM_DEVICE_PTRS = 1
GSM_VALIDATE = 2
GSM_OUT_DEVICE = 1
GSM_OPT_TIME_KERNELS = 1
GSM_OPT_TWO_PASS = 2
GSM_OPT_COMPRESSED_FRONTIERS = 4
GSM_OPT_INJECT_LOOKBACK_STALL = 8
GSM_OPT_INJECT_SORT_STALL = 16
GSM_OPT_COUNT_PROBES = 32
GSM_OPT_INJECT_SCAN_STALL = 64

MAX_K = 16

# The public names of the C ABI (include/gsm.h); tests check the library
# exports each of them.
EXPORTED = [
    "gsm_default_options", "gsm_create", "gsm_destroy", "gsm_last_error", "gsm_status_string",
    "gsm_load_graph", "gsm_query_create", "gsm_query_destroy", "gsm_query_restrict",
    "gsm_count", "gsm_enumerate", "gsm_enumerate_many", "gsm_last_rows", "gsm_candidates",
    "gsm_plan_order", "gsm_query_symmetry", "gsm_kernel_stats", "gsm_last_run_stats",
    "gsm_candidates_static", "gsm_run_batch", "gsm_batch_get_stats", "gsm_batch_configure",
    "gsm_count_distinct", "gsm_server_start", "gsm_submit", "gsm_poll", "gsm_server_stop",
    "gsm_result_free",
]
GSM_BATCH_AUTOTUNE = 1
GSM_MODE_COUNT = 0
GSM_MODE_ENUMERATE = 1
GSM_STATIC_SCRATCH_BITMAP_BYTES = 8 << 20

_alloc_fn = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
_free_fn = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t,
                            ctypes.c_void_p)


class gsm_options(ctypes.Structure):
    _fields_ = [("mem_budget_bytes", ctypes.c_size_t), ("stream", ctypes.c_void_p),
                ("alloc", _alloc_fn), ("free", _free_fn), ("alloc_ctx", ctypes.c_void_p),
                ("block_size", ctypes.c_int32), ("chunk_rows", ctypes.c_int64),
                ("filter_rounds", ctypes.c_int32), ("flags", ctypes.c_int32),
                ("copy_slots", ctypes.c_int32), ("lookback_spin_limit", ctypes.c_int32),
                ("lookahead", ctypes.c_int32), ("hub_bitmap_bytes", ctypes.c_int64),
                ("host_workers", ctypes.c_int32)]


class gsm_kernel_stat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("launches", ctypes.c_uint64),
                ("total_ms", ctypes.c_double), ("algo_bytes", ctypes.c_double),
                ("items", ctypes.c_uint64), ("probe_bytes", ctypes.c_double)]


class gsm_batch_stats(ctypes.Structure):
    _fields_ = [("block_size", ctypes.c_int32), ("grid", ctypes.c_int32),
                ("tuned", ctypes.c_int32), ("overflowed", ctypes.c_int32),
                ("batches", ctypes.c_uint64), ("graph_launches", ctypes.c_uint64),
                ("graphs_built", ctypes.c_uint64), ("fallbacks", ctypes.c_uint64),
                ("kernels_per_graph", ctypes.c_uint64), ("last_ms", ctypes.c_double)]


class gsm_result(ctypes.Structure):
    _fields_ = [("count", ctypes.c_uint64), ("status", ctypes.c_int32),
                ("t_submit_ns", ctypes.c_int64), ("t_admit_ns", ctypes.c_int64),
                ("t_done_ns", ctypes.c_int64), ("k", ctypes.c_int32),
                ("on_device", ctypes.c_int32), ("rows", ctypes.POINTER(ctypes.c_int32))]


class gsm_run_stats(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int32), ("order", ctypes.c_int32 * 16),
                ("cand_size", ctypes.c_uint64 * 16), ("frontier", ctypes.c_uint64 * 16),
                ("candidates", ctypes.c_uint64 * 16), ("chunks", ctypes.c_uint64),
                ("peak_bytes", ctypes.c_uint64), ("kernel_launches", ctypes.c_uint64)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{os.path.basename(LIB_PATH)} not built ({LIB_PATH}); run "
                          "python -m paper_2003_01527_gb300.build" + (" --debug" if DEBUG else ""))
    lib = ctypes.CDLL(LIB_PATH)
    vp, i32, i64, u64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64
    sig = {
        "gsm_default_options": (None, [ctypes.POINTER(gsm_options)]),
        "gsm_create": (i32, [ctypes.POINTER(vp), i32, ctypes.POINTER(gsm_options)]),
        "gsm_destroy": (None, [vp]),
        "gsm_last_error": (ctypes.c_char_p, [vp]),
        "gsm_status_string": (ctypes.c_char_p, [i32]),
        "gsm_load_graph": (i32, [vp, i32, i64, vp, vp, vp, i32]),
        "gsm_query_create": (i32, [vp, i32, i32, vp, vp, ctypes.POINTER(vp)]),
        "gsm_query_destroy": (None, [vp]),
        "gsm_query_restrict": (i32, [vp, i32, i32, i32]),
        "gsm_count": (i32, [vp, vp, ctypes.POINTER(u64)]),
        "gsm_count_distinct": (i32, [vp, vp, ctypes.POINTER(u64), ctypes.POINTER(u64)]),
        "gsm_enumerate": (i32, [vp, vp, vp, u64, ctypes.POINTER(u64), i32]),
        "gsm_enumerate_many": (i32, [vp, i32, vp, vp, vp, vp, i32]),
        "gsm_last_rows": (i32, [vp, vp, u64, u64, i32]),
        "gsm_candidates": (i32, [vp, vp, vp, vp]),
        "gsm_plan_order": (i32, [i32, i32, vp, vp, vp, vp]),
        "gsm_query_symmetry": (i32, [i32, i32, vp, vp, vp, vp, i32, vp]),
        "gsm_candidates_static": (i32, [i32, i64, vp, vp, vp, vp, vp, vp, i32, vp]),
        "gsm_run_batch": (i32, [vp, vp, i32, vp, vp, i32]),
        "gsm_result_free": (None, [vp, ctypes.POINTER(gsm_result)]),
        "gsm_batch_get_stats": (i32, [vp, ctypes.POINTER(gsm_batch_stats)]),
        "gsm_batch_configure": (i32, [vp, u64, u64, u64, u64]),
        "gsm_server_start": (i32, [vp, i32, i32]),
        "gsm_submit": (i32, [vp, vp, i32, ctypes.POINTER(u64)]),
        "gsm_poll": (i32, [vp, u64, ctypes.POINTER(gsm_result)]),
        "gsm_server_stop": (i32, [vp]),
        "gsm_kernel_stats": (i32, [vp, ctypes.POINTER(gsm_kernel_stat), i32,
                                   ctypes.POINTER(i32), i32]),
        "gsm_last_run_stats": (i32, [vp, ctypes.POINTER(gsm_run_stats)]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


_lib = _load()


class GsmError(RuntimeError):
    def __init__(self, status: int, message: str = ""):
        self.status = status
        name = _lib.gsm_status_string(status).decode()
        super().__init__(f"{name}: {message}" if message else name)


def _ptr(a) -> int:
    """Raw address of a numpy array or torch tensor (contiguous)."""
    if a is None:
        return 0
    if hasattr(a, "data_ptr"):
        return int(a.data_ptr())
    return int(a.ctypes.data)


def _is_cuda(a) -> bool:
    return hasattr(a, "is_cuda") and bool(a.is_cuda)


# ----------------------------------------------------------- C-name wrappers

def gsm_status_string(status: int) -> str:
    return _lib.gsm_status_string(status).decode()


def gsm_default_options() -> gsm_options:
    opt = gsm_options()
    _lib.gsm_default_options(ctypes.byref(opt))
    return opt


def gsm_create(device: int, opt: gsm_options | None) -> int:
    h = ctypes.c_void_p()
    st = _lib.gsm_create(ctypes.byref(h), device, ctypes.byref(opt) if opt is not None else None)
    if st != GSM_OK:
        raise GsmError(st, "gsm_create")
    return h.value


def gsm_destroy(ctx: int) -> None:
    _lib.gsm_destroy(ctx)


def gsm_last_error(ctx: int) -> str:
    return _lib.gsm_last_error(ctx).decode()


def _check(ctx, st, ok=(GSM_OK,)):
    if st not in ok:
        raise GsmError(st, gsm_last_error(ctx) if ctx else "")
    return st


def gsm_load_graph(ctx: int, n: int, nnz: int, row_ptr, col, labels, flags: int) -> None:
    _check(ctx, _lib.gsm_load_graph(ctx, n, nnz, _ptr(row_ptr), _ptr(col), _ptr(labels), flags))


def gsm_query_create(ctx: int, k: int, m: int, edges, labels) -> int:
    h = ctypes.c_void_p()
    _check(ctx, _lib.gsm_query_create(ctx, k, m, _ptr(edges), _ptr(labels), ctypes.byref(h)))
    return h.value


def gsm_query_destroy(q: int) -> None:
    _lib.gsm_query_destroy(q)


def gsm_query_restrict(q: int, u: int, lo: int, hi: int) -> None:
    st = _lib.gsm_query_restrict(q, u, lo, hi)
    if st != GSM_OK:
        raise GsmError(st, "gsm_query_restrict")


def gsm_count(ctx: int, q: int) -> int:
    c = ctypes.c_uint64()
    _check(ctx, _lib.gsm_count(ctx, q, ctypes.byref(c)))
    return c.value


def gsm_count_distinct(ctx: int, q: int) -> tuple[int, int]:
    """(distinct subgraphs, |Aut(Q)|)."""
    c, a = ctypes.c_uint64(), ctypes.c_uint64()
    _check(ctx, _lib.gsm_count_distinct(ctx, q, ctypes.byref(c), ctypes.byref(a)))
    return c.value, a.value


def gsm_enumerate(ctx: int, q: int, out, cap_rows: int, flags: int) -> tuple[int, int]:
    """Returns (count, status); status is GSM_OK or GSM_ERR_TRUNCATED."""
    c = ctypes.c_uint64()
    st = _lib.gsm_enumerate(ctx, q, _ptr(out), cap_rows, ctypes.byref(c), flags)
    _check(ctx, st, (GSM_OK, GSM_ERR_TRUNCATED))
    return c.value, st


def gsm_enumerate_many(ctx: int, queries, outs, cap_rows, flags: int) -> tuple[np.ndarray, int]:
    """queries: gsm_query handles; outs: buffers (host, or device with
    GSM_OUT_DEVICE); cap_rows: capacities in rows.  Returns (uint64 counts,
    status); status is GSM_OK or GSM_ERR_TRUNCATED."""
    nq = len(queries)
    qa = (ctypes.c_void_p * max(nq, 1))(*queries)
    oa = (ctypes.c_void_p * max(nq, 1))(*[_ptr(o) for o in outs])
    caps = np.ascontiguousarray(np.asarray(cap_rows, dtype=np.uint64).reshape(nq))
    counts = np.zeros(max(nq, 1), dtype=np.uint64)
    st = _lib.gsm_enumerate_many(ctx, nq, qa, oa, _ptr(caps), _ptr(counts), flags)
    _check(ctx, st, (GSM_OK, GSM_ERR_TRUNCATED))
    return counts[:nq], st


def gsm_last_rows(ctx: int, out, first: int, nrows: int, flags: int) -> None:
    _check(ctx, _lib.gsm_last_rows(ctx, _ptr(out), first, nrows, flags))


def gsm_candidates(ctx: int, q: int, bitmaps, sizes) -> None:
    _check(ctx, _lib.gsm_candidates(ctx, q, _ptr(bitmaps), _ptr(sizes)))


def gsm_candidates_static(n: int, nnz: int, row_ptr, col, labels, q: int, bitmaps, sizes,
                          flags: int = 0, stream=None) -> None:
    """The allocation-free candidate filter (see include/gsm.h): the graph is
    device memory the caller owns; bitmaps/sizes are host arrays, or device
    tensors with flags=GSM_OUT_DEVICE."""
    st = _lib.gsm_candidates_static(n, nnz, _ptr(row_ptr), _ptr(col), _ptr(labels), q,
                                    _ptr(bitmaps), _ptr(sizes), flags,
                                    int(getattr(stream, "cuda_stream", stream or 0)))
    if st != GSM_OK:
        raise GsmError(st, "gsm_candidates_static")


def _copy_rows(r: gsm_result):
    """A copy of the rows of a result: a numpy array (host rows) or a CUDA
    tensor (device rows; the device copy may still be running)."""
    k, c = int(r.k), int(r.count)
    if not r.rows or c == 0:
        if r.on_device:
            import torch
            return torch.zeros((0, max(k, 1)), dtype=torch.int32, device="cuda")
        return np.zeros((0, max(k, 1)), dtype=np.int32)
    if r.on_device:
        import torch
        ptr = ctypes.cast(r.rows, ctypes.c_void_p).value
        return torch.as_tensor(_DevicePtr(ptr, c * k), device="cuda").clone().view(c, k)
    return np.ctypeslib.as_array(r.rows, shape=(c * k,)).reshape(c, k).copy()


def _take_rows(ctx: int, r: gsm_result):
    """Copies the rows of a result (see _copy_rows), then releases the
    library's buffer."""
    return _take_all(ctx, [r])[0]


def _take_all(ctx: int, results):
    """_copy_rows of every result, one device synchronisation, then every
    library buffer released.  Device results whose rows follow one another
    in memory (a listing batch puts them in one block, at most 12 bytes
    apart) are copied with one copy per such run and returned as views into
    it; the copy never reads past a result's rows by more than that gap."""
    out = [None] * len(results)
    dev = sorted((ctypes.cast(r.rows, ctypes.c_void_p).value, 4 * int(r.count) * int(r.k), j)
                 for j, r in enumerate(results) if r.on_device and r.rows and r.count)
    if len(dev) > 1:
        import torch
        runs, cur = [], [dev[0]]
        for e in dev[1:]:
            p0, n0, _ = cur[-1]
            if 0 <= e[0] - (p0 + n0) < 16:
                cur.append(e)
            else:
                runs.append(cur)
                cur = [e]
        runs.append(cur)
        for run in runs:
            if len(run) < 2:
                continue
            lo = run[0][0]
            hi = run[-1][0] + run[-1][1]
            span = torch.as_tensor(_DevicePtr(lo, (hi - lo) // 4), device="cuda").clone()
            for ptr, _, j in run:
                c, k = int(results[j].count), int(results[j].k)
                a = (ptr - lo) // 4
                out[j] = span[a:a + c * k].view(c, k)
    for j, r in enumerate(results):
        if out[j] is None:
            out[j] = _copy_rows(r)
    if dev:
        import torch
        torch.cuda.synchronize()  # the copies are done before the buffers go
    for r in results:
        _lib.gsm_result_free(ctx, ctypes.byref(r))
    return out


class _DevicePtr:
    """A CUDA array interface over a raw device pointer (int32 elements)."""

    def __init__(self, ptr: int, n: int):
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": "<i4",
                                         "data": (ptr, False), "version": 2}


def gsm_run_batch(ctx: int, queries, flags: int = 0, enumerate: bool = False):
    """queries: sequence of gsm_query handles.  Returns uint64 counts, or with
    enumerate=True (counts, rows): rows[j] = the sorted rows of query j, a
    numpy array (host) or, with flags & GSM_OUT_DEVICE, a CUDA tensor."""
    nq = len(queries)
    arr = (ctypes.c_void_p * max(nq, 1))(*queries)
    counts = np.zeros(max(nq, 1), dtype=np.uint64)
    res = (gsm_result * max(nq, 1))() if enumerate else None
    _check(ctx, _lib.gsm_run_batch(ctx, arr, nq, _ptr(counts), res, flags))
    if not enumerate:
        return counts[:nq]
    rows = _take_all(ctx, [res[j] for j in range(nq)])
    return counts[:nq], rows


def gsm_result_free(ctx: int, r: gsm_result) -> None:
    _lib.gsm_result_free(ctx, ctypes.byref(r))


def gsm_batch_get_stats(ctx: int) -> dict:
    s = gsm_batch_stats()
    _check(ctx, _lib.gsm_batch_get_stats(ctx, ctypes.byref(s)))
    return {name: getattr(s, name) for name, _ in gsm_batch_stats._fields_}


def gsm_batch_configure(ctx: int, cap_rows: int = 0, cap_elems: int = 0, cap_items: int = 0,
                        cap_result_elems: int = 0):
    _check(ctx, _lib.gsm_batch_configure(ctx, cap_rows, cap_elems, cap_items, cap_result_elems))


def gsm_server_start(ctx: int, lanes: int = 2, max_batch: int = 256) -> None:
    _check(ctx, _lib.gsm_server_start(ctx, lanes, max_batch))


def gsm_submit(ctx: int, q: int, mode: int = GSM_MODE_COUNT) -> int:
    t = ctypes.c_uint64()
    _check(ctx, _lib.gsm_submit(ctx, q, mode, ctypes.byref(t)))
    return t.value


def gsm_poll(ctx: int, ticket: int):
    """None while pending, else a dict with count, status and timestamps (ns),
    and in enumerate mode "rows" (numpy int32 [count, k], sorted; the
    library's buffer is released)."""
    r = gsm_result()
    st = _lib.gsm_poll(ctx, ticket, ctypes.byref(r))
    if st == GSM_PENDING:
        return None
    _check(ctx, st)
    out = {"count": r.count, "status": r.status, "t_submit_ns": r.t_submit_ns,
           "t_admit_ns": r.t_admit_ns, "t_done_ns": r.t_done_ns}
    if r.rows:
        out["rows"] = _take_rows(ctx, r)
    return out


def gsm_server_stop(ctx: int) -> None:
    _check(ctx, _lib.gsm_server_stop(ctx))


def gsm_query_symmetry(k: int, edges, labels=None) -> tuple[int, list[tuple[int, int]]]:
    """(|Aut(Q)|, ordering constraints [(u, v): f(u) < f(v)]) of a query."""
    e = np.ascontiguousarray(np.asarray(edges, dtype=np.int32).reshape(-1))
    lab = None if labels is None else np.ascontiguousarray(np.asarray(labels, dtype=np.int32))
    cap = k * (k - 1) // 2
    pairs = np.zeros(max(2 * cap, 2), dtype=np.int32)
    aut = ctypes.c_uint64()
    n = ctypes.c_int32()
    st = _lib.gsm_query_symmetry(k, e.size // 2, _ptr(e) if e.size else None,
                                 _ptr(lab) if lab is not None else None, ctypes.byref(aut),
                                 _ptr(pairs), cap, ctypes.byref(n))
    if st != GSM_OK:
        raise GsmError(st, "gsm_query_symmetry")
    return aut.value, [(int(pairs[2 * t]), int(pairs[2 * t + 1])) for t in range(n.value)]


def gsm_plan_order(k: int, edges, cand_sizes=None) -> tuple[np.ndarray, np.ndarray]:
    e = np.ascontiguousarray(np.asarray(edges, dtype=np.int32).reshape(-1))
    order = np.zeros(k, dtype=np.int32)
    parent = np.zeros(k, dtype=np.int32)
    cs = None if cand_sizes is None else np.ascontiguousarray(cand_sizes, dtype=np.uint64)
    st = _lib.gsm_plan_order(k, e.size // 2, _ptr(e) if e.size else None, _ptr(cs),
                             _ptr(order), _ptr(parent))
    if st != GSM_OK:
        raise GsmError(st, "gsm_plan_order")
    return order, parent


def gsm_kernel_stats(ctx: int, reset: bool = False) -> list[dict]:
    arr = (gsm_kernel_stat * 16)()
    n = ctypes.c_int32()
    _check(ctx, _lib.gsm_kernel_stats(ctx, arr, 16, ctypes.byref(n), int(reset)))
    return [{"name": arr[i].name.decode(), "launches": arr[i].launches,
             "total_ms": arr[i].total_ms, "algo_bytes": arr[i].algo_bytes,
             "items": arr[i].items, "probe_bytes": arr[i].probe_bytes}
            for i in range(min(n.value, 16))]


def gsm_last_run_stats(ctx: int) -> dict:
    s = gsm_run_stats()
    _check(ctx, _lib.gsm_last_run_stats(ctx, ctypes.byref(s)))
    k = s.k
    return {"k": k, "order": list(s.order[:k]), "cand_size": list(s.cand_size[:k]),
            "frontier": list(s.frontier[:k + 1]), "candidates": list(s.candidates[:k]),
            "chunks": s.chunks, "peak_bytes": s.peak_bytes,
            "kernel_launches": s.kernel_launches}


# ----------------------------------------------------------- convenience


class Query:
    def __init__(self, matcher: "Matcher", k: int, edges, labels=None):
        e = np.ascontiguousarray(np.asarray(edges, dtype=np.int32).reshape(-1))
        lab = None if labels is None else np.ascontiguousarray(labels, dtype=np.int32)
        self.k = int(k)
        self.m = e.size // 2
        self._e, self._lab = e, lab
        self.handle = gsm_query_create(matcher.ctx, k, self.m, e if e.size else None, lab)

    def restrict(self, u: int, lo: int, hi: int) -> "Query":
        gsm_query_restrict(self.handle, u, lo, hi)
        return self

    def close(self):
        if self.handle:
            gsm_query_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Matcher:
    """One libgsm context on one CUDA device, fed by torch's allocator.

    stream: a torch.cuda.Stream (or raw cudaStream_t) the context issues all
    work on; None creates a dedicated stream (self.stream)."""

    def __init__(self, device: int = 0, mem_budget_bytes: int = 0, stream=None,
                 block_size: int = 0, chunk_rows: int = 0, time_kernels: bool = False,
                 torch_allocator: bool = True, filter_rounds: int = 0, copy_slots: int = 0,
                 two_pass: bool = False, compressed: bool = False, lookback_spin_limit: int = 0,
                 inject_lookback_stall: bool = False, alloc_hook=None, lookahead: int = 0,
                 hub_bitmap_bytes: int = 0, host_workers: int = 0,
                 inject_sort_stall: bool = False, count_probes: bool = False,
                 inject_scan_stall: bool = False):
        import torch
        self.device = device
        opt = gsm_default_options()
        opt.mem_budget_bytes = mem_budget_bytes
        if stream is None:
            # a dedicated torch stream: every library kernel and copy runs on
            # it, so events recorded on self.stream bracket the library's work
            stream = torch.cuda.Stream(device=device)
        self.stream = stream
        opt.stream = ctypes.c_void_p(int(stream.cuda_stream) if hasattr(stream, "cuda_stream")
                                     else int(stream))
        opt.block_size = block_size
        opt.chunk_rows = chunk_rows
        opt.filter_rounds = filter_rounds
        opt.copy_slots = copy_slots
        opt.lookback_spin_limit = lookback_spin_limit
        opt.lookahead = lookahead
        opt.hub_bitmap_bytes = hub_bitmap_bytes
        opt.host_workers = host_workers
        opt.flags = (GSM_OPT_TIME_KERNELS if time_kernels else 0) | \
            (GSM_OPT_TWO_PASS if two_pass else 0) | \
            (GSM_OPT_COMPRESSED_FRONTIERS if compressed else 0) | \
            (GSM_OPT_INJECT_LOOKBACK_STALL if inject_lookback_stall else 0) | \
            (GSM_OPT_INJECT_SORT_STALL if inject_sort_stall else 0) | \
            (GSM_OPT_COUNT_PROBES if count_probes else 0) | \
            (GSM_OPT_INJECT_SCAN_STALL if inject_scan_stall else 0)
        if torch_allocator:
            dev = device

            def _alloc(_ctx, nbytes, stream_ptr):
                # alloc_hook(nbytes) -> False makes this allocation fail (tests)
                if alloc_hook is not None and not alloc_hook(int(nbytes)):
                    return None
                try:
                    return torch.cuda.caching_allocator_alloc(int(nbytes), dev, stream_ptr)
                except Exception:
                    return None

            def _free(_ctx, ptr, _nbytes, _stream):
                torch.cuda.caching_allocator_delete(ptr)

            self._cb = (_alloc_fn(_alloc), _free_fn(_free))
            opt.alloc, opt.free = self._cb
        self.ctx = gsm_create(device, opt)
        self.n = 0

    def close(self):
        if getattr(self, "ctx", None):
            gsm_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def load_graph(self, row_ptr, col, labels=None, validate: bool = False):
        """row_ptr/col/labels: numpy arrays (host) or CUDA torch tensors."""
        dev = _is_cuda(row_ptr)
        if not dev:
            row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int32)
            col = np.ascontiguousarray(col, dtype=np.int32)
            if labels is not None:
                labels = np.ascontiguousarray(labels, dtype=np.int32)
        n = int(row_ptr.shape[0]) - 1
        nnz = int(col.shape[0])
        flags = (GSM_DEVICE_PTRS if dev else 0) | (GSM_VALIDATE if validate else 0)
        gsm_load_graph(self.ctx, n, nnz, row_ptr, col if nnz else None, labels, flags)
        self.n = n

    def query(self, k: int, edges, labels=None) -> Query:
        return Query(self, k, edges, labels)

    def count(self, q: Query) -> int:
        return gsm_count(self.ctx, q.handle)

    def count_distinct(self, q: Query) -> tuple[int, int]:
        """(distinct subgraphs, automorphisms of the query)."""
        return gsm_count_distinct(self.ctx, q.handle)

    def enumerate(self, q: Query, cap_rows: int | None = None, out=None):
        """Returns (rows, count).  With out=None the rows come back as a numpy
        array of min(count, cap_rows) x k; out may be a CUDA int32 tensor of
        cap_rows*k elements (rows stay on the device)."""
        if out is not None:
            cap = int(out.numel()) // q.k if cap_rows is None else cap_rows
            flags = GSM_OUT_DEVICE if _is_cuda(out) else 0
            count, _ = gsm_enumerate(self.ctx, q.handle, out, cap, flags)
            return out, count
        if cap_rows is None:
            count, _ = gsm_enumerate(self.ctx, q.handle, None, 0, 0)
            buf = np.empty((max(count, 1), q.k), dtype=np.int32)
            gsm_last_rows(self.ctx, buf, 0, count, 0)
            return buf[:count], count
        buf = np.empty((max(cap_rows, 1), q.k), dtype=np.int32)
        count, _ = gsm_enumerate(self.ctx, q.handle, buf if cap_rows else None, cap_rows, 0)
        return buf[:min(count, cap_rows)], count

    def enumerate_many(self, queries, outs) -> list[int]:
        """Lists every Query of `queries` into the matching buffer of `outs`
        (int32 numpy arrays or tensors of cap_rows*k elements, all on the host
        or all CUDA); copies overlap the next query's compute.  Returns the
        counts."""
        flags = GSM_OUT_DEVICE if outs and _is_cuda(outs[0]) else 0
        caps = [int(o.numel() if hasattr(o, "numel") else o.size) // q.k
                for q, o in zip(queries, outs)]
        counts, _ = gsm_enumerate_many(self.ctx, [q.handle for q in queries], outs, caps, flags)
        return [int(c) for c in counts]

    def candidates(self, q: Query):
        nw = (self.n + 31) // 32
        bm = np.zeros((q.k, max(nw, 1)), dtype=np.uint32)
        sizes = np.zeros(q.k, dtype=np.uint64)
        gsm_candidates(self.ctx, q.handle, bm, sizes)
        return bm[:, :nw], sizes

    def run_batch(self, queries, autotune: bool = False, enumerate: bool = False,
                  device: bool = False):
        """Counts of every Query in `queries`, computed as one batch; with
        enumerate=True, (counts, rows) with each query's sorted rows (numpy,
        or CUDA tensors with device=True)."""
        flags = (GSM_BATCH_AUTOTUNE if autotune else 0) | (GSM_OUT_DEVICE if device else 0)
        r = gsm_run_batch(self.ctx, [q.handle for q in queries], flags, enumerate)
        if not enumerate:
            return [int(c) for c in r]
        return [int(c) for c in r[0]], r[1]

    def batch_stats(self) -> dict:
        return gsm_batch_get_stats(self.ctx)

    def kernel_stats(self, reset: bool = False):
        return gsm_kernel_stats(self.ctx, reset)

    def last_run_stats(self):
        return gsm_last_run_stats(self.ctx)


def unpack_bitmaps(bm: np.ndarray, n: int) -> np.ndarray:
    """uint32 bitmaps [k, words] -> uint8 [k, n] (bit v%32 of word v/32)."""
    bits = np.unpackbits(bm.view(np.uint8).reshape(bm.shape[0], -1), axis=1, bitorder="little")
    return bits[:, :n]
