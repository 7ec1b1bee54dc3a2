"""Thin ctypes binding of ``liblb.so`` (include/lb.h).

Every function here only marshals arguments (numpy arrays, torch tensors,
ints) into the C ABI; all graph work runs in the library's CUDA kernels.
The binding never falls back to anything else: if ``liblb.so`` is missing
it raises ImportError-style errors at load time.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblb.so")

# lb_strategy
LB_BS, LB_EP, LB_WD, LB_NS, LB_HP, LB_NS_PHYS, LB_EP_NOCHUNK, LB_AUTO = 0, 1, 2, 3, 4, 5, 6, 15
STRATEGIES = {"BS": LB_BS, "EP": LB_EP, "WD": LB_WD, "NS": LB_NS, "HP": LB_HP, "NS_PHYS": LB_NS_PHYS,
              "EP_NOCHUNK": LB_EP_NOCHUNK, "AUTO": LB_AUTO}
# lb_status
LB_OK, LB_ERR_ARG, LB_ERR_OOM, LB_ERR_CUDA, LB_ERR_OVERFLOW = 0, -1, -2, -3, -4
LB_ERR_TIMEOUT, LB_ERR_UNSUPPORTED, LB_ERR_INTERNAL = -5, -6, -7
STATUS_NAMES = {0: "LB_OK", -1: "LB_ERR_ARG", -2: "LB_ERR_OOM", -3: "LB_ERR_CUDA", -4: "LB_ERR_OVERFLOW",
                -5: "LB_ERR_TIMEOUT", -6: "LB_ERR_UNSUPPORTED", -7: "LB_ERR_INTERNAL"}
LB_KIND_BFS, LB_KIND_SSSP = 0, 1


class LbError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class lb_options(ctypes.Structure):
    _fields_ = [("hist_bins", ctypes.c_int32), ("mdt_override", ctypes.c_int32), ("hp_threshold", ctypes.c_int32),
                ("loop_mode", ctypes.c_int32), ("wd_tile", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32),
                ("hp_mode", ctypes.c_int32), ("hp_warp_max", ctypes.c_int32), ("ns_mode", ctypes.c_int32),
                ("thread_max", ctypes.c_int32), ("hp_depth", ctypes.c_int32), ("small_edges", ctypes.c_int32),
                ("test_barrier_skip", ctypes.c_int32), ("bitmap_place", ctypes.c_int32),
                ("reserved", ctypes.c_int32 * 2)]


class lb_mem_stats(ctypes.Structure):
    _fields_ = [(k, ctypes.c_int64) for k in (
        "csr_offsets", "csr_cols", "csr_weights", "status", "visited", "node_lists", "tile_starts", "coo_src",
        "edge_lists", "sub_lists", "control", "extra_total", "base_total", "resident", "ns_children", "mdt",
        "ns_split")]

    def as_dict(self):
        return {k: int(getattr(self, k)) for k, _ in self._fields_}


class lb_query_stats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int64), ("steps", ctypes.c_int64), ("edges_relaxed", ctypes.c_int64),
                ("pushes", ctypes.c_int64), ("mdt", ctypes.c_int64), ("status", ctypes.c_int32),
                ("strategy", ctypes.c_int32), ("device_ms", ctypes.c_double)]

    def as_dict(self):
        return {k: (float(getattr(self, k)) if k == "device_ms" else int(getattr(self, k))) for k, _ in self._fields_}


class lb_server_options(ctypes.Structure):
    _fields_ = [("slots", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32), ("tile", ctypes.c_int32),
                ("idle_us", ctypes.c_int32), ("mem_fraction", ctypes.c_double), ("launch_ms", ctypes.c_int32),
                ("policy", ctypes.c_int32), ("items", ctypes.c_int32), ("reserved", ctypes.c_int32 * 5)]


class lb_server_info_t(ctypes.Structure):
    _fields_ = [("slots", ctypes.c_int32), ("grid", ctypes.c_int32), ("slot_bytes", ctypes.c_int64),
                ("slot_n", ctypes.c_int64), ("kernel_launches", ctypes.c_int64), ("submitted", ctypes.c_int64),
                ("completed", ctypes.c_int64), ("pool_bytes", ctypes.c_int64), ("pool_free", ctypes.c_int64),
                ("pending", ctypes.c_int64)]

    def as_dict(self):
        return {k: int(getattr(self, k)) for k, _ in self._fields_}


class lb_completion(ctypes.Structure):
    _fields_ = [("ticket", ctypes.c_uint64), ("status", ctypes.c_int32), ("graph", ctypes.c_int32),
                ("iterations", ctypes.c_int64), ("edges_relaxed", ctypes.c_int64), ("device_ns", ctypes.c_int64)]


class lb_slot_state_t(ctypes.Structure):
    _fields_ = [("slot", ctypes.c_int32), ("graph", ctypes.c_int32), ("kind", ctypes.c_int32), ("level", ctypes.c_int32),
                ("job_kind", ctypes.c_int32), ("job_tiles", ctypes.c_int32), ("job_done", ctypes.c_int32),
                ("job_gen", ctypes.c_int32), ("claim", ctypes.c_int64), ("in_cnt", ctypes.c_int64),
                ("in_edges", ctypes.c_int64), ("error", ctypes.c_int32), ("pad", ctypes.c_int32),
                ("ticket", ctypes.c_int64)]


class lb_server_state_t(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("consumed", ctypes.c_int64), ("completed", ctypes.c_int64),
                ("acked", ctypes.c_int64), ("active", ctypes.c_int32), ("stopping", ctypes.c_int32),
                ("admit_lock", ctypes.c_int32), ("kernel_error", ctypes.c_int32), ("kernel_running", ctypes.c_int32),
                ("busy_slots", ctypes.c_int32), ("listed", ctypes.c_int32), ("pad", ctypes.c_int32),
                ("prof", ctypes.c_int64 * 8), ("slot", lb_slot_state_t * 16)]


class lb_step_record(ctypes.Structure):
    _fields_ = [("level", ctypes.c_int32), ("mode", ctypes.c_int32), ("list_size", ctypes.c_int64),
                ("edges", ctypes.c_int64), ("t_ns", ctypes.c_int64)]


_lib = None
_alloc_keepalive = []  # every allocator callback pair ever installed


def _load():
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with paper_1711_00231_gb300._build.build()")
    lib = ctypes.CDLL(LIB_PATH)
    P, i64, i32, st = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int
    sig = {
        "lb_graph_create": ([P, P, P, i64, i64, ctypes.POINTER(P)], st),
        "lb_graph_create_dev": ([P, P, P, i64, i64, ctypes.POINTER(P)], st),
        "lb_graph_destroy": ([P], st),
        "lb_graph_info": ([P, P, P, P, P], st),
        "lb_set_options": ([P, ctypes.POINTER(lb_options)], st),
        "lb_get_options": ([P, ctypes.POINTER(lb_options)], st),
        "lb_bfs": ([P, i32, st, P], st),
        "lb_sssp": ([P, i32, st, P], st),
        "lb_bfs_batch": ([P, P, i64, st, P], st),
        "lb_sssp_batch": ([P, P, i64, st, P], st),
        "lb_bfs_dev": ([P, i32, st, P, P, P], st),
        "lb_sssp_dev": ([P, i32, st, P, P, P], st),
        "lb_last_stats": ([P, ctypes.POINTER(lb_query_stats)], st),
        "lb_last_trace": ([P, P, i64, ctypes.POINTER(i64)], st),
        "lb_mem_report": ([P, st, ctypes.POINTER(lb_mem_stats)], st),
        "lb_release_workspaces": ([P], st),
        "lb_mdt": ([P, i32, P, P, P], st),
        "lb_wd_offsets": ([P, i64, i64, P, P, P], st),
        "lb_set_allocator": ([P, P, P], st),
        "lb_bfs_wd_noalloc": ([P, P, i64, i64, i32, P, P], st),
        "lb_autotune": ([P, i32, st, P, i32, ctypes.POINTER(lb_options), ctypes.POINTER(ctypes.c_double)], st),
        "lb_server_create": ([P, i32, ctypes.POINTER(lb_server_options), ctypes.POINTER(P)], st),
        "lb_server_destroy": ([P], st),
        "lb_server_info": ([P, ctypes.POINTER(lb_server_info_t)], st),
        "lb_server_submit": ([P, i32, i32, i32, P, ctypes.POINTER(ctypes.c_uint64)], st),
        "lb_server_poll": ([P, P, i32, ctypes.POINTER(i32)], st),
        "lb_server_stop": ([P], st),
        "lb_server_autotune": ([P, i32, ctypes.POINTER(lb_server_options), P, P, P, i32,
                                ctypes.POINTER(lb_server_options), ctypes.POINTER(ctypes.c_double)], st),
        "lb_server_state": ([P, ctypes.POINTER(lb_server_state_t)], st),
        "lb_last_error": ([], ctypes.c_char_p),
        "lb_version": ([], ctypes.c_char_p),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    _lib = lib
    return lib


def lib():
    return _load()


def _check(rc: int):
    if rc != LB_OK:
        raise LbError(rc, _load().lb_last_error().decode(errors="replace"))


def _ptr(x) -> Optional[int]:
    """Data pointer of a numpy array or torch tensor (contiguous), or None."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be contiguous")
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr()
    raise TypeError(f"unsupported buffer type {type(x)}")


def _need(buf, count: int, what: str = "output") -> None:
    """Device buffers cannot be checked by the C ABI: refuse one that is
    smaller than the graph before the kernels write past its end."""
    if buf is None:
        return
    have = buf.numel() if hasattr(buf, "numel") else np.asarray(buf).size
    if have < count:
        raise ValueError(f"{what} buffer holds {have} elements, the graph needs {count}")
    esz = buf.element_size() if hasattr(buf, "element_size") else np.asarray(buf).itemsize
    if esz != 4:
        raise ValueError(f"{what} buffer must have 4-byte elements")


def _stream_handle(stream) -> Optional[int]:
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


# ------------------------------------------------------------ C-ABI calls


def lb_version() -> str:
    return _load().lb_version().decode()


def lb_last_error() -> str:
    return _load().lb_last_error().decode(errors="replace")


def lb_graph_create(offsets, cols, weights, n: int, m: int) -> int:
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    col = np.ascontiguousarray(cols, dtype=np.int32)
    w = None if weights is None else np.ascontiguousarray(weights, dtype=np.uint32)
    if off.size != n + 1 or col.size != m or (w is not None and w.size != m):
        raise ValueError("array sizes do not match n / m")
    h = ctypes.c_void_p()
    _check(_load().lb_graph_create(_ptr(off), _ptr(col), _ptr(w), n, m, ctypes.byref(h)))
    return h.value


def lb_graph_create_dev(offsets_dev, cols_dev, weights_dev, n: int, m: int) -> int:
    h = ctypes.c_void_p()
    _check(_load().lb_graph_create_dev(_ptr(offsets_dev), _ptr(cols_dev), _ptr(weights_dev), n, m, ctypes.byref(h)))
    return h.value


def lb_graph_destroy(g: int) -> None:
    _check(_load().lb_graph_destroy(g))


def lb_graph_info(g: int):
    n, m, w, d = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int32(), ctypes.c_int32()
    _check(_load().lb_graph_info(g, ctypes.byref(n), ctypes.byref(m), ctypes.byref(w), ctypes.byref(d)))
    return dict(n=n.value, m=m.value, weighted=bool(w.value), device=d.value)


def lb_set_options(g: int, **kw) -> None:
    o = lb_options()
    _check(_load().lb_get_options(g, ctypes.byref(o)))
    for k, v in kw.items():
        if not hasattr(o, k) or k == "reserved":
            raise KeyError(k)
        setattr(o, k, int(v))
    _check(_load().lb_set_options(g, ctypes.byref(o)))


def lb_get_options(g: int) -> dict:
    o = lb_options()
    _check(_load().lb_get_options(g, ctypes.byref(o)))
    return {k: int(getattr(o, k)) for k, _ in o._fields_ if k != "reserved"}


def _strategy(s) -> int:
    return STRATEGIES[s.upper()] if isinstance(s, str) else int(s)


def lb_bfs(g: int, src: int, strategy, levels_out: np.ndarray) -> int:
    """Host-output BFS; returns the lb_status (raises on argument errors)."""
    rc = _load().lb_bfs(g, src, _strategy(strategy), _ptr(levels_out))
    if rc not in (LB_OK,):
        _check(rc)
    return rc


def lb_sssp(g: int, src: int, strategy, dist_out: np.ndarray) -> int:
    """Host-output SSSP; returns LB_OK or LB_ERR_OVERFLOW, raises otherwise."""
    rc = _load().lb_sssp(g, src, _strategy(strategy), _ptr(dist_out))
    if rc not in (LB_OK, LB_ERR_OVERFLOW):
        _check(rc)
    return rc


def _sources(srcs) -> np.ndarray:
    a = np.ascontiguousarray(np.asarray(srcs, dtype=np.int64))
    if a.ndim != 1 or (a.size and (a.min() < -(1 << 31) or a.max() >= (1 << 31))):
        raise ValueError("sources must be a 1-D sequence of int32 vertex ids")
    return a.astype(np.int32)


def lb_bfs_batch(g: int, srcs, strategy, levels_out: np.ndarray) -> int:
    """Host-output BFS from every source (results row by row in levels_out,
    k x n int32); returns the lb_status (raises on other errors)."""
    a = _sources(srcs)
    rc = _load().lb_bfs_batch(g, _ptr(a), a.size, _strategy(strategy), _ptr(levels_out))
    if rc != LB_OK:
        _check(rc)
    return rc


def lb_sssp_batch(g: int, srcs, strategy, dist_out: np.ndarray) -> int:
    """Host-output SSSP from every source (k x n uint32); returns LB_OK or
    LB_ERR_OVERFLOW, raises otherwise."""
    a = _sources(srcs)
    rc = _load().lb_sssp_batch(g, _ptr(a), a.size, _strategy(strategy), _ptr(dist_out))
    if rc not in (LB_OK, LB_ERR_OVERFLOW):
        _check(rc)
    return rc


def lb_bfs_dev(g: int, src: int, strategy, out_dev, parents_dev=None, stream=None) -> None:
    _check(_load().lb_bfs_dev(g, src, _strategy(strategy), _ptr(out_dev), _ptr(parents_dev), _stream_handle(stream)))


def lb_sssp_dev(g: int, src: int, strategy, out_dev, parents_dev=None, stream=None) -> None:
    _check(_load().lb_sssp_dev(g, src, _strategy(strategy), _ptr(out_dev), _ptr(parents_dev),
                               _stream_handle(stream)))


def lb_last_stats(g: int) -> dict:
    s = lb_query_stats()
    _check(_load().lb_last_stats(g, ctypes.byref(s)))
    return s.as_dict()


def lb_last_trace(g: int, cap: int = 4096) -> np.ndarray:
    buf = (lb_step_record * cap)()
    ln = ctypes.c_int64()
    _check(_load().lb_last_trace(g, ctypes.cast(buf, ctypes.c_void_p), cap, ctypes.byref(ln)))
    k = min(ln.value, cap)
    return np.array([(buf[i].level, buf[i].mode, buf[i].list_size, buf[i].edges, buf[i].t_ns) for i in range(k)],
                    dtype=[("level", np.int32), ("mode", np.int32), ("list_size", np.int64), ("edges", np.int64),
                           ("t_ns", np.int64)])


def lb_mem_report(g: int, strategy) -> dict:
    s = lb_mem_stats()
    _check(_load().lb_mem_report(g, _strategy(strategy), ctypes.byref(s)))
    return s.as_dict()


def lb_release_workspaces(g: int) -> None:
    _check(_load().lb_release_workspaces(g))


def lb_autotune(g: int, kind: int, strategy, srcs):
    """Picks the fastest options for (kind, strategy) on these sources and
    keeps them on the graph; returns (options dict, mean ms per query)."""
    a = np.ascontiguousarray(srcs, dtype=np.int32)
    o = lb_options()
    ms = ctypes.c_double()
    _check(_load().lb_autotune(g, kind, _strategy(strategy), _ptr(a), a.size, ctypes.byref(o), ctypes.byref(ms)))
    return {k: int(getattr(o, k)) for k, _ in o._fields_ if k != "reserved"}, float(ms.value)


def lb_mdt(g: int, bins: int = 10):
    mdt, md, b = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int32()
    _check(_load().lb_mdt(g, bins, ctypes.byref(mdt), ctypes.byref(md), ctypes.byref(b)))
    return mdt.value, md.value, b.value


def lb_wd_offsets(deg, T: int):
    d = np.ascontiguousarray(deg, dtype=np.int64)
    no = np.empty(T, dtype=np.int64)
    eo = np.empty(T, dtype=np.int64)
    ept = ctypes.c_int64()
    _check(_load().lb_wd_offsets(_ptr(d) if d.size else None, d.size, T, _ptr(no), _ptr(eo), ctypes.byref(ept)))
    return ept.value, no, eo


def lb_bfs_wd_noalloc(offsets_dev, cols_dev, n: int, m: int, src: int, levels_dev, stream=None) -> None:
    """BFS (workload decomposition) that allocates no device memory: for
    callers whose GPU memory belongs to another allocator or that must not
    call cudaMalloc while serving.  Scratch comes from a fixed array inside
    the library; n <= 131072, m <= 16777216."""
    if n <= (1 << 17) and m <= (1 << 24):
        _need(levels_dev, n, "levels")
    _check(_load().lb_bfs_wd_noalloc(_ptr(offsets_dev), _ptr(cols_dev), n, m, src, _ptr(levels_dev),
                                     _stream_handle(stream)))


def lb_server_autotune(graphs, requests, **base) -> tuple:
    """Best server options for a sample of requests [(graph, src, kind)]:
    returns (options dict, queries/s)."""
    arr = (ctypes.c_void_p * len(graphs))(*graphs)
    g = np.ascontiguousarray([r[0] for r in requests], dtype=np.int32)
    sr = np.ascontiguousarray([r[1] for r in requests], dtype=np.int32)
    k = np.ascontiguousarray([r[2] for r in requests], dtype=np.int32)
    b = lb_server_options(**base)
    o = lb_server_options()
    q = ctypes.c_double()
    _check(_load().lb_server_autotune(ctypes.cast(arr, ctypes.c_void_p), len(graphs), ctypes.byref(b), _ptr(g), _ptr(sr),
                                      _ptr(k), len(requests), ctypes.byref(o), ctypes.byref(q)))
    return {f: (float(getattr(o, f)) if f == "mem_fraction" else int(getattr(o, f)))
            for f, _ in o._fields_ if f != "reserved"}, float(q.value)


def lb_server_create(graphs, slots: int = 0, ctas_per_sm: int = 0, tile: int = 0, idle_us: int = 0,
                     mem_fraction: float = 0.0, launch_ms: int = 0, policy: int = 0, items: int = 0) -> int:
    """Persistent multi-query engine over resident graphs (lb_graph handles)."""
    arr = (ctypes.c_void_p * len(graphs))(*graphs)
    o = lb_server_options(slots=slots, ctas_per_sm=ctas_per_sm, tile=tile, idle_us=idle_us, mem_fraction=mem_fraction,
                          launch_ms=launch_ms, policy=policy, items=items)
    h = ctypes.c_void_p()
    _check(_load().lb_server_create(ctypes.cast(arr, ctypes.c_void_p), len(graphs), ctypes.byref(o), ctypes.byref(h)))
    return h.value


def lb_server_destroy(s: int) -> None:
    _check(_load().lb_server_destroy(s))


def lb_server_info(s: int) -> dict:
    i = lb_server_info_t()
    _check(_load().lb_server_info(s, ctypes.byref(i)))
    return i.as_dict()


def lb_server_submit(s: int, graph: int, src: int, kind: int, out_dev) -> int:
    t = ctypes.c_uint64()
    _check(_load().lb_server_submit(s, graph, src, kind, _ptr(out_dev), ctypes.byref(t)))
    return int(t.value)


_POLL_CAP = 4096
_poll_buf = None


def lb_server_poll(s: int, cap: int = _POLL_CAP):
    """List of completion dicts (ticket, status, graph, iterations,
    edges_relaxed, device_ns)."""
    global _poll_buf
    if _poll_buf is None or len(_poll_buf) < cap:
        _poll_buf = (lb_completion * cap)()
    n = ctypes.c_int32()
    _check(_load().lb_server_poll(s, ctypes.cast(_poll_buf, ctypes.c_void_p), cap, ctypes.byref(n)))
    return [(int(c.ticket), int(c.status), int(c.graph), int(c.iterations), int(c.edges_relaxed), int(c.device_ns))
            for c in _poll_buf[:n.value]]


def lb_server_state(s: int) -> dict:
    """Diagnostic snapshot of the serving engine (counters and busy slots)."""
    x = lb_server_state_t()
    _check(_load().lb_server_state(s, ctypes.byref(x)))
    d = {k: int(getattr(x, k)) for k, _ in x._fields_ if k not in ("slot", "pad", "prof")}
    d["prof"] = [int(v) for v in x.prof]
    d["slots"] = [{k: int(getattr(x.slot[i], k)) for k, _ in lb_slot_state_t._fields_ if k != "pad"}
                  for i in range(x.listed)]
    return d


def lb_server_stop(s: int) -> None:
    _check(_load().lb_server_stop(s))


_ALLOC_T = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
_FREE_T = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)


def lb_set_allocator(alloc_fn=None, free_fn=None) -> None:
    """Install Python callables alloc(bytes) -> int and free(ptr) as the
    library's device allocator (None, None restores cudaMalloc).  A graph
    keeps the allocator it was created with, so every installed pair stays
    alive for the life of the process."""
    if alloc_fn is None:
        _check(_load().lb_set_allocator(None, None, None))
        return
    a = _ALLOC_T(lambda size, ctx: alloc_fn(int(size)) or 0)
    f = _FREE_T(lambda ptr, ctx: free_fn(int(ptr)) if ptr else None)
    _check(_load().lb_set_allocator(ctypes.cast(a, ctypes.c_void_p), ctypes.cast(f, ctypes.c_void_p), None))
    _alloc_keepalive.append((a, f))


def use_torch_allocator() -> None:
    """Route the library's device allocations through PyTorch's caching
    allocator (memory then shows up in torch.cuda.memory_allocated())."""
    import torch

    def alloc(size: int) -> int:
        try:
            return int(torch.cuda.caching_allocator_alloc(size))
        except RuntimeError:
            return 0

    def free(ptr: int) -> None:
        torch.cuda.caching_allocator_delete(ptr)

    lb_set_allocator(alloc, free)


# ------------------------------------------------------------ convenience


class Graph:
    """Owns an lb_graph handle; methods are the C-ABI calls above."""

    def __init__(self, offsets, cols, weights=None, n: Optional[int] = None, m: Optional[int] = None,
                 device_arrays: bool = False):
        if n is None:
            n = int(len(offsets) - 1)
        if m is None:
            m = int(len(cols))
        self.n, self.m = n, m
        self.weighted = weights is not None
        if device_arrays:
            self.h = lb_graph_create_dev(offsets, cols, weights, n, m)
        else:
            self.h = lb_graph_create(offsets, cols, weights, n, m)

    @classmethod
    def from_csr(cls, g):
        return cls(g.offsets, g.cols, g.weights, g.n, g.m)

    def close(self):
        if getattr(self, "h", None):
            lb_graph_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def bfs(self, src: int, strategy="WD") -> np.ndarray:
        out = np.empty(self.n, dtype=np.int32)
        lb_bfs(self.h, src, strategy, out)
        return out

    def sssp(self, src: int, strategy="WD"):
        out = np.empty(self.n, dtype=np.uint32)
        rc = lb_sssp(self.h, src, strategy, out)
        return out, rc

    def _batch_out(self, srcs, out, dtype):
        k = len(srcs)
        if out is None:
            out = np.empty((k, self.n), dtype=dtype)
        if not isinstance(out, np.ndarray) or out.dtype != dtype or out.size != k * self.n:
            raise ValueError(f"output must be a {dtype.__name__} array of {k} x {self.n} elements")
        return out

    def bfs_batch(self, srcs, strategy="WD", out=None) -> np.ndarray:
        """Levels from every source, one row per source (pass pinned host
        memory as out to overlap the copies with the traversals)."""
        out = self._batch_out(srcs, out, np.int32)
        lb_bfs_batch(self.h, srcs, strategy, out)
        return out

    def sssp_batch(self, srcs, strategy="WD", out=None):
        out = self._batch_out(srcs, out, np.uint32)
        rc = lb_sssp_batch(self.h, srcs, strategy, out)
        return out, rc

    def bfs_dev(self, src, strategy, out_dev, parents_dev=None, stream=None):
        _need(out_dev, self.n)
        _need(parents_dev, self.n, "parents")
        lb_bfs_dev(self.h, src, strategy, out_dev, parents_dev, stream)

    def sssp_dev(self, src, strategy, out_dev, parents_dev=None, stream=None):
        _need(out_dev, self.n)
        _need(parents_dev, self.n, "parents")
        lb_sssp_dev(self.h, src, strategy, out_dev, parents_dev, stream)

    def stats(self) -> dict:
        return lb_last_stats(self.h)

    def trace(self) -> np.ndarray:
        return lb_last_trace(self.h)

    def mem_report(self, strategy) -> dict:
        return lb_mem_report(self.h, strategy)

    def set_options(self, **kw):
        lb_set_options(self.h, **kw)

    def options(self) -> dict:
        return lb_get_options(self.h)

    def mdt(self, bins: int = 10):
        return lb_mdt(self.h, bins)

    def autotune(self, kind: str, strategy, srcs):
        """kind: "bfs", "sssp" or "both" (one BFS and one SSSP per source)."""
        return lb_autotune(self.h, {"bfs": LB_KIND_BFS, "sssp": LB_KIND_SSSP, "both": 2}[kind], strategy, srcs)

    def release(self):
        lb_release_workspaces(self.h)
