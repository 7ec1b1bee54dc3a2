"""CPU oracle: plain, slow, obviously correct BFS / SSSP and the schedule
artefacts of the load-balancing strategies (see ``oracle.c`` for the paper
passages each function follows).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import
this package.  It shares no code with the CUDA library and never imports it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

UNREACHED = 0xFFFFFFFF
SATURATED = 0xFFFFFFFE


def build(force: bool = False) -> str:
    """Compile ``liboracle.so`` with gcc if missing or stale."""
    with _lock:
        if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
            tmp = _LIB + f".tmp{os.getpid()}"
            subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-o", tmp, _SRC])
            os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32
        sigs = {
            "oracle_bfs": ([i64, P, P, i32, P], i64),
            "oracle_dijkstra": ([i64, P, P, P, i32, P], ctypes.c_int),
            "oracle_bellman_ford": ([i64, P, P, P, i32, P], ctypes.c_int),
            "oracle_floyd_warshall": ([i64, P, P, P, i32, P], ctypes.c_int),
            "oracle_check_dist": ([i64, P, P, P, i32, P, P], ctypes.c_int),
            "oracle_check_parents": ([i64, P, P, P, i32, P, P, P], ctypes.c_int),
            "oracle_mdt": ([i64, P, i32, P, P, P], i64),
            "oracle_wd_offsets": ([i64, P, i64, P, P], i64),
            "oracle_ns_chunks": ([i64, i64, P, i64], i64),
            "oracle_ns_split": ([i64, P, i64, P], i64),
            "oracle_hp_schedule": ([i64, P, i64, i64, i32, i32, P, P, P, i64], i64),
        }
        for name, (args, res) in sigs.items():
            f = getattr(lib, name)
            f.argtypes = args
            f.restype = res
        _lib = lib
    return _lib


def _p(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data


def _csr(g):
    off = np.ascontiguousarray(g.offsets, dtype=np.int64)
    col = np.ascontiguousarray(g.cols, dtype=np.int32)
    w = None if g.weights is None else np.ascontiguousarray(g.weights, dtype=np.uint32)
    return off, col, w


def bfs(g, src: int):
    """Levels (int32, -1 unreachable) and the number of BFS levels."""
    off, col, _ = _csr(g)
    lev = np.empty(g.n, dtype=np.int32)
    nlev = _load().oracle_bfs(g.n, _p(off), _p(col), src, _p(lev))
    if nlev < 0:
        raise ValueError("oracle_bfs: bad arguments")
    return lev, int(nlev)


def _sp(fn, g, src: int, unit: bool):
    off, col, w = _csr(g)
    if unit:
        w = None
    dist = np.empty(g.n, dtype=np.uint32)
    rc = fn(g.n, _p(off), _p(col), _p(w), src, _p(dist))
    if rc < 0:
        raise ValueError(f"{fn.__name__}: error {rc}")
    return dist, bool(rc == 1)


def dijkstra(g, src: int, unit: bool = False):
    """(dist uint32, overflow flag).  ``unit`` ignores the weights (w = 1)."""
    return _sp(_load().oracle_dijkstra, g, src, unit)


def bellman_ford(g, src: int, unit: bool = False):
    return _sp(_load().oracle_bellman_ford, g, src, unit)


def floyd_warshall(g, src: int, unit: bool = False):
    if g.n > 512:
        raise ValueError("floyd_warshall is for n <= 512")
    return _sp(_load().oracle_floyd_warshall, g, src, unit)


def check_dist(g, src: int, dist, unit: bool = False):
    """0 if ``dist`` (uint32; BFS levels viewed as uint32) satisfies the
    shortest-path invariants, else (code, vertex)."""
    off, col, w = _csr(g)
    if unit:
        w = None
    d = np.ascontiguousarray(np.asarray(dist).view(np.uint32) if np.asarray(dist).dtype == np.int32
                             else np.asarray(dist, dtype=np.uint32))
    bad = ctypes.c_int64(-1)
    rc = _load().oracle_check_dist(g.n, _p(off), _p(col), _p(w), src, _p(d), ctypes.addressof(bad))
    return 0 if rc == 0 else (rc, bad.value)


def check_parents(g, src: int, dist, parent, unit: bool = False):
    off, col, w = _csr(g)
    if unit:
        w = None
    d = np.ascontiguousarray(np.asarray(dist).view(np.uint32) if np.asarray(dist).dtype == np.int32
                             else np.asarray(dist, dtype=np.uint32))
    p = np.ascontiguousarray(parent, dtype=np.int32)
    bad = ctypes.c_int64(-1)
    rc = _load().oracle_check_parents(g.n, _p(off), _p(col), _p(w), src, _p(d), _p(p), ctypes.addressof(bad))
    return 0 if rc == 0 else (rc, bad.value)


def mdt(offsets, bins: int = 10):
    """(MDT, maxDeg, binIndex, histogram) of the histogram heuristic."""
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    n = off.size - 1
    maxdeg = ctypes.c_int64(0)
    b = ctypes.c_int32(0)
    hist = np.zeros(max(bins, 1), dtype=np.int64)
    r = _load().oracle_mdt(n, _p(off), bins, ctypes.addressof(maxdeg), ctypes.addressof(b), _p(hist))
    if r < 0:
        raise ValueError("oracle_mdt: bad arguments")
    return int(r), int(maxdeg.value), int(b.value), hist


def wd_offsets(deg, T: int):
    """(edgesPerThread, NodeOffset[T], EdgeOffset[T]) for a worklist with
    out-degrees ``deg`` cut over T threads."""
    d = np.ascontiguousarray(deg, dtype=np.int64)
    no = np.empty(T, dtype=np.int64)
    eo = np.empty(T, dtype=np.int64)
    ept = _load().oracle_wd_offsets(d.size, _p(d), T, _p(no), _p(eo))
    if ept < 0:
        raise ValueError("oracle_wd_offsets: bad arguments")
    return int(ept), no, eo


def ns_chunks(deg: int, mdt_: int):
    cap = max(1, -(-deg // max(mdt_, 1)))
    out = np.empty(cap, dtype=np.int64)
    k = _load().oracle_ns_chunks(deg, mdt_, _p(out), cap)
    if k < 0:
        raise ValueError("oracle_ns_chunks: bad arguments")
    return out[:k].copy()


def ns_split(offsets, mdt_: int):
    """(children created, nodes split)."""
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    ns = ctypes.c_int64(0)
    ch = _load().oracle_ns_split(off.size - 1, _p(off), mdt_, ctypes.addressof(ns))
    if ch < 0:
        raise ValueError("oracle_ns_split: bad arguments")
    return int(ch), int(ns.value)


def hp_schedule(deg, mdt_: int, threshold: int, cap: int = 1 << 16, depth: int = 1, bins: int = 10):
    """Steps of hierarchical processing over one super worklist: arrays of
    (list size, edges relaxed, mode 0 = sub-iteration / 1 = WD).  depth > 1:
    the first `depth` lists of the chain each take their own MDT (the
    histogram rule over the sub-list's remaining degrees, `bins` bins); the
    super list uses mdt_."""
    d = np.ascontiguousarray(deg, dtype=np.int64)
    ls = np.empty(cap, dtype=np.int64)
    ed = np.empty(cap, dtype=np.int64)
    md = np.empty(cap, dtype=np.int32)
    k = _load().oracle_hp_schedule(d.size, _p(d), mdt_, threshold, depth, bins, _p(ls), _p(ed), _p(md), cap)
    if k < 0:
        raise ValueError("oracle_hp_schedule: bad arguments")
    k = min(int(k), cap)
    return ls[:k].copy(), ed[:k].copy(), md[:k].copy()


def m_reached(g, dist) -> int:
    """Directed edges whose source is reached (each counted once): the
    traversed-edge count of a traversal that produced ``dist``."""
    d = np.asarray(dist)
    reached = (d.view(np.uint32) if d.dtype == np.int32 else d.astype(np.uint32)) != UNREACHED
    return int(np.diff(np.asarray(g.offsets, dtype=np.int64))[reached].sum())
