"""Seeded synthetic graph inputs shared by the CPU oracle and the GPU path.

Holds no traversal arithmetic: it only makes graphs (cleaned CSR: no
self-loops, no duplicate (u, v), adjacency sorted by destination), integer
edge weights and source draws, from one counter-based generator (splitmix64
outputs indexed by a per-purpose counter; see ``graphgen.c``).

The paper's evaluation graphs (GTgraph R-MAT and Erdos-Renyi graphs, DIMACS
USA road networks and Graph500 graphs; Section IV, Table II) are not
available here.  ``rmat`` stands in for the skewed low-diameter R-MAT and
Graph500 graphs, ``grid`` for the high-diameter near-uniform-degree road
networks, and ``erdos_renyi`` for the ER graphs.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass, field
from fractions import Fraction
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "graphgen.c")
_LIB = os.path.join(_HERE, "libgraphgen.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile ``libgraphgen.so`` with gcc if it is missing or stale."""
    with _lock:
        if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
            tmp = _LIB + f".tmp{os.getpid()}"
            subprocess.check_call(["gcc", "-O3", "-std=gnu11", "-fPIC", "-shared", "-pthread", "-o", tmp, _SRC])
            os.replace(tmp, _LIB)
    return _LIB


class _Csr(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int64),
        ("m", ctypes.c_int64),
        ("offsets", ctypes.POINTER(ctypes.c_int64)),
        ("cols", ctypes.POINTER(ctypes.c_int32)),
        ("weights", ctypes.POINTER(ctypes.c_uint32)),
    ]


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        i64, u64, u32, i32 = ctypes.c_int64, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int
        lib.gg_rmat.argtypes = [i32, i64, u64, u64, u64, u64, i32, u32, u32, i32, ctypes.POINTER(_Csr)]
        lib.gg_er.argtypes = [i64, i64, u64, i32, u32, u32, i32, ctypes.POINTER(_Csr)]
        lib.gg_grid.argtypes = [i64, i64, u64, i32, u32, u32, ctypes.POINTER(_Csr)]
        lib.gg_free.argtypes = [ctypes.POINTER(_Csr)]
        lib.gg_draw.argtypes = [u64, u64]
        lib.gg_draw.restype = u64
        lib.gg_stream.argtypes = [u64, u64]
        lib.gg_stream.restype = u64
        lib.gg_fill_weights.argtypes = [i64, u64, u32, u32, ctypes.c_void_p]
        lib.gg_pick_sources.argtypes = [i64, ctypes.c_void_p, i64, u64, ctypes.c_void_p]
        lib.gg_pick_sources.restype = i64
        for f in (lib.gg_rmat, lib.gg_er, lib.gg_grid):
            f.restype = ctypes.c_int
        _lib = lib
    return _lib


@dataclass
class CSRGraph:
    """A directed graph in CSR form: ``offsets`` int64 (n+1), ``cols`` int32
    (m), ``weights`` uint32 (m) or None."""

    n: int
    m: int
    offsets: np.ndarray
    cols: np.ndarray
    weights: Optional[np.ndarray]
    name: str = ""
    meta: dict = field(default_factory=dict)

    def degrees(self) -> np.ndarray:
        return np.diff(self.offsets)


def _take(csr: _Csr, name: str, meta: dict) -> CSRGraph:
    """Copy the C-allocated arrays into numpy and free them."""
    lib = _load()
    n, m = int(csr.n), int(csr.m)
    off = np.ctypeslib.as_array(csr.offsets, shape=(n + 1,)).copy()
    cols = np.ctypeslib.as_array(csr.cols, shape=(max(m, 1),))[:m].copy()
    w = None
    if bool(csr.weights):
        w = np.ctypeslib.as_array(csr.weights, shape=(max(m, 1),))[:m].copy()
    lib.gg_free(ctypes.byref(csr))
    return CSRGraph(n, m, off, cols, w, name, meta)


def _threshold(x: Fraction) -> int:
    """floor(x * 2^32), clamped to 2^32 - 1 (x = 1 then admits every draw but
    the all-ones one, which is accepted as the rounding of a 32-bit draw)."""
    t = (x.numerator << 32) // x.denominator
    return min(t, (1 << 32) - 1)


def _check(rc: int, what: str):
    if rc == -1:
        raise MemoryError(f"{what}: out of host memory")
    if rc != 0:
        raise ValueError(f"{what}: bad arguments (rc={rc})")


def rmat(scale: int, edge_factor: int, a="0.57", b="0.19", c="0.19", seed: int = 1,
         weights: Optional[Sequence[int]] = (1, 255), nthreads: int = 0) -> CSRGraph:
    """R-MAT graph with 2^scale vertices and edge_factor * 2^scale generated
    directed edges (before self-loop and duplicate removal).  ``a``, ``b``,
    ``c`` are decimal strings (d = 1 - a - b - c); their 32-bit thresholds are
    computed exactly so every platform produces the same graph."""
    fa, fb, fc = Fraction(str(a)), Fraction(str(b)), Fraction(str(c))
    if fa < 0 or fb < 0 or fc < 0 or fa + fb + fc > 1:
        raise ValueError("bad R-MAT probabilities")
    lib = _load()
    csr = _Csr()
    lo, hi = (weights if weights is not None else (0, 0))
    rc = lib.gg_rmat(scale, edge_factor << scale, _threshold(fa), _threshold(fa + fb), _threshold(fa + fb + fc),
                     seed, int(weights is not None), lo, hi, nthreads, ctypes.byref(csr))
    _check(rc, "rmat")
    meta = dict(kind="rmat", scale=scale, edge_factor=edge_factor, a=str(a), b=str(b), c=str(c), seed=seed,
                weights=None if weights is None else tuple(weights), generated_edges=edge_factor << scale)
    return _take(csr, f"rmat{scale}_ef{edge_factor}", meta)


def erdos_renyi(n: int, nedges: int, seed: int = 1, weights: Optional[Sequence[int]] = (1, 255),
                nthreads: int = 0) -> CSRGraph:
    """Uniform random directed graph: ``nedges`` independent (u, v) draws,
    self-loops and duplicates removed."""
    lib = _load()
    csr = _Csr()
    lo, hi = (weights if weights is not None else (0, 0))
    rc = lib.gg_er(n, nedges, seed, int(weights is not None), lo, hi, nthreads, ctypes.byref(csr))
    _check(rc, "erdos_renyi")
    meta = dict(kind="er", n=n, generated_edges=nedges, seed=seed, weights=None if weights is None else tuple(weights))
    return _take(csr, f"er_n{n}_m{nedges}", meta)


def grid(rows: int, cols: int, seed: int = 1, weights: Optional[Sequence[int]] = (1, 1000)) -> CSRGraph:
    """4-neighbour grid, vertex id r*cols+c, one weight per undirected edge."""
    lib = _load()
    csr = _Csr()
    lo, hi = (weights if weights is not None else (0, 0))
    rc = lib.gg_grid(rows, cols, seed, int(weights is not None), lo, hi, ctypes.byref(csr))
    _check(rc, "grid")
    meta = dict(kind="grid", rows=rows, cols=cols, seed=seed, weights=None if weights is None else tuple(weights))
    return _take(csr, f"grid{rows}x{cols}", meta)


def from_edges(n: int, src, dst, w=None, clean: bool = True, name: str = "edges") -> CSRGraph:
    """CSR from explicit edge arrays (small hand-made graphs).  With
    ``clean`` self-loops and duplicate (u, v) pairs are dropped (the first
    weight of a duplicate is kept); without it multi-edges and self-loops
    are kept as given."""
    src = np.asarray(src, dtype=np.int64)
    dst = np.asarray(dst, dtype=np.int64)
    if src.shape != dst.shape or (src.size and (src.min() < 0 or dst.min() < 0 or src.max() >= n or dst.max() >= n)):
        raise ValueError("bad edge arrays")
    ww = None if w is None else np.asarray(w, dtype=np.uint64)
    order = np.lexsort((np.arange(src.size), dst, src))
    src, dst = src[order], dst[order]
    if ww is not None:
        ww = ww[order]
    if clean and src.size:
        keep = src != dst
        first = np.ones(src.size, dtype=bool)
        first[1:] = (src[1:] != src[:-1]) | (dst[1:] != dst[:-1])
        keep &= first
        src, dst = src[keep], dst[keep]
        if ww is not None:
            ww = ww[keep]
    off = np.zeros(n + 1, dtype=np.int64)
    np.add.at(off, src + 1, 1)
    off = np.cumsum(off)
    return CSRGraph(n, int(dst.size), off, dst.astype(np.int32), None if ww is None else ww.astype(np.uint32), name,
                    dict(kind="edges"))


def fill_weights(g: CSRGraph, seed: int = 1, lo: int = 1, hi: int = 255) -> CSRGraph:
    """Attach uniform U[lo, hi] weights drawn per CSR edge index."""
    w = np.empty(g.m, dtype=np.uint32)
    if g.m:
        _load().gg_fill_weights(g.m, seed, lo, hi, w.ctypes.data)
    g.weights = w
    return g


def pick_sources(g: CSRGraph, count: int, seed: int = 1) -> np.ndarray:
    """``count`` distinct sources drawn uniformly among out-degree > 0 vertices."""
    out = np.empty(max(count, 1), dtype=np.int32)
    off = np.ascontiguousarray(g.offsets, dtype=np.int64)
    k = _load().gg_pick_sources(g.n, off.ctypes.data, count, seed, out.ctypes.data)
    if k < 0:
        raise MemoryError("pick_sources")
    return out[:k].copy()


def max_degree_vertex(g: CSRGraph) -> int:
    """Highest out-degree vertex, smallest id on ties."""
    return int(np.argmax(g.degrees()))


def draw(stream_seed: int, k: int) -> int:
    """k-th output of splitmix64 seeded with ``stream_seed`` (for tests)."""
    return int(_load().gg_draw(stream_seed, k))


def stream(seed: int, tag: int) -> int:
    return int(_load().gg_stream(seed, tag))
