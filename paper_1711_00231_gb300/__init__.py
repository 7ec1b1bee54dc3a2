"""GB300 (sm_103a) frontier BFS / SSSP with the dynamic load-balancing
strategies of arXiv 1711.00231 (workload decomposition, node splitting,
hierarchical processing) beside the node-based and edge-based baselines.

The compute path is ``liblb.so`` (CUDA, C ABI in include/lb.h); ``lb`` is
its thin ctypes binding.  Build with ``paper_1711_00231_gb300._build.build()``.
"""
from . import lb  # noqa: F401
from .lb import Graph, LbError, STRATEGIES  # noqa: F401

__all__ = ["lb", "Graph", "LbError", "STRATEGIES"]
