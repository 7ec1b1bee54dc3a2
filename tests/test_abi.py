"""CPU-only checks of the C-ABI library: it builds, loads, exports every
function include/lb.h declares, its ctypes mirrors match the C struct
layouts, and host-side argument validation answers without touching a GPU."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

from paper_1711_00231_gb300 import _build
from paper_1711_00231_gb300 import lb

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lb.h")


@pytest.fixture(scope="module", autouse=True)
def built():
    _build.build()


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lb_[a-z_0-9]+)\s*\(", src)))


def test_exports_every_declared_symbol():
    names = declared_functions()
    assert len(names) >= 18
    libc = ctypes.CDLL(lb.LIB_PATH)
    missing = [n for n in names if not hasattr(libc, n)]
    assert not missing, missing
    out = subprocess.run(["nm", "-D", "--defined-only", lb.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (lb_\w+)", out))
    assert set(names) <= exported


def test_struct_layouts_match_header(tmp_path):
    prog = tmp_path / "layout.c"
    prog.write_text(r'''
#include <stdio.h>
#include <stddef.h>
#include "lb.h"
int main(void) {
  printf("%zu %zu %zu %zu\n", sizeof(lb_options), sizeof(lb_mem_stats), sizeof(lb_query_stats), sizeof(lb_step_record));
  printf("%zu %zu %zu %zu\n", offsetof(lb_query_stats, status), offsetof(lb_query_stats, device_ms), offsetof(lb_mem_stats, ns_split), offsetof(lb_step_record, t_ns));
  printf("%zu %zu %zu %zu\n", sizeof(lb_server_state_t), sizeof(lb_slot_state_t), offsetof(lb_server_state_t, slot), offsetof(lb_slot_state_t, ticket));
  printf("%zu %zu %zu %zu %zu %zu %zu %zu\n", offsetof(lb_options, hp_mode), offsetof(lb_options, hp_warp_max),
         offsetof(lb_options, ns_mode), offsetof(lb_options, thread_max), offsetof(lb_options, hp_depth),
         offsetof(lb_options, small_edges), offsetof(lb_options, bitmap_place), sizeof(lb_options));
  printf("%zu %zu %zu %zu %zu %zu\n", offsetof(lb_server_options, mem_fraction), offsetof(lb_server_options, launch_ms),
         offsetof(lb_server_options, policy), sizeof(lb_server_options), offsetof(lb_server_info_t, pending),
         sizeof(lb_server_info_t));
  return 0;
}''')
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)])
    a, b, c, d, e = subprocess.check_output([str(exe)], text=True).strip().splitlines()
    sizes = [int(x) for x in a.split()]
    offs = [int(x) for x in b.split()]
    assert sizes == [ctypes.sizeof(lb.lb_options), ctypes.sizeof(lb.lb_mem_stats), ctypes.sizeof(lb.lb_query_stats),
                     ctypes.sizeof(lb.lb_step_record)]
    assert offs == [lb.lb_query_stats.status.offset, lb.lb_query_stats.device_ms.offset, lb.lb_mem_stats.ns_split.offset,
                    lb.lb_step_record.t_ns.offset]
    assert [int(x) for x in c.split()] == [ctypes.sizeof(lb.lb_server_state_t), ctypes.sizeof(lb.lb_slot_state_t),
                                           lb.lb_server_state_t.slot.offset, lb.lb_slot_state_t.ticket.offset]
    assert [int(x) for x in d.split()] == [lb.lb_options.hp_mode.offset, lb.lb_options.hp_warp_max.offset,
                                           lb.lb_options.ns_mode.offset, lb.lb_options.thread_max.offset,
                                           lb.lb_options.hp_depth.offset, lb.lb_options.small_edges.offset,
                                           lb.lb_options.bitmap_place.offset, ctypes.sizeof(lb.lb_options)]
    assert [int(x) for x in e.split()] == [lb.lb_server_options.mem_fraction.offset,
                                           lb.lb_server_options.launch_ms.offset, lb.lb_server_options.policy.offset,
                                           ctypes.sizeof(lb.lb_server_options), lb.lb_server_info_t.pending.offset,
                                           ctypes.sizeof(lb.lb_server_info_t)]


def test_version_and_error_string():
    assert "sm_103a" in lb.lb_version()
    assert isinstance(lb.lb_last_error(), str)


@pytest.mark.parametrize("off,col,n,m,msg", [
    ([1, 1, 3], [1, 0, 1], 2, 3, "offsets[0]"),
    ([0, 2, 1], [1, 0], 2, 2, "offsets[n]"),
    ([0, 2, 1, 3], [1, 0, 1], 3, 3, "decrease"),
    ([0, 1, 3], [1, 0, 2], 2, 3, "out of range"),
    ([0, 1, 3], [1, 0, -1], 2, 3, "out of range"),
])
def test_graph_create_rejects_malformed_csr(off, col, n, m, msg):
    with pytest.raises(lb.LbError) as ei:
        lb.lb_graph_create(np.array(off), np.array(col), None, n, m)
    assert ei.value.status == lb.LB_ERR_ARG and msg in str(ei.value)


def test_argument_errors_need_no_gpu():
    L = lb.lib()
    h = ctypes.c_void_p()
    assert L.lb_graph_create(None, None, None, 3, 0, ctypes.byref(h)) == lb.LB_ERR_ARG
    off = np.zeros(2, np.int64)
    assert L.lb_graph_create(off.ctypes.data, None, None, 0, 0, ctypes.byref(h)) == lb.LB_ERR_ARG
    assert L.lb_graph_create(off.ctypes.data, None, None, 1 << 31, 0, ctypes.byref(h)) == lb.LB_ERR_ARG
    assert L.lb_graph_destroy(None) == lb.LB_OK
    assert L.lb_bfs(None, 0, 0, None) == lb.LB_ERR_ARG
    assert L.lb_sssp_dev(None, 0, 0, None, None, None) == lb.LB_ERR_ARG
    srcs = np.zeros(2, dtype=np.int32)
    assert L.lb_bfs_batch(None, srcs.ctypes.data, 2, 0, None) == lb.LB_ERR_ARG
    assert L.lb_sssp_batch(None, srcs.ctypes.data, 2, 0, None) == lb.LB_ERR_ARG
    st = lb.lb_query_stats()
    assert L.lb_last_stats(None, ctypes.byref(st)) == lb.LB_ERR_ARG
    ms = lb.lb_mem_stats()
    assert L.lb_mem_report(None, 0, ctypes.byref(ms)) == lb.LB_ERR_ARG
    assert L.lb_mdt(None, 10, None, None, None) == lb.LB_ERR_ARG
    deg = np.array([5, 7], np.int64)
    no = np.zeros(4, np.int64)
    ept = ctypes.c_int64()
    assert L.lb_wd_offsets(deg.ctypes.data, 2, 0, no.ctypes.data, no.ctypes.data, ctypes.byref(ept)) == lb.LB_ERR_ARG
    bad = np.array([5, -1], np.int64)
    assert L.lb_wd_offsets(bad.ctypes.data, 2, 4, no.ctypes.data, no.ctypes.data, ctypes.byref(ept)) == lb.LB_ERR_ARG
    fn = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)(lambda s, c: 0)
    assert L.lb_set_allocator(ctypes.cast(fn, ctypes.c_void_p), None, None) == lb.LB_ERR_ARG
    assert L.lb_set_allocator(None, None, None) == lb.LB_OK


def test_server_argument_errors_need_no_gpu():
    L = lb.lib()
    h = ctypes.c_void_p()
    assert L.lb_server_create(None, 0, None, ctypes.byref(h)) == lb.LB_ERR_ARG
    assert L.lb_server_create(None, 1, None, None) == lb.LB_ERR_ARG
    tick = ctypes.c_uint64()
    assert L.lb_server_submit(None, 0, 0, 0, None, ctypes.byref(tick)) == lb.LB_ERR_ARG
    n = ctypes.c_int32()
    assert L.lb_server_poll(None, None, 0, ctypes.byref(n)) == lb.LB_ERR_ARG
    assert L.lb_server_state(None, None) == lb.LB_ERR_ARG
    assert L.lb_server_info(None, None) == lb.LB_ERR_ARG
    assert L.lb_server_stop(None) == lb.LB_ERR_ARG
    assert L.lb_server_destroy(None) == lb.LB_OK


def test_binding_names_match_header():
    for name in declared_functions():
        assert hasattr(lb, name), f"binding lacks {name}"


def test_batch_sources_are_marshalled_as_int32():
    # the batched calls take any 1-D sequence of vertex ids; the binding
    # passes it as a contiguous int32 array and refuses what cannot be one
    a = lb._sources([3, 1, 2])
    assert a.dtype == np.int32 and a.flags["C_CONTIGUOUS"] and a.tolist() == [3, 1, 2]
    assert lb._sources([]).size == 0
    with pytest.raises(ValueError):
        lb._sources([[0, 1]])
    with pytest.raises(ValueError):
        lb._sources([1 << 31])
