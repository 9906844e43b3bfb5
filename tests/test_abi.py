"""C ABI checks that need no GPU: the library builds and loads, exports every
symbol include/fg.h declares, rejects bad arguments on the host before any CUDA
call, and its host-only partitioner returns valid partitions."""
import ctypes
import re

import numpy as np
import pytest

from paper_2103_14915_gb300 import build as fgbuild
from paper_2103_14915_gb300 import fg, inputs

HEADER = fgbuild.ROOT / "include" / "fg.h"


@pytest.fixture(scope="module")
def lib():
    fgbuild.build()
    return fg.load()


def declared_functions():
    text = HEADER.read_text()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(fg_[a-z_]+)\s*\(", text)))


def test_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert len(names) >= 13
    for name in names:
        assert hasattr(lib, name), name
        assert ctypes.cast(getattr(lib, name), ctypes.c_void_p).value
    assert set(names) == set(fg.EXPORTS)


def test_every_declaration_is_documented():
    """Each declared entry point follows a comment block (within the few lines
    above it, or shares one with the declarations right before it)."""
    lines = HEADER.read_text().splitlines()
    undocumented, seen = [], []
    for i, line in enumerate(lines):
        m = re.match(r"^(?:fg_status|void|const char|[a-z_0-9]+_t)\s*\*?\s*(fg_[a-z_]+)\s*\(", line)
        if not m:
            continue
        seen.append(m.group(1))
        window = "\n".join(lines[max(0, i - 12):i])
        if "*/" not in window:
            undocumented.append(m.group(1))
    assert sorted(set(seen)) == declared_functions()
    assert not undocumented, undocumented


def test_struct_sizes_match_header(lib):
    o = fg.fg_default_opts()
    assert o.struct_size == ctypes.sizeof(fg.fg_opts)
    go = fg.fg_default_graph_opts()
    assert go.struct_size == ctypes.sizeof(fg.fg_graph_opts)
    so = fg.fg_default_server_opts()
    assert so.struct_size == ctypes.sizeof(fg.fg_server_opts)
    assert so.lanes == 4 and so.max_batch == 256 and abs(so.alpha - 0.15) < 1e-7
    assert all(so.opts[k].struct_size == ctypes.sizeof(fg.fg_opts) for k in range(3))
    assert go.partition_method == fg.FG_PART_AUTO and o.mode == fg.FG_MODE_BUFFERED


def _csr():
    g = inputs.grid(8, 8, 0, 0, seed=1, weights=(1, 9))
    return g


@pytest.mark.parametrize("case", ["n0", "rp0", "rpn", "decreasing", "col_range", "neg_w", "null_col", "null_out"])
def test_graph_create_rejects_bad_csr_on_host(lib, case):
    g = _csr()
    n, m, rp, col, w = g.n, g.m, g.row_ptr.copy(), g.col.copy(), g.w.copy()
    if case == "n0":
        n = 0
    elif case == "rp0":
        rp[0] = 1
    elif case == "rpn":
        rp[-1] = m - 1
    elif case == "decreasing":
        rp[5] = rp[6] + 1
    elif case == "col_range":
        col[3] = n
    elif case == "neg_w":
        w[7] = -1
    elif case == "null_col":
        col = None
    if case == "null_out":
        st = lib.fg_graph_create(n, m, rp.ctypes.data, col.ctypes.data, w.ctypes.data, 0, None)
    else:
        st, h = fg.fg_graph_create(n, m, rp, col, w)
        assert h is None
    assert st == fg.FG_ERR_INVALID_ARG
    assert fg.fg_last_error()


def test_graph_create_rejects_huge_m(lib):
    rp = np.zeros(2, dtype=np.int64)
    st, _ = fg.fg_graph_create(1, 1 << 32, rp, rp)
    assert st == fg.FG_ERR_UNSUPPORTED


def test_batch_rejects_null_graph(lib):
    src = np.zeros(4, dtype=np.int32)
    out = np.zeros(16, dtype=np.uint32)
    assert fg.fg_sssp_batch(None, src, 4, out) == fg.FG_ERR_INVALID_ARG
    assert fg.fg_bfs_batch(None, src, 4, out) == fg.FG_ERR_INVALID_ARG
    assert fg.fg_ppr_batch(None, src, 4, 0.15, 1e-4, out) == fg.FG_ERR_INVALID_ARG
    assert fg.fg_sssp_batch_noalloc(None, src, 4, out) == fg.FG_ERR_INVALID_ARG
    st, _ = fg.fg_server_create(None, fg.fg_default_server_opts())
    assert st == fg.FG_ERR_INVALID_ARG
    st, _ = fg.fg_server_submit(None, fg.FG_QUERY_SSSP, 0)
    assert st == fg.FG_ERR_INVALID_ARG
    st, _ = fg.fg_server_poll(None)
    assert st == fg.FG_ERR_INVALID_ARG
    assert fg.fg_server_release(None, 1) == fg.FG_ERR_INVALID_ARG
    assert fg.fg_server_destroy(None) == fg.FG_OK
    st, _, _ = fg.fg_tune_opts(None, fg.FG_QUERY_SSSP, src, 4)
    assert st == fg.FG_ERR_INVALID_ARG
    st, _ = fg.fg_graph_info(None)
    assert st == fg.FG_ERR_INVALID_ARG
    assert fg.fg_graph_destroy(None) == fg.FG_OK


def test_bad_graph_opts(lib):
    g = _csr()
    for method, S in ((7, 0), (fg.FG_PART_GROW, 100), (fg.FG_PART_GROW, 16), (fg.FG_PART_GROW, 8192)):
        go = fg.fg_default_graph_opts(partition_method=method, partition_vertices=S)
        st, _ = fg.fg_graph_create_ex(g.n, g.m, g.row_ptr, g.col, g.w, 0, go)
        assert st == fg.FG_ERR_INVALID_ARG


def _cut(g, perm, S):
    part = np.empty(g.n, dtype=np.int64)
    part[perm] = np.arange(g.n) // S
    src = np.repeat(np.arange(g.n), np.diff(g.row_ptr))
    return int((part[src] != part[g.col]).sum())


@pytest.mark.parametrize("S", [64, 1024])
def test_partition_plan_is_a_permutation_with_compact_regions(lib, S):
    g = inputs.grid(256, 256, 500, 100, seed=4)
    perm = np.empty(g.n, dtype=np.int32)
    assert fg.fg_partition_plan(g.n, g.row_ptr, g.col, fg.FG_PART_GROW, S, perm) == fg.FG_OK
    assert np.array_equal(np.sort(perm), np.arange(g.n))
    for j in range(0, g.n, S):  # ascending original ids inside a partition
        assert np.all(np.diff(perm[j:j + S]) > 0)
    rng = np.empty(g.n, dtype=np.int32)
    assert fg.fg_partition_plan(g.n, g.row_ptr, g.col, fg.FG_PART_RANGE, S, rng) == fg.FG_OK
    assert np.array_equal(rng, np.arange(g.n))
    grow_cut, range_cut = _cut(g, perm, S), _cut(g, rng, S)
    assert grow_cut < 0.6 * range_cut, (grow_cut, range_cut)


def test_degree_plan_orders_by_degree_and_keeps_hub_arcs_inside(lib):
    g = inputs.rmat(12, 16, seed=3)
    S = 256
    perm = np.empty(g.n, dtype=np.int32)
    assert fg.fg_partition_plan(g.n, g.row_ptr, g.col, fg.FG_PART_DEGREE, S, perm) == fg.FG_OK
    assert np.array_equal(np.sort(perm), np.arange(g.n))
    deg = np.diff(g.row_ptr)[perm]
    assert np.all(np.diff(deg) <= 0)  # out-degree non-increasing along the internal order
    ties = np.flatnonzero(np.diff(deg) == 0)
    assert np.all(perm[ties] < perm[ties + 1])  # stable: equal degrees keep id order
    rng = np.arange(g.n, dtype=np.int32)
    assert _cut(g, perm, S) < _cut(g, rng, S)  # hubs sharing partitions keep some arcs inside
    assert fg.fg_partition_plan(g.n, None, None, fg.FG_PART_DEGREE, S, perm) == fg.FG_ERR_INVALID_ARG


def test_partition_plan_bad_args(lib):
    perm = np.empty(4, dtype=np.int32)
    assert fg.fg_partition_plan(4, None, None, fg.FG_PART_GROW, 2, perm) == fg.FG_ERR_INVALID_ARG
    assert fg.fg_partition_plan(4, None, None, 9, 2, perm) == fg.FG_ERR_INVALID_ARG


def test_application_entry_points_reject_bad_arguments_on_the_host(lib):
    """The NCP sweep, landmark labeling and BC entry points check their
    arguments before any CUDA call (so these run without a GPU)."""
    p = np.zeros(4, dtype=np.float32)
    cnt = np.zeros(1, dtype=np.int32)
    assert fg.fg_ncp_sweep(None, p, 1, 4, None, None, cnt) == fg.FG_ERR_INVALID_ARG
    lab = np.zeros(16, dtype=np.uint32)
    pairs = np.zeros(2, dtype=np.int32)
    est = np.zeros(1, dtype=np.uint64)
    assert fg.fg_ll_build_labels(None, 4, 4, lab) == fg.FG_ERR_INVALID_ARG
    assert fg.fg_ll_build_labels(lab, 0, 4, lab) == fg.FG_ERR_INVALID_ARG
    assert fg.fg_ll_build_labels(lab, 4, 0, lab) == fg.FG_ERR_INVALID_ARG
    assert fg.fg_ll_query(lab, 4, 4, pairs, -1, est) == fg.FG_ERR_INVALID_ARG
    assert fg.fg_ll_query(lab, 4, 0, pairs, 1, est) == fg.FG_ERR_INVALID_ARG
    assert fg.fg_ll_query(None, 4, 4, pairs, 1, est) == fg.FG_ERR_INVALID_ARG
    assert fg.fg_ll_query(lab, 4, 4, pairs, 0, est) == fg.FG_OK  # empty batch: nothing to launch
    src = np.zeros(1, dtype=np.int32)
    bc = np.zeros(4, dtype=np.float64)
    st, _ = fg.fg_bc_accumulate(None, src, 1, lab, True, bc)
    assert st == fg.FG_ERR_INVALID_ARG
    assert ctypes.sizeof(fg.fg_bc_info_t) == 16
    paths = np.zeros(8, dtype=np.int32)
    assert fg.fg_rw_batch(None, src, 1, 3, 0, paths) == fg.FG_ERR_INVALID_ARG
    assert fg.fg_dfs_batch(None, src, 1, paths) == fg.FG_ERR_INVALID_ARG
    pf = np.zeros(64, dtype=np.float32)
    assert fg.fg_ppr_local_batch(None, src, 1, 0.15, 1e-4, 64, paths, pf, cnt) == fg.FG_ERR_INVALID_ARG
