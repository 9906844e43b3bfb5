"""DFS queries (fg_dfs_batch) against the oracle's DFS, bit for bit.

The discovery order is unique once the neighbour order is fixed (the graph's
arc order), so every rank must match. Cases: identity and relabelled vertex
orders, undirected and directed graphs (unreached vertices), a path and a long
cycle (stack depth n - 1), hubs with hundreds of arcs (the 32-arc scan), a
single vertex, repeated sources, and a source outside the graph.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_2103_14915_gb300 import fg, inputs

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2103_14915_gb300 import build
    build.build()
    fg.load()
    assert torch.cuda.is_available()


def _dfs(h, g, srcs):
    s_d = torch.from_numpy(np.asarray(srcs, dtype=np.int32)).to(DEV)
    out = torch.empty((len(srcs), g.n), dtype=torch.int32, device=DEV)
    st = fg.fg_dfs_batch(h, s_d, len(srcs), out)
    return st, out.cpu().numpy().view(np.uint32)


@pytest.mark.parametrize("method", [fg.FG_PART_RANGE, fg.FG_PART_GROW])
def test_graphs_match_the_oracle(method):
    graphs = [inputs.grid(30, 40, 300, 50, seed=90),
              inputs.rmat(11, 8, seed=91),                       # hubs
              inputs.rmat(10, 4, seed=92, directed=True),        # unreached vertices
              inputs.from_edges(500, [(i, i + 1) for i in range(499)]),
              inputs.from_edges(700, [(i, (i + 1) % 700) for i in range(700)], directed=True)]
    rng = np.random.default_rng(93)
    for g in graphs:
        st, h = fg.fg_graph_create_ex(g.n, g.m, g.row_ptr, g.col, g.w, 0,
                                      fg.fg_default_graph_opts(partition_method=method, partition_vertices=64))
        fg.check(st)
        try:
            srcs = rng.integers(0, g.n, size=40).astype(np.int32)
            srcs[:3] = srcs[0]
            st, got = _dfs(h, g, srcs)
            fg.check(st)
            assert np.array_equal(got, oracle.dfs(g, srcs))
        finally:
            fg.fg_graph_destroy(h)


def test_single_vertex_and_bad_source():
    g = inputs.from_edges(1, [])
    st, h = fg.fg_graph_create_ex(g.n, g.m, g.row_ptr, g.col, g.w, 0, fg.fg_default_graph_opts())
    fg.check(st)
    try:
        st, got = _dfs(h, g, [0, 0])
        fg.check(st)
        assert got.tolist() == [[0], [0]]
        st, got = _dfs(h, g, [0, 3])
        assert st == fg.FG_ERR_INVALID_ARG and got[0, 0] == 0 and got[1, 0] == 0xFFFFFFFF
    finally:
        fg.fg_graph_destroy(h)
