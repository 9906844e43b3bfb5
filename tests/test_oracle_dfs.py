"""Pins of the oracle's DFS against closed forms and an independent library.

DFS (a query type of the framework, Sec. 3) is read as recursive preorder from
the source with out-neighbours in the order the graph lists them; disc[v] is
the rank at which v is discovered. Pins:
- an undirected path, from an inner vertex k: the walk goes down to 0 first
  (the smaller neighbour is listed first), then up: disc[k - j] = j and
  disc[k + j] = k + j;
- a complete binary tree from the root: the classic preorder numbering;
- networkx's DFS preorder (graphs built with each vertex's neighbours in CSR
  order) on random directed and undirected graphs, unreached vertices
  included;
- planted mistake 10 (neighbours scanned from the last arc) fails.
"""
import numpy as np
import pytest

import oracle
from paper_2103_14915_gb300 import inputs

nx = pytest.importorskip("networkx")
UNREACHED = np.uint32(0xFFFFFFFF)


def test_path_from_an_inner_vertex():
    n, k = 21, 8
    g = inputs.from_edges(n, [(i, i + 1) for i in range(n - 1)])
    d = oracle.dfs(g, [k])[0]
    exp = np.empty(n, dtype=np.uint32)
    for j in range(k + 1):
        exp[k - j] = j
    for j in range(1, n - k):
        exp[k + j] = k + j
    assert np.array_equal(d, exp)


def _preorder_binary(depth):
    """Preorder ranks of a complete binary tree in heap numbering (children 2i+1, 2i+2)."""
    n = (1 << (depth + 1)) - 1
    rank = np.empty(n, dtype=np.uint32)
    nxt = 0

    def visit(i):
        nonlocal nxt
        rank[i] = nxt
        nxt += 1
        for c in (2 * i + 1, 2 * i + 2):
            if c < n:
                visit(c)
    visit(0)
    return rank


def test_complete_binary_tree_preorder():
    depth = 7
    n = (1 << (depth + 1)) - 1
    g = inputs.from_edges(n, [(i, c) for i in range(n) for c in (2 * i + 1, 2 * i + 2) if c < n])
    assert np.array_equal(oracle.dfs(g, [0])[0], _preorder_binary(depth))


@pytest.mark.parametrize("directed", [False, True])
def test_random_graphs_against_networkx(directed):
    for trial in range(5):
        g = inputs.rmat(8, 3, seed=300 + trial, directed=directed)
        G = nx.DiGraph() if directed else nx.Graph()
        G.add_nodes_from(range(g.n))
        for u in range(g.n):  # each vertex's neighbours in CSR order
            for e in range(g.row_ptr[u], g.row_ptr[u + 1]):
                G.add_edge(u, int(g.col[e]))
        srcs = np.random.default_rng(trial).choice(g.n, size=8, replace=False)
        got = oracle.dfs(g, srcs)
        for i, s in enumerate(srcs):
            exp = np.full(g.n, UNREACHED, dtype=np.uint32)
            for r, v in enumerate(nx.dfs_preorder_nodes(G, int(s))):
                exp[v] = r
            assert np.array_equal(got[i], exp)


def test_planted_mistake_10_is_caught():
    oracle.set_mutation(10)
    try:
        with pytest.raises(AssertionError):
            test_path_from_an_inner_vertex()
    finally:
        oracle.set_mutation(0)
