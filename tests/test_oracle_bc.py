"""Pins of the oracle's betweenness centrality (BC) against facts fixed by the
mathematics or by an independent library, not by the oracle itself.

BC (Sec. 1, 6.1) runs one SSSP (weighted graph) or BFS (unweighted graph) per
sampled source and accumulates Brandes' dependencies; the oracle returns
bc(v) = sum over the sources s != v of delta_s(v), delta_s(v) = sum over pairs
(s, t) of the share of shortest s-t paths through v. Pins:
- a path of n vertices, all sources: bc(i) = 2 i (n - 1 - i) (ordered pairs with
  i strictly inside), with unit or arbitrary positive weights (a tree);
- a star, all sources: the centre carries every ordered leaf pair;
- networkx's independent Brandes implementation on small random graphs
  (weighted, unweighted with many tied paths, directed, source subsets);
- unweighted, all sources: the centralities sum to the number of inner
  vertices over all ordered pairs' shortest paths, sum of (hops(s, t) - 1),
  hop counts from scipy;
- planted mistake 8 (the dependency without its "1 +") fails.
"""
import numpy as np
import pytest

import oracle
from paper_2103_14915_gb300 import inputs

nx = pytest.importorskip("networkx")


def _nx_graph(g, weighted):
    G = nx.DiGraph() if g.directed else nx.Graph()
    G.add_nodes_from(range(g.n))
    for u in range(g.n):
        for e in range(g.row_ptr[u], g.row_ptr[u + 1]):
            G.add_edge(u, int(g.col[e]), weight=int(g.w[e]) if (weighted and g.w is not None) else 1)
    return G


def _nx_bc(g, srcs, weighted):
    """Sum over s in srcs, t in V of the share of shortest s-t paths through v (networkx)."""
    G = _nx_graph(g, weighted)
    b = nx.betweenness_centrality_subset(G, sources=list(map(int, srcs)), targets=list(range(g.n)),
                                         normalized=False, weight="weight" if weighted else None)
    scale = 1.0 if g.directed else 2.0  # networkx halves undirected subset sums
    return np.array([b[v] * scale for v in range(g.n)])


@pytest.mark.parametrize("weighted", [False, True])
def test_path_closed_form(weighted):
    n = 31
    rng = np.random.default_rng(5)
    edges = [(i, i + 1, int(rng.integers(1, 100))) for i in range(n - 1)]
    g = inputs.from_edges(n, edges)
    b, smax, exact = oracle.bc(g, np.arange(n), weighted)
    assert exact and smax == 1.0  # a tree: one shortest path per pair
    assert np.array_equal(b, np.array([2.0 * i * (n - 1 - i) for i in range(n)]))


def test_star_closed_form():
    n = 25
    g = inputs.from_edges(n, [(0, i, 3) for i in range(1, n)])
    b, _, _ = oracle.bc(g, np.arange(n), True)
    assert b[0] == (n - 1) * (n - 2) and np.all(b[1:] == 0)


@pytest.mark.parametrize("weighted", [False, True])
def test_random_graphs_against_networkx(weighted):
    rng = np.random.default_rng(6 + weighted)
    for trial in range(5):
        g = inputs.rmat(7, 4, seed=200 + trial, weights=(1, 5))  # small weights: tied shortest paths too
        srcs = rng.choice(g.n, size=20, replace=False)
        b, smax, exact = oracle.bc(g, srcs, weighted)
        assert exact and smax >= 2.0  # some pairs have several shortest paths
        np.testing.assert_allclose(b, _nx_bc(g, srcs, weighted), rtol=1e-12, atol=1e-9)


def test_directed_graph_against_networkx():
    g = inputs.rmat(7, 6, seed=210, directed=True, weights=(1, 20))
    srcs = np.arange(0, g.n, 3)
    for weighted in (False, True):
        b, _, _ = oracle.bc(g, srcs, weighted)
        np.testing.assert_allclose(b, _nx_bc(g, srcs, weighted), rtol=1e-12, atol=1e-9)


def test_grid_with_many_tied_paths():
    # unweighted 6 x 7 grid: path counts are binomial coefficients
    g = inputs.grid(6, 7, 0, 0, seed=1)
    b, smax, exact = oracle.bc(g, np.arange(g.n), False)
    assert exact and smax == 462.0  # C(11, 5): corner to opposite corner
    np.testing.assert_allclose(b, _nx_bc(g, np.arange(g.n), False), rtol=1e-12)


def test_zero_weight_arcs_are_rejected():
    g = inputs.from_edges(3, [(0, 1, 0), (1, 2, 4)])
    with pytest.raises(ValueError):
        oracle.bc(g, [0], True)
    b, _, _ = oracle.bc(g, [0], False)  # as BFS the weights are ignored
    assert b[1] == 1.0


def test_planted_mistake_8_is_caught():
    n = 9
    g = inputs.from_edges(n, [(i, i + 1) for i in range(n - 1)])
    oracle.set_mutation(8)
    try:
        b, _, _ = oracle.bc(g, np.arange(n), False)
    finally:
        oracle.set_mutation(0)
    assert not np.array_equal(b, np.array([2.0 * i * (n - 1 - i) for i in range(n)]))


def test_total_centrality_counts_inner_vertices():
    sp = pytest.importorskip("scipy.sparse")
    csg = pytest.importorskip("scipy.sparse.csgraph")
    for trial in range(4):
        g = inputs.rmat(7, 3, seed=220 + trial)
        m = sp.csr_matrix((np.ones(g.m), g.col, g.row_ptr), shape=(g.n, g.n))
        hops = csg.shortest_path(m, unweighted=True, directed=True)
        reach = np.isfinite(hops) & (hops > 0)
        b, _, exact = oracle.bc(g, np.arange(g.n), False)
        assert exact
        np.testing.assert_allclose(b.sum(), (hops[reach] - 1).sum(), rtol=1e-12)
