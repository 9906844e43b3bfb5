"""Pins for the CPU oracle: each check ties it to something other than itself.

* SSSP / BFS: Floyd-Warshall (scipy, an independent algorithm and library) on
  graphs of <= 64 vertices, closed forms (path, cycle, full grid = Manhattan
  distance), and the implementation-free certificate.
* PPR power iteration: the dense solve pi = alpha (I - (1-alpha) P^T)^-1 e_s
  (numpy.linalg.solve) on <= 64 vertices, and closed forms for a single edge,
  a star and the complete graph K_n, plus sum(pi) = 1.
* FP64 push: the error bound 0 <= pi(t) - p(t) <= eps * d(t) on undirected
  graphs, mass conservation and the termination condition.
* Planted mistakes (oracle mutations 1..5) must each fail one of these pins.
"""
import numpy as np
import pytest
import scipy.sparse as sp
from scipy.sparse.csgraph import floyd_warshall

import oracle
from paper_2103_14915_gb300 import inputs as I

INF = np.uint32(0xFFFFFFFF)


def random_small_graph(n, p, seed, directed, weighted=True, isolated=2):
    rng = np.random.default_rng(seed)
    edges = []
    for u in range(n - isolated):
        for v in range(n - isolated):
            if u != v and (directed or u < v) and rng.random() < p:
                edges.append((u, v, int(rng.integers(1, 50))) if weighted else (u, v))
    if not edges:
        edges = [(0, 1, 1) if weighted else (0, 1)]
    return I.from_edges(n, edges, directed=directed, name=f"small{seed}")


def fw_matrix(g, unit=False):
    n = g.n
    rows = np.repeat(np.arange(n), np.diff(g.row_ptr))
    data = np.ones(g.m) if (unit or g.w is None) else g.w.astype(np.float64)
    a = sp.csr_matrix((data, (rows, g.col)), shape=(n, n))
    d = floyd_warshall(a, directed=True)
    out = np.full((n, n), INF, dtype=np.uint32)
    fin = np.isfinite(d)
    out[fin] = d[fin].astype(np.uint32)
    return out


GRAPHS = [(n, p, s, dr) for s, (n, p) in enumerate([(8, .4), (17, .2), (33, .1), (64, .06), (64, .12)])
          for dr in (False, True)]


@pytest.mark.parametrize("n,p,seed,directed", GRAPHS)
def test_sssp_matches_floyd_warshall(n, p, seed, directed):
    g = random_small_graph(n, p, seed, directed)
    srcs = np.arange(n, dtype=np.int32)
    assert np.array_equal(oracle.sssp(g, srcs), fw_matrix(g))


@pytest.mark.parametrize("n,p,seed,directed", GRAPHS)
def test_bfs_matches_unit_floyd_warshall(n, p, seed, directed):
    g = random_small_graph(n, p, seed + 100, directed, weighted=False)
    srcs = np.arange(n, dtype=np.int32)
    assert np.array_equal(oracle.bfs(g, srcs), fw_matrix(g, unit=True))


def test_closed_forms_path_and_cycle():
    n, w = 40, 7
    path = I.from_edges(n, [(i, i + 1, w) for i in range(n - 1)])
    cyc = I.from_edges(n, [(i, (i + 1) % n, w) for i in range(n)])
    for s in (0, 13, n - 1):
        idx = np.arange(n)
        assert np.array_equal(oracle.sssp(path, [s])[0], (w * np.abs(idx - s)).astype(np.uint32))
        ring = np.minimum(np.abs(idx - s), n - np.abs(idx - s))
        assert np.array_equal(oracle.sssp(cyc, [s])[0], (w * ring).astype(np.uint32))
        assert np.array_equal(oracle.bfs(cyc, [s])[0], ring.astype(np.uint32))


def test_closed_form_full_grid_manhattan():
    rows, cols, w = 48, 37, 5
    g = I.grid(rows, cols, drop_per_10000=0, diag_per_10000=0, seed=3)
    r, c = np.divmod(np.arange(rows * cols), cols)
    srcs = [0, cols * 20 + 11, rows * cols - 1]
    lv = oracle.bfs(g, srcs)
    g.w = np.full(g.m, w, dtype=np.int32)
    dd = oracle.sssp(g, srcs)
    for i, s in enumerate(srcs):
        sr, sc = divmod(s, cols)
        man = np.abs(r - sr) + np.abs(c - sc)
        assert np.array_equal(lv[i], man.astype(np.uint32))
        assert np.array_equal(dd[i], (w * man).astype(np.uint32))


def test_certificate_accepts_oracle_and_rejects_planted_errors():
    g = I.rmat(10, 8, seed=5, weights=(1, 255))
    srcs = I.sources_uniform(g, 8, 9)
    d = oracle.sssp(g, srcs)
    lv = oracle.bfs(g, srcs)
    assert oracle.certificate_batch(g, srcs, d, weighted=True) == 0
    assert oracle.certificate_batch(g, srcs, lv, weighted=False) == 0
    rng = np.random.default_rng(0)
    reach = np.flatnonzero((d[0] != INF) & (np.arange(g.n) != srcs[0]))
    for delta in (-1, +1, +1000):
        bad = d[0].copy()
        v = rng.choice(reach)
        bad[v] = np.uint32(int(bad[v]) + delta)
        assert oracle.sssp_certificate(g, int(srcs[0]), bad) != 0
    bad = d[0].copy()
    bad[reach[0]] = INF
    assert oracle.sssp_certificate(g, int(srcs[0]), bad) != 0
    bad = d[0].copy()
    bad[srcs[0]] = 1
    assert oracle.sssp_certificate(g, int(srcs[0]), bad) == 1
    bad = lv[1].copy()
    bad[np.flatnonzero(lv[1] == 2)[0]] = 1
    assert oracle.bfs_certificate(g, int(srcs[1]), bad) != 0


def dense_ppr(g, s, alpha):
    """pi = alpha (I - (1-alpha) P^T)^-1 e_s with P = D^-1 A and dangling rows = e_s^T."""
    n = g.n
    P = np.zeros((n, n))
    for v in range(n):
        nb = g.col[g.row_ptr[v]:g.row_ptr[v + 1]]
        if nb.size == 0:
            P[v, s] = 1.0
        else:
            P[v, nb] += 1.0 / nb.size
    e = np.zeros(n)
    e[s] = 1.0
    return alpha * np.linalg.solve(np.eye(n) - (1 - alpha) * P.T, e)


@pytest.mark.parametrize("n,p,seed,directed", GRAPHS)
def test_ppr_power_matches_dense_solve(n, p, seed, directed):
    g = random_small_graph(n, p, seed + 200, directed, weighted=False)
    srcs = np.arange(0, n, max(1, n // 8), dtype=np.int32)
    pi = oracle.ppr_power(g, srcs, 0.15, tol=1e-13)
    for i, s in enumerate(srcs):
        ref = dense_ppr(g, int(s), 0.15)
        assert np.max(np.abs(pi[i] - ref)) <= 1e-10
        assert abs(pi[i].sum() - 1.0) <= 1e-10


def test_ppr_closed_forms():
    a = 0.15
    edge = I.from_edges(2, [(0, 1)])
    pi = oracle.ppr_power(edge, [0], a, tol=1e-14)[0]
    assert np.allclose(pi, [1 / (2 - a), (1 - a) / (2 - a)], rtol=0, atol=1e-12)
    nl = 9
    star = I.from_edges(nl + 1, [(0, i) for i in range(1, nl + 1)])
    pi = oracle.ppr_power(star, [0], a, tol=1e-14)[0]
    assert abs(pi[0] - 1 / (2 - a)) < 1e-12
    assert np.allclose(pi[1:], (1 - a) / (nl * (2 - a)), rtol=0, atol=1e-12)
    for n in (3, 6, 11):
        kn = I.from_edges(n, [(u, v) for u in range(n) for v in range(u + 1, n)])
        pi = oracle.ppr_power(kn, [2], a, tol=1e-14)[0]
        ps = (a * (n - 1) + 1 - a) / (n - a)
        assert abs(pi[2] - ps) < 1e-12
        assert np.allclose(np.delete(pi, 2), (1 - ps) / (n - 1), rtol=0, atol=1e-12)


@pytest.mark.parametrize("eps", [1e-4, 1e-6])
def test_ppr_push_bound_and_mass(eps):
    g = I.rmat(11, 8, seed=21)
    srcs = I.sources_logdeg(g, 6, 3)
    pi = oracle.ppr_power(g, srcs, 0.15)
    deg = np.diff(g.row_ptr)
    for i, s in enumerate(srcs):
        p, r, k = oracle.ppr_push(g, int(s), 0.15, eps)
        assert k > 0
        assert abs(p.sum() + r.sum() - 1.0) <= 1e-12
        assert np.all(r < eps * np.maximum(deg, 1))
        diff = pi[i] - p
        assert np.all(diff >= -1e-12)
        assert np.all(diff <= eps * deg + 1e-12)


def test_ppr_directed_dangling_mass():
    g = I.rmat(9, 4, seed=4, directed=True)
    assert (np.diff(g.row_ptr) == 0).any()
    srcs = I.sources_uniform(g, 4, 1)
    pi = oracle.ppr_power(g, srcs, 0.15)
    for i, s in enumerate(srcs):
        assert abs(pi[i].sum() - 1.0) < 1e-10
        p, r, _ = oracle.ppr_push(g, int(s), 0.15, 1e-7)
        assert abs(p.sum() + r.sum() - 1.0) < 1e-12
        diff = pi[i] - p
        assert diff.min() >= -1e-12 and diff.max() <= r.sum() + 1e-12


def _pins_fail(kind):
    """Run the relevant pins; return True if any fails (used with a planted mistake)."""
    try:
        if kind == "sssp":
            for args in GRAPHS[:6]:
                test_sssp_matches_floyd_warshall(*args)
            test_closed_forms_path_and_cycle()
            test_closed_form_full_grid_manhattan()
        elif kind == "bfs":
            for args in GRAPHS[:6]:
                test_bfs_matches_unit_floyd_warshall(*args)
        elif kind == "ppr":
            for args in GRAPHS[:6]:
                test_ppr_power_matches_dense_solve(*args)
            test_ppr_closed_forms()
            test_ppr_directed_dangling_mass()
    except AssertionError:
        return True
    return False


@pytest.mark.parametrize("mutation,kind", [(1, "sssp"), (2, "sssp"), (3, "bfs"), (4, "ppr"), (5, "ppr")])
def test_planted_mistakes_are_caught(mutation, kind):
    assert not _pins_fail(kind)
    oracle.set_mutation(mutation)
    try:
        assert _pins_fail(kind), f"mutation {mutation} escaped the {kind} pins"
    finally:
        oracle.set_mutation(0)
    assert not _pins_fail(kind)
