"""Pins of the oracle's landmark-labeling (LL) query against facts fixed by the
mathematics, not by the oracle itself.

LL (Sec. 1, 6.1) runs a batch of SSSPs from landmark vertices; the labels of v
are its distances from the landmarks, and the distance estimate of (u, v) is
min over landmarks s reaching both of d(s, u) + d(s, v). Pins:
- a path graph with landmarks at both ends: the estimate has a closed form;
- a landmark on every shortest path (the centre of a star, the root of a tree
  whose pairs lie in different subtrees) makes the estimate exact;
- for every graph: exact when u is a landmark, never below the true distance
  (true distances from scipy's independent shortest-path routine);
- landmarks that reach neither end give "no estimate" (UINT64_MAX);
- sums beyond 2^32 are exact;
- planted mistake 7 (the unreachable sentinel taken as a distance) fails.
"""
import numpy as np
import pytest

import oracle
from paper_2103_14915_gb300 import inputs

scipy_sp = pytest.importorskip("scipy.sparse")
csgraph = pytest.importorskip("scipy.sparse.csgraph")

U64 = np.iinfo(np.uint64).max
INF32 = np.uint32(0xFFFFFFFF)


def _labels_from_truth(g, landmarks):
    """Labels built from scipy's Dijkstra (independent of the oracle's SSSP)."""
    rp, col, w = g.row_ptr, g.col, g.w if g.w is not None else np.ones(g.m, dtype=np.int32)
    a = scipy_sp.csr_matrix((w.astype(np.float64), col, rp), shape=(g.n, g.n))
    d = csgraph.dijkstra(a, directed=True, indices=np.asarray(landmarks))
    lab = np.where(np.isinf(d), float(INF32), d).astype(np.uint64).astype(np.uint32)
    return np.ascontiguousarray(lab.T), a


def _truth(a, pairs):
    d = csgraph.dijkstra(a, directed=True, indices=pairs[:, 0])
    return d[np.arange(len(pairs)), pairs[:, 1]]


def test_path_graph_closed_form():
    n = 57
    g = inputs.from_edges(n, [(i, i + 1) for i in range(n - 1)])
    rows = oracle.sssp(g, [0, n - 1])  # the oracle's own SSSP rows, as the application uses them
    lab = oracle.ll_labels(rows)
    u, v = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    pairs = np.stack([u.ravel(), v.ravel()], axis=1).astype(np.int32)
    got = oracle.ll_query(lab, pairs)
    exp = np.minimum(u + v, 2 * (n - 1) - u - v).ravel().astype(np.uint64)
    assert np.array_equal(got, exp)


def test_landmark_on_every_shortest_path_gives_exact_distances():
    # star: centre 0, leaves 1..40 with weights; every leaf-leaf path passes the centre
    rng = np.random.default_rng(3)
    n = 41
    g = inputs.from_edges(n, [(0, i, int(rng.integers(1, 100))) for i in range(1, n)])
    lab, a = _labels_from_truth(g, [0])
    pairs = rng.integers(0, n, size=(300, 2)).astype(np.int32)
    pairs = pairs[pairs[:, 0] != pairs[:, 1]]  # u = v: the empty path does not pass the centre
    assert np.array_equal(oracle.ll_query(lab, pairs), _truth(a, pairs).astype(np.uint64))


def test_random_graphs_landmark_exact_and_upper_bound():
    rng = np.random.default_rng(4)
    for trial in range(6):
        g = inputs.rmat(8, 4, seed=100 + trial, weights=(1, 50))
        lms = rng.choice(g.n, size=12, replace=False)
        lab, a = _labels_from_truth(g, lms)
        pairs = rng.integers(0, g.n, size=(2000, 2)).astype(np.int32)
        pairs[:200, 0] = rng.choice(lms, size=200)  # u is a landmark
        est = oracle.ll_query(lab, pairs)
        true = _truth(a, pairs)
        reach = np.isfinite(true)
        # exact where u is a landmark (the landmark's own label is 0)
        assert np.array_equal(est[:200][reach[:200]], true[:200][reach[:200]].astype(np.uint64))
        # an upper bound everywhere it exists (undirected: d(u,v) <= d(s,u) + d(s,v))
        has = est != U64
        assert np.all(est[has].astype(np.float64) >= true[has])
        assert np.any(est[has].astype(np.float64) > true[has])  # and not exact in general


def test_unreachable_landmarks_give_no_estimate():
    # two components: landmarks only in the first
    edges = [(i, i + 1, 2) for i in range(9)] + [(10 + i, 11 + i, 3) for i in range(9)]
    g = inputs.from_edges(20, edges)
    lab, _ = _labels_from_truth(g, [0, 4])
    pairs = np.array([[12, 15], [3, 14], [1, 8], [19, 19]], dtype=np.int32)
    got = oracle.ll_query(lab, pairs)
    assert got[0] == U64 and got[1] == U64 and got[3] == U64
    assert got[2] == 14  # via landmark 0: 2 + 16; via landmark 4: 6 + 8


def test_sums_beyond_32_bits_are_exact():
    big = np.uint32(0xFFFFFFFE)
    lab = np.array([[big, 7], [big, INF32], [1, big]], dtype=np.uint32)
    got = oracle.ll_query(lab, np.array([[0, 1], [0, 2], [1, 2]], dtype=np.int32))
    assert got[0] == 2 * int(big) and got[1] == min(int(big) + 1, 7 + int(big)) and got[2] == int(big) + 1


def test_planted_mistake_7_is_caught():
    edges = [(i, i + 1, 2) for i in range(9)] + [(10 + i, 11 + i, 3) for i in range(9)]
    g = inputs.from_edges(20, edges)
    lab, _ = _labels_from_truth(g, [0, 4])
    pairs = np.array([[12, 15]], dtype=np.int32)
    oracle.set_mutation(7)
    try:
        got = oracle.ll_query(lab, pairs)
    finally:
        oracle.set_mutation(0)
    assert got[0] != U64  # the mistake turns "no estimate" into a finite number
