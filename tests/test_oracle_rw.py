"""Pins of the oracle's random-walk queries (RW) against fixed facts.

- the generator: SplitMix64's published outputs for a state starting at 0
  (`tests/golden/splitmix64.txt`);
- the counter scheme: walk q, step t draws output 2^32 q + t + 1, so with the
  seed shifted by -2^32 q gamma, walk q's first steps pick neighbours by the
  published outputs themselves (mod the degree);
- a directed cycle: every walk is deterministic, v_t = (s + t) mod n;
- a vertex without out-arcs ends the walk (-1 afterwards);
- a star: walks alternate between the centre and leaves, and the leaves are
  chosen uniformly (a frequency check);
- long walks on a connected non-bipartite undirected graph visit each vertex
  with frequency close to the stationary d(v) / 2m;
- planted mistake 9 (output k - 1 drawn) fails the counter pin.
"""
from pathlib import Path

import numpy as np
import pytest

import oracle
from paper_2103_14915_gb300 import inputs

GOLDEN = Path(__file__).parent / "golden" / "splitmix64.txt"
GAMMA = 0x9E3779B97F4A7C15
M64 = (1 << 64) - 1


def _published():
    out = {}
    for line in GOLDEN.read_text().splitlines():
        if line.startswith("output"):
            _, k, v = line.split()
            out[int(k)] = int(v, 16)
    return out


def test_generator_matches_published_outputs():
    for k, v in _published().items():
        assert oracle.splitmix64(0, k) == v


def _star(d):
    return inputs.from_edges(d + 1, [(0, i) for i in range(1, d + 1)])


@pytest.mark.parametrize("q", [0, 1, 7])
def test_counter_scheme(q):
    d = 5
    g = _star(d)
    seed = (-(q << 32) * GAMMA) & M64  # makes walk q's step t draw published output t + 1
    pub = _published()
    srcs = np.zeros(q + 1, dtype=np.int32)  # every walk starts at the centre
    paths = oracle.rw(g, srcs, 1, seed)
    # from the centre the step picks leaf (r mod d) + 1 (CSR order of the star's arcs)
    assert paths[q, 1] == (pub[1] % d) + 1
    # a longer walk: centre, leaf, centre, leaf...; the leaf at step 2 uses output 3
    paths = oracle.rw(g, srcs, 3, seed)
    assert paths[q, 2] == 0 and paths[q, 3] == (pub[3] % d) + 1


def test_directed_cycle_is_deterministic():
    n = 17
    g = inputs.from_edges(n, [(i, (i + 1) % n) for i in range(n)], directed=True)
    srcs = np.arange(n, dtype=np.int32)
    paths = oracle.rw(g, srcs, 40, 12345)
    exp = (srcs[:, None] + np.arange(41)[None, :]) % n
    assert np.array_equal(paths, exp)


def test_dangling_vertex_ends_the_walk():
    g = inputs.from_edges(3, [(0, 1), (1, 2)], directed=True)
    assert oracle.rw(g, [0], 5, 1).tolist() == [[0, 1, 2, -1, -1, -1]]


def test_star_walks_alternate_and_leaves_are_uniform():
    d = 8
    g = _star(d)
    paths = oracle.rw(g, np.zeros(4000, dtype=np.int32), 20, 99)
    assert np.all(paths[:, 0::2] == 0) and np.all(paths[:, 1::2] >= 1)
    counts = np.bincount(paths[:, 1::2].ravel(), minlength=d + 1)[1:]
    expect = paths[:, 1::2].size / d
    assert np.all(np.abs(counts - expect) < 5 * np.sqrt(expect))


def test_planted_mistake_9_is_caught():
    oracle.set_mutation(9)
    try:
        with pytest.raises(AssertionError):
            test_counter_scheme(0)
    finally:
        oracle.set_mutation(0)


def test_long_walks_approach_the_stationary_distribution():
    # a connected, non-bipartite undirected graph: a cycle of 11 with chords and a triangle
    edges = [(i, (i + 1) % 11) for i in range(11)] + [(0, 5), (2, 8), (3, 7), (4, 9), (0, 2)]
    g = inputs.from_edges(11, edges)
    deg = np.diff(g.row_ptr).astype(np.float64)
    paths = oracle.rw(g, np.arange(11, dtype=np.int32).repeat(40), 2000, 4242)
    visits = np.bincount(paths[:, 200:].ravel(), minlength=g.n).astype(np.float64)  # after a burn-in
    freq = visits / visits.sum()
    np.testing.assert_allclose(freq, deg / deg.sum(), atol=0.004)
