"""Random-walk queries (fg_rw_batch) against the oracle's walks, bit for bit.

Both sides draw the same counter-based SplitMix64 outputs from their own code
(written from the generator's published definition), so every walk must be
identical. Cases: identity and relabelled vertex orders, a directed graph with
dangling vertices (walks that end early), length 0, lengths around the 32-entry
staging chunk, repeated sources, seeds near 2^64, walk indices past 2^16, and
source ids outside the graph (rows of -1).
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


def _walks(h, srcs, length, seed):
    s_d = torch.from_numpy(np.asarray(srcs, dtype=np.int32)).to(DEV)
    out = torch.empty((len(srcs), length + 1), dtype=torch.int32, device=DEV)
    fg.check(fg.fg_rw_batch(h, s_d, len(srcs), length, seed, out))
    fg.check(fg.fg_sync())
    return out.cpu().numpy()


@pytest.mark.parametrize("method", [fg.FG_PART_RANGE, fg.FG_PART_GROW])
@pytest.mark.parametrize("length", [0, 1, 31, 32, 33, 80])
def test_walks_match_the_oracle(method, length):
    g = inputs.rmat(11, 8, seed=80)
    st, h = fg.fg_graph_create_ex(g.n, g.m, g.row_ptr, g.col, g.w, 0,
                                  fg.fg_default_graph_opts(partition_method=method, partition_vertices=64))
    fg.check(st)
    try:
        rng = np.random.default_rng(length)
        srcs = rng.integers(0, g.n, size=1000).astype(np.int32)
        srcs[:10] = srcs[0]  # the same source, different walks
        for seed in (0, 12345, (1 << 64) - 7):
            assert np.array_equal(_walks(h, srcs, length, seed), oracle.rw(g, srcs, length, seed))
    finally:
        fg.fg_graph_destroy(h)


def test_directed_graph_with_dangling_vertices_and_many_walks():
    g = inputs.rmat(10, 4, seed=81, directed=True)
    st, h = fg.fg_graph_create_ex(g.n, g.m, g.row_ptr, g.col, g.w, 0, fg.fg_default_graph_opts())
    fg.check(st)
    try:
        srcs = np.random.default_rng(82).integers(0, g.n, size=70000).astype(np.int32)  # walk ids past 2^16
        got = _walks(h, srcs, 20, 777)
        ref = oracle.rw(g, srcs, 20, 777)
        assert np.array_equal(got, ref)
        assert (ref == -1).any()  # some walks ended at a dangling vertex
    finally:
        fg.fg_graph_destroy(h)


def test_sources_outside_the_graph_give_rows_of_minus_one():
    g = inputs.grid(10, 10, 0, 0, seed=1)
    st, h = fg.fg_graph_create_ex(g.n, g.m, g.row_ptr, g.col, g.w, 0, fg.fg_default_graph_opts())
    fg.check(st)
    try:
        got = _walks(h, [5, -1, g.n, 7], 6, 3)
        assert np.all(got[1] == -1) and np.all(got[2] == -1)
        ref = oracle.rw(g, [5, 0, 0, 7], 6, 3)  # walk indices 0 and 3 as in the GPU call
        assert np.array_equal(got[0], ref[0]) and np.array_equal(got[3], ref[3])
    finally:
        fg.fg_graph_destroy(h)
