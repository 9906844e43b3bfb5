"""Degenerate inputs of the method on the GPU path: a single vertex, a graph without arcs, isolated
sources, zero weights, an empty batch, and distances that overflow 32 bits."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_2103_14915_gb300 import fg, inputs

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
INF = np.uint32(0xFFFFFFFF)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2103_14915_gb300 import build
    build.build()
    fg.load()
    assert torch.cuda.is_available()


def _create(g):
    st, h = fg.fg_graph_create_ex(g.n, g.m, g.row_ptr, g.col, g.w, 0, fg.fg_default_graph_opts())
    fg.check(st)
    return h


def _run(h, g, kind, srcs, **opts):
    s_d = torch.tensor(np.asarray(srcs, dtype=np.int32), device=DEV)
    out = torch.empty((len(srcs), g.n), dtype=torch.int32, device=DEV)
    f = fg.fg_sssp_batch if kind == "sssp" else fg.fg_bfs_batch
    fg.check(f(h, s_d, len(srcs), out, None, fg.fg_default_opts(watchdog_ms=10000, **opts)))
    st = fg.fg_sync()
    return st, out.cpu().numpy().view(np.uint32)


@pytest.mark.parametrize("mode", [fg.FG_MODE_BUFFERED, fg.FG_MODE_PLAIN])
def test_single_vertex(mode):
    g = inputs.from_edges(1, [])
    h = _create(g)
    try:
        for kind in ("sssp", "bfs"):
            st, out = _run(h, g, kind, [0, 0], mode=mode)
            assert st == fg.FG_OK and out.tolist() == [[0], [0]]
        s_d = torch.zeros(1, dtype=torch.int32, device=DEV)
        p = torch.empty((1, 1), dtype=torch.float32, device=DEV)
        r = torch.empty_like(p)
        mass = torch.empty(1, dtype=torch.float64, device=DEV)
        fg.check(fg.fg_ppr_batch(h, s_d, 1, 0.15, 1e-4, p, r, mass, None, fg.fg_default_opts(mode=mode)))
        fg.check(fg.fg_sync())
        # a dangling source keeps returning (1 - alpha) of its residual to itself: p -> 1
        assert abs(float(mass[0]) - 1.0) <= 1e-6 and abs(float(p[0, 0]) + float(r[0, 0]) - 1.0) <= 1e-6
        assert float(r[0, 0]) < 1e-4
    finally:
        fg.fg_graph_destroy(h)


def test_graph_without_arcs():
    g = inputs.from_edges(300, [])
    h = _create(g)
    try:
        srcs = [0, 299, 150]
        for kind in ("sssp", "bfs"):
            st, out = _run(h, g, kind, srcs)
            assert st == fg.FG_OK
            exp = np.full((3, 300), INF, dtype=np.uint32)
            for i, s in enumerate(srcs):
                exp[i, s] = 0
            assert np.array_equal(out, exp)
    finally:
        fg.fg_graph_destroy(h)


def test_isolated_source_in_a_graph_with_arcs():
    g = inputs.grid(20, 20, 0, 0, seed=1, weights=(1, 9))
    # append two isolated vertices
    rp = np.concatenate([g.row_ptr, [g.row_ptr[-1], g.row_ptr[-1]]]).astype(np.int64)
    st, h = fg.fg_graph_create_ex(g.n + 2, g.m, rp, g.col, g.w, 0, fg.fg_default_graph_opts())
    fg.check(st)
    try:
        n = g.n + 2
        gg = inputs.Graph(n=n, row_ptr=rp, col=g.col, w=g.w, directed=False, name="grid+isolated")
        srcs = [n - 1, 0, n - 2]
        for kind in ("sssp", "bfs"):
            st, out = _run(h, gg, kind, srcs)
            assert st == fg.FG_OK
            ref = oracle.sssp(gg, srcs) if kind == "sssp" else oracle.bfs(gg, srcs)
            assert np.array_equal(out, ref)
    finally:
        fg.fg_graph_destroy(h)


def test_zero_weights():
    # a weighted cycle with some zero-weight edges, plus chords
    n = 64
    edges = [(i, (i + 1) % n, 0 if i % 3 == 0 else 5) for i in range(n)] + [(i, (i + 17) % n, 7) for i in range(0, n, 5)]
    g = inputs.from_edges(n, edges)
    h = _create(g)
    try:
        srcs = [0, 13, 63]
        st, out = _run(h, g, "sssp", srcs)
        assert st == fg.FG_OK and np.array_equal(out, oracle.sssp(g, srcs))
    finally:
        fg.fg_graph_destroy(h)


def test_empty_batch_is_rejected_on_the_host():
    g = inputs.grid(8, 8, 0, 0, seed=1)
    h = _create(g)
    try:
        s_d = torch.zeros(1, dtype=torch.int32, device=DEV)
        out = torch.empty((1, g.n), dtype=torch.int32, device=DEV)
        assert fg.fg_sssp_batch(h, s_d, 0, out, None, None) == fg.FG_ERR_INVALID_ARG
        assert fg.fg_bfs_batch(h, s_d, -1, out, None, None) == fg.FG_ERR_INVALID_ARG
    finally:
        fg.fg_graph_destroy(h)


@pytest.mark.parametrize("mode", [fg.FG_MODE_BUFFERED, fg.FG_MODE_PLAIN])
def test_distance_overflow_is_reported(mode):
    # a path whose length passes 2^32 - 1: the sum saturates and the batch reports FG_ERR_OVERFLOW
    big = 2**31 - 1
    g = inputs.from_edges(4, [(0, 1, big), (1, 2, big), (2, 3, big)])
    h = _create(g)
    try:
        st, out = _run(h, g, "sssp", [0], mode=mode)
        assert st == fg.FG_ERR_OVERFLOW
        assert out[0, 0] == 0 and out[0, 1] == big and out[0, 2] == 2 * big
    finally:
        fg.fg_graph_destroy(h)
