"""Parity of sampled betweenness centrality (fg_bc_accumulate) with the oracle.

The oracle computes its own distances (Dijkstra / BFS), path counts and
Brandes dependencies; the GPU chain is fg_sssp_batch / fg_bfs_batch and then
fg_bc_accumulate. The kernel is also run on the oracle's own distance rows
(uploaded), so its input does not come from the CUDA path. While every path
count stays below 2^53 both sides perform the same FP64 operations in the same
order and agree bit for bit; past 2^53 (unweighted grids) the call reports
`inexact` and the results agree to rounding.
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


def _graph(g, method=fg.FG_PART_GROW, S=64):
    st, h = fg.fg_graph_create_ex(g.n, g.m, g.row_ptr, g.col, g.w, 0,
                                  fg.fg_default_graph_opts(partition_method=method, partition_vertices=S))
    fg.check(st)
    return h


def _gpu_bc(h, g, srcs, weighted, bc=None, rows=None):
    s_d = torch.from_numpy(np.asarray(srcs, dtype=np.int32)).to(DEV)
    nq = len(srcs)
    if rows is None:
        dist = torch.empty((nq, g.n), dtype=torch.int32, device=DEV)
        f = fg.fg_sssp_batch if weighted else fg.fg_bfs_batch
        fg.check(f(h, s_d, nq, dist, None, None))
    else:
        dist = torch.from_numpy(np.ascontiguousarray(rows).view(np.int32)).to(DEV)
    acc = bc is not None
    out = bc if acc else torch.empty(g.n, dtype=torch.float64, device=DEV)
    st, info = fg.fg_bc_accumulate(h, s_d, nq, dist, weighted, out, acc)
    fg.check(st)
    return out.cpu().numpy(), info


@pytest.mark.parametrize("method", [fg.FG_PART_RANGE, fg.FG_PART_GROW])
@pytest.mark.parametrize("weighted", [True, False])
def test_small_graphs_bit_exact(method, weighted):
    rng = np.random.default_rng(3 + weighted)
    graphs = [inputs.grid(12, 13, 300, 50, seed=70, weights=(1, 20)),
              inputs.rmat(10, 8, seed=71, weights=(1, 9)),
              inputs.rmat(9, 6, seed=72, directed=True, weights=(1, 30)),
              inputs.from_edges(40, [(i, i + 1, 1 + i % 3) for i in range(39)])]
    for g in graphs:
        h = _graph(g, method)
        try:
            srcs = rng.choice(g.n, size=min(g.n, 37), replace=False)
            got, info = _gpu_bc(h, g, srcs, weighted)
            ref, smax, exact = oracle.bc(g, srcs, weighted)
            assert exact and info.inexact == 0
            assert info.sigma_max == smax
            assert np.array_equal(got, ref)
            # the kernel on the oracle's own distance rows
            rows = oracle.sssp(g, srcs) if weighted else oracle.bfs(g, srcs)
            got2, _ = _gpu_bc(h, g, srcs, weighted, rows=rows)
            assert np.array_equal(got2, ref)
        finally:
            fg.fg_graph_destroy(h)


def test_accumulate_over_calls_duplicates_and_isolated_sources():
    g = inputs.rmat(10, 8, seed=73, weights=(1, 50))
    # an isolated vertex appended as a source
    rp = np.concatenate([g.row_ptr, [g.row_ptr[-1]]]).astype(np.int64)
    gg = inputs.Graph(n=g.n + 1, row_ptr=rp, col=g.col, w=g.w, directed=False, name="rmat+isolated")
    h = _graph(gg)
    try:
        srcs = np.array([5, 17, 5, gg.n - 1, 200, 301], dtype=np.int32)  # a duplicate and the isolated vertex
        whole, _ = _gpu_bc(h, gg, srcs, True)
        ref, _, exact = oracle.bc(gg, srcs, True)
        assert exact and np.array_equal(whole, ref)
        bc = torch.zeros(gg.n, dtype=torch.float64, device=DEV)
        _gpu_bc(h, gg, srcs[:2], True, bc=bc)
        _gpu_bc(h, gg, srcs[2:], True, bc=bc)
        assert np.array_equal(bc.cpu().numpy(), whole)  # same additions in the same order
    finally:
        fg.fg_graph_destroy(h)


def test_path_counts_past_2_53_are_reported():
    g = inputs.grid(40, 40, 0, 0, seed=1)  # unweighted lattice: path counts up to C(78, 39)
    h = _graph(g)
    try:
        srcs = np.array([0, 39, 1599, 820], dtype=np.int32)
        got, info = _gpu_bc(h, g, srcs, False)
        ref, smax, exact = oracle.bc(g, srcs, False)
        assert not exact and info.inexact == 1 and info.sigma_max > 2.0**53
        np.testing.assert_allclose(got, ref, rtol=1e-9)
        assert info.waves == 78 + 1
    finally:
        fg.fg_graph_destroy(h)


def test_bad_inputs():
    g = inputs.from_edges(5, [(0, 1, 0), (1, 2, 3), (2, 3, 1), (3, 4, 2)])
    h = _graph(g, fg.FG_PART_RANGE, 0)
    try:
        s_d = torch.tensor([0, 2], dtype=torch.int32, device=DEV)
        dist = torch.empty((2, g.n), dtype=torch.int32, device=DEV)
        fg.check(fg.fg_bfs_batch(h, s_d, 2, dist, None, None))
        bc = torch.empty(g.n, dtype=torch.float64, device=DEV)
        st, _ = fg.fg_bc_accumulate(h, s_d, 2, dist, True, bc)
        assert st == fg.FG_ERR_UNSUPPORTED  # a weight-0 arc
        st, info = fg.fg_bc_accumulate(h, s_d, 2, dist, False, bc)
        fg.check(st)
        ref, _, _ = oracle.bc(g, [0, 2], False)
        assert np.array_equal(bc.cpu().numpy(), ref)
        swapped = torch.flip(dist, dims=[0]).contiguous()  # rows that do not start at their sources
        st, _ = fg.fg_bc_accumulate(h, s_d, 2, swapped, False, bc)
        assert st == fg.FG_ERR_INVALID_ARG
        # the graph stays usable after a device-reported error
        st, _ = fg.fg_bc_accumulate(h, s_d, 2, dist, False, bc)
        fg.check(st)
        assert np.array_equal(bc.cpu().numpy(), ref)
    finally:
        fg.fg_graph_destroy(h)


@pytest.mark.slow
@pytest.mark.parametrize("name,weighted", [("grid1024_bfs_sssp", True), ("rmat22_ppr", False)])
def test_bc_application_full_size(name, weighted):
    """BC as the paper runs it: 100 random sources, SSSP on the weighted grid,
    BFS on the R-MAT scale-22 social stand-in; every vertex's centrality against
    the oracle."""
    g = inputs.workload_graph(name)
    h = _graph(g, fg.FG_PART_GROW if weighted else fg.FG_PART_AUTO, 0)
    try:
        srcs = inputs.sources_uniform(g, 100, seed=74)
        got, info = _gpu_bc(h, g, srcs, weighted)
        ref, smax, exact = oracle.bc(g, srcs, weighted)
        assert info.inexact == (0 if exact else 1)
        if exact:
            assert info.sigma_max == smax
            assert np.array_equal(got, ref)
        else:
            np.testing.assert_allclose(got, ref, rtol=1e-9)
    finally:
        fg.fg_graph_destroy(h)
