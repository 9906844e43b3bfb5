"""Schedule autotuner (fg_tune_opts): picks a schedule at least as fast as the default, and the
schedule it picks computes the same exact distances."""
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


@pytest.mark.parametrize("make,method,S", [
    (lambda: inputs.grid(96, 96, 500, 100, seed=7, weights=(100, 10000)), fg.FG_PART_GROW, 256),
    (lambda: inputs.rmat(12, 16, seed=9, weights=(1, 255)), fg.FG_PART_RANGE, 256),
], ids=["grid", "rmat"])
@pytest.mark.parametrize("kind", [fg.FG_QUERY_SSSP, fg.FG_QUERY_BFS])
def test_tuned_schedule_is_exact_and_not_slower(make, method, S, kind):
    g = make()
    go = fg.fg_default_graph_opts(partition_method=method, partition_vertices=S)
    st, h = fg.fg_graph_create_ex(g.n, g.m, g.row_ptr, g.col, g.w, 0, go)
    fg.check(st)
    try:
        srcs = inputs.sources_uniform(g, 64, seed=3)
        s_d = torch.from_numpy(srcs).to(DEV)
        st, best, rep = fg.fg_tune_opts(h, kind, s_d, len(srcs))
        fg.check(st)
        assert rep.candidates >= 2 and rep.best_ms <= rep.default_ms
        assert best.struct_size == fg.fg_default_opts().struct_size
        st, again, rep2 = fg.fg_tune_opts(h, kind, s_d, len(srcs) - 1)  # same power-of-two bucket
        fg.check(st)
        assert rep2.candidates == 0 and bytes(again) == bytes(best)
        out = torch.empty((len(srcs), g.n), dtype=torch.int32, device=DEV)
        f = fg.fg_sssp_batch if kind == fg.FG_QUERY_SSSP else fg.fg_bfs_batch
        fg.check(f(h, s_d, len(srcs), out, None, best))
        fg.check(fg.fg_sync())
        rows = [0, 63]
        ref = oracle.sssp(g, srcs[rows]) if kind == fg.FG_QUERY_SSSP else oracle.bfs(g, srcs[rows])
        assert np.array_equal(out.cpu().numpy().view(np.uint32)[rows], ref)
    finally:
        fg.fg_graph_destroy(h)


def test_ppr_keeps_the_default_schedule():
    g = inputs.rmat(10, 8, seed=4)
    st, h = fg.fg_graph_create_ex(g.n, g.m, g.row_ptr, g.col, g.w, 0, fg.fg_default_graph_opts())
    fg.check(st)
    try:
        s_d = torch.from_numpy(inputs.sources_uniform(g, 16, seed=5)).to(DEV)
        st, best, rep = fg.fg_tune_opts(h, fg.FG_QUERY_PPR, s_d, 16)
        fg.check(st)
        assert rep.candidates == 1 and best.sched == fg.FG_SCHED_FIFO and best.sched_window == 0
    finally:
        fg.fg_graph_destroy(h)


def test_tuner_resolves_the_group_and_keeps_results_exact():
    """The tuner's group, window and batch-split choices change the work, not the distances."""
    g = inputs.rmat(12, 16, seed=13, weights=(1, 255))
    st, h = fg.fg_graph_create_ex(g.n, g.m, g.row_ptr, g.col, g.w, 0, fg.fg_default_graph_opts())
    fg.check(st)
    try:
        srcs = inputs.sources_uniform(g, 96, seed=8)
        s_d = torch.from_numpy(srcs).to(DEV)
        st, best, rep = fg.fg_tune_opts(h, fg.FG_QUERY_SSSP, s_d, len(srcs))
        fg.check(st)
        assert best.group in (1, 16, 32, 64)
        assert rep.candidates >= 4  # default, two other groups, and half the batch at least
        out = torch.empty((len(srcs), g.n), dtype=torch.int32, device=DEV)
        fg.check(fg.fg_sssp_batch(h, s_d, len(srcs), out, None, best))
        fg.check(fg.fg_sync())
        assert np.array_equal(out.cpu().numpy().view(np.uint32)[[0, 95]], oracle.sssp(g, srcs[[0, 95]]))
        _, stats = fg.fg_stats(h)
        assert stats.group == best.group
    finally:
        fg.fg_graph_destroy(h)


def test_ppr_tuning_takes_the_callers_alpha_and_eps():
    g = inputs.rmat(10, 8, seed=4)
    st, h = fg.fg_graph_create_ex(g.n, g.m, g.row_ptr, g.col, g.w, 0, fg.fg_default_graph_opts())
    fg.check(st)
    try:
        s_d = torch.from_numpy(inputs.sources_uniform(g, 16, seed=5)).to(DEV)
        st, a, ra = fg.fg_tune_opts_ex(h, fg.FG_QUERY_PPR, s_d, 16, 0.15, 1e-7)
        fg.check(st)
        assert ra.candidates == 1
        # another (alpha, eps) is timed again, not served from the cache of the first
        st, b, rb = fg.fg_tune_opts_ex(h, fg.FG_QUERY_PPR, s_d, 16, 0.2, 1e-5)
        fg.check(st)
        assert rb.candidates == 1
        st, c, rc = fg.fg_tune_opts_ex(h, fg.FG_QUERY_PPR, s_d, 16, 0.15, 1e-7)
        fg.check(st)
        assert rc.candidates == 0  # cached
        assert fg.fg_tune_opts_ex(h, fg.FG_QUERY_PPR, s_d, 16, 1.5, 1e-7)[0] == fg.FG_ERR_INVALID_ARG
    finally:
        fg.fg_graph_destroy(h)
