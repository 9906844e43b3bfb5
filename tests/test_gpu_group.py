"""The group engine (opts.group = 8, 16, 32: one lane per query, a group's values
of one vertex in one line) against the oracle, bit for bit, and against the
one-query-per-warp engine (opts.group = 1).

Covers partial groups (nq not a multiple of G), duplicate sources, hubs (vertices
with more than 4,096 arcs, relaxed in chunks spread over blocks) including a
hub source and hubs at exactly the chunk boundary, every partitioner, the
per-group value window, directed graphs, and query batches split across
launches.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_2103_14915_gb300 import fg, inputs

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
HUB = 4096


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2103_14915_gb300 import build
    build.build()
    fg.load()
    assert torch.cuda.is_available()


def hub_graph():
    """Three stars joined in a path (centres of 9,002, 4,099 and 4,096 arcs: a
    hub of three chunks, a hub of two, and the largest vertex that is not a
    hub), with shortcuts between the first two stars' leaves."""
    edges = []
    n = 0
    centres = []
    for leaves in (9001, 4097, 4095):
        c = n
        centres.append(c)
        for i in range(1, leaves + 1):
            edges.append((c, c + i, 1 + (i * 37) % 200))
        n += leaves + 1
    for a, b in zip(centres, centres[1:]):
        edges.append((a, b, 5))
    for i in range(1, 4000, 7):
        edges.append((i, centres[1] + 1 + (i * 13) % 4000, 3 + i % 50))
    return inputs.from_edges(n, edges, name="hubs")


def graphs():
    gs = [hub_graph(), inputs.rmat(11, 16, seed=2, weights=(1, 255)),
          inputs.rmat(10, 8, seed=3, directed=True, weights=(1, 255)),
          inputs.grid(30, 41, 500, 100, seed=3, weights=(100, 10000))]
    k5 = inputs.from_edges(5, [(u, v, 1 + u + v) for u in range(5) for v in range(u + 1, 5)], name="K5")
    gs.append(k5)
    return gs


GRAPHS = graphs()


def run(h, g, kind, srcs, **opts):
    srcs = np.ascontiguousarray(srcs, dtype=np.int32)
    s_d = torch.from_numpy(srcs).to(DEV)
    out = torch.empty((len(srcs), g.n), dtype=torch.int32, device=DEV)
    o = fg.fg_default_opts(**dict(dict(watchdog_ms=20000), **opts))
    f = fg.fg_sssp_batch if kind == "sssp" else fg.fg_bfs_batch
    fg.check(f(h, s_d, len(srcs), out, None, o))
    fg.check(fg.fg_sync())
    return out.cpu().numpy().view(np.uint32)


def create(g, method=fg.FG_PART_AUTO, S=0):
    st, h = fg.fg_graph_create_ex(g.n, g.m, g.row_ptr, g.col, g.w, 0,
                                  fg.fg_default_graph_opts(partition_method=method, partition_vertices=S))
    fg.check(st)
    return h


@pytest.mark.parametrize("gi", range(len(GRAPHS)), ids=[g.name or f"g{i}" for i, g in enumerate(GRAPHS)])
@pytest.mark.parametrize("G", [8, 16, 32, 64])
def test_group_engine_exact(gi, G):
    g = GRAPHS[gi]
    h = create(g, fg.FG_PART_RANGE, 64)
    try:
        for nq in (1, G - 1, 2 * G + 3):
            srcs = (np.arange(nq) * 7919 + 11) % g.n
            if nq > 2:
                srcs[1] = srcs[0]   # duplicate
                srcs[2] = 0         # the first hub's centre on the hub graph
            for kind in ("sssp", "bfs"):
                got = run(h, g, kind, srcs, group=G)
                ref = oracle.sssp(g, srcs) if kind == "sssp" else oracle.bfs(g, srcs)
                assert np.array_equal(got, ref), (g.name, kind, nq, G)
    finally:
        fg.fg_graph_destroy(h)


@pytest.mark.parametrize("method,S", [(fg.FG_PART_RANGE, 32), (fg.FG_PART_GROW, 128), (fg.FG_PART_DEGREE, 64),
                                      (fg.FG_PART_AUTO, 0)])
def test_group_engine_every_partitioner(method, S):
    g = inputs.rmat(12, 16, seed=9, weights=(1, 255))
    h = create(g, method, S)
    try:
        srcs = inputs.sources_uniform(g, 37, 4)
        for kind in ("sssp", "bfs"):
            ref = oracle.sssp(g, srcs) if kind == "sssp" else oracle.bfs(g, srcs)
            assert np.array_equal(run(h, g, kind, srcs, group=16), ref)
            assert np.array_equal(run(h, g, kind, srcs, group=1), ref)
    finally:
        fg.fg_graph_destroy(h)


@pytest.mark.parametrize("window", [1, 4, 64, 1000])
def test_group_engine_window_never_changes_results(window):
    g = inputs.rmat(11, 16, seed=6, weights=(1, 255))
    h = create(g, fg.FG_PART_RANGE, 128)
    try:
        srcs = inputs.sources_uniform(g, 40, 8)
        ref = oracle.sssp(g, srcs)
        got = run(h, g, "sssp", srcs, group=16, sched=fg.FG_SCHED_PRIORITY, sched_window=window)
        assert np.array_equal(got, ref)
        # BFS ignores the window (its rounds are levels)
        got = run(h, g, "bfs", srcs, group=16, sched=fg.FG_SCHED_PRIORITY, sched_window=window)
        assert np.array_equal(got, oracle.bfs(g, srcs))
    finally:
        fg.fg_graph_destroy(h)


def test_group_engine_split_batches_and_stats():
    g = inputs.rmat(10, 16, seed=12, weights=(1, 255))
    h = create(g, fg.FG_PART_RANGE, 64)
    try:
        srcs = inputs.sources_uniform(g, 50, 2)
        ref = oracle.sssp(g, srcs)
        got = run(h, g, "sssp", srcs, group=8, query_batch=16, group_order=1)  # four launches, the last partial
        assert np.array_equal(got, ref)
        st, s = fg.fg_stats(h)
        fg.check(st)
        assert s.launches == 8 and s.rounds > 0 and s.visits > 0
        got = run(h, g, "sssp", srcs, group=8, query_batch=16)  # the same after ordering (two more kernels)
        assert np.array_equal(got, ref)
        assert fg.fg_stats(h)[1].launches == 10
        # lane relaxations cover at least the arcs a sequential Dijkstra scans
        deg = np.diff(g.row_ptr)
        dijkstra_arcs = int(sum(deg[ref[q] != 0xFFFFFFFF].sum() for q in range(len(srcs))))
        assert s.edges >= dijkstra_arcs
    finally:
        fg.fg_graph_destroy(h)


def test_group_engine_bad_source_and_empty_graph():
    g = inputs.from_edges(40, [], name="empty")
    h = create(g, fg.FG_PART_RANGE, 32)
    try:
        srcs = np.array([0, 39, 17], dtype=np.int32)
        got = run(h, g, "sssp", srcs, group=8)
        assert np.array_equal(got, oracle.sssp(g, srcs))
        s_d = torch.tensor([3, 40], dtype=torch.int32, device=DEV)
        out = torch.empty((2, g.n), dtype=torch.int32, device=DEV)
        fg.check(fg.fg_bfs_batch(h, s_d, 2, out, None, fg.fg_default_opts(group=8)))
        assert fg.fg_sync() == fg.FG_ERR_INVALID_ARG
    finally:
        fg.fg_graph_destroy(h)


def test_group_option_is_checked_on_the_host():
    g = inputs.rmat(8, 8, seed=1, weights=(1, 255))
    h = create(g)
    try:
        s_d = torch.zeros(1, dtype=torch.int32, device=DEV)
        out = torch.empty((1, g.n), dtype=torch.int32, device=DEV)
        assert fg.fg_sssp_batch(h, s_d, 1, out, None, fg.fg_default_opts(group=12)) == fg.FG_ERR_INVALID_ARG
        # groups of 64 run FIFO rounds only
        o = fg.fg_default_opts(group=64, sched=fg.FG_SCHED_PRIORITY, sched_window=16)
        assert fg.fg_sssp_batch(h, s_d, 1, out, None, o) == fg.FG_ERR_UNSUPPORTED
    finally:
        fg.fg_graph_destroy(h)


@pytest.mark.parametrize("G", [8, 32, 64])
def test_group_order_keeps_rows(G):
    """Queries are regrouped by two-hop reach inside the library; every row still
    belongs to its own source, with duplicates, hubs, isolated vertices and
    launches split by query_batch, for both group orders."""
    g = inputs.rmat(11, 16, seed=13, weights=(1, 255))
    h = create(g, fg.FG_PART_RANGE, 64)
    try:
        deg = np.diff(g.row_ptr)
        srcs = inputs.sources_uniform(g, 3 * G + 5, 21).astype(np.int32)
        srcs[4] = srcs[9]                     # duplicate
        srcs[5] = int(np.argmax(deg))         # the largest hub
        if (deg == 0).any():
            srcs[6] = int(np.flatnonzero(deg == 0)[0])  # no arcs
        for kind in ("sssp", "bfs"):
            ref = oracle.sssp(g, srcs) if kind == "sssp" else oracle.bfs(g, srcs)
            for order in (0, 1):
                for qb in (0, G + 3):
                    got = run(h, g, kind, srcs, group=G, group_order=order, query_batch=qb)
                    assert np.array_equal(got, ref), (kind, order, qb)
        # an out-of-range source among reordered queries is still reported
        bad = srcs.copy()
        bad[7] = g.n
        s_d = torch.from_numpy(bad).to(DEV)
        out = torch.empty((len(bad), g.n), dtype=torch.int32, device=DEV)
        fg.check(fg.fg_sssp_batch(h, s_d, len(bad), out, None, fg.fg_default_opts(group=G)))
        assert fg.fg_sync() == fg.FG_ERR_INVALID_ARG
        assert fg.fg_sssp_batch(h, s_d, len(bad), out, None, fg.fg_default_opts(group=G, group_order=2)) \
            == fg.FG_ERR_INVALID_ARG
    finally:
        fg.fg_graph_destroy(h)


def test_staging_self_check_is_clean():
    """With check_staging every staged row-offset and pending-mask word is
    compared on the device with global memory right after its bulk-copy wait;
    no mismatch is reported on graphs with hubs, partitions of 32 to 1,024
    vertices and every group size, and the results stay exact."""
    cases = [(hub_graph(), fg.FG_PART_RANGE, 64), (inputs.rmat(12, 16, seed=9, weights=(1, 255)), fg.FG_PART_AUTO, 0),
             (inputs.rmat(10, 8, seed=3, directed=True, weights=(1, 255)), fg.FG_PART_GROW, 32),
             (inputs.grid(30, 41, 500, 100, seed=3, weights=(100, 10000)), fg.FG_PART_GROW, 128)]
    for g, method, S in cases:
        h = create(g, method, S)
        try:
            srcs = inputs.sources_uniform(g, 40, 5)
            for G in (8, 16, 32, 64):
                for kind in ("sssp", "bfs"):
                    got = run(h, g, kind, srcs, group=G, check_staging=1)
                    ref = oracle.sssp(g, srcs) if kind == "sssp" else oracle.bfs(g, srcs)
                    assert np.array_equal(got, ref), (g.name, G, kind)
        finally:
            fg.fg_graph_destroy(h)


def test_group_64_split_batches_and_hub_masks():
    """Groups of 64: 64-bit pending masks (query 2l + j at bit 32j + l), hub
    chunks whose lanes span both mask words, and a batch split into launches
    whose last group is partial."""
    g = hub_graph()
    h = create(g, fg.FG_PART_RANGE, 128)
    try:
        deg = np.diff(g.row_ptr)
        hubs = np.flatnonzero(deg > 512)
        srcs = inputs.sources_uniform(g, 150, 9).astype(np.int32)
        srcs[::7] = hubs[np.arange(len(srcs[::7])) % len(hubs)]  # hubs in both halves of several groups
        for kind in ("sssp", "bfs"):
            ref = oracle.sssp(g, srcs) if kind == "sssp" else oracle.bfs(g, srcs)
            for qb in (0, 70):
                got = run(h, g, kind, srcs, group=64, query_batch=qb)
                assert np.array_equal(got, ref), (kind, qb)
    finally:
        fg.fg_graph_destroy(h)
