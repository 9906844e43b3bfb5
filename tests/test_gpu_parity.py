"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

SSSP distances and BFS levels must be bit-exact. PPR must satisfy, per vertex,
|p(t) - pi(t)| <= eps * deg(t) + 1e-6 against the FP64 power-iteration oracle on
undirected graphs (the residual bound at termination, r(v) < eps * d(v)), and
mass |sum p + sum r - 1| <= 1e-5.
"""
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


class DevGraph:
    def __init__(self, g, method=fg.FG_PART_AUTO, S=0):
        self.g = g
        go = fg.fg_default_graph_opts(partition_method=method, partition_vertices=S)
        st, self.h = fg.fg_graph_create_ex(g.n, g.m, g.row_ptr, g.col, g.w, 0, go)
        fg.check(st)

    def close(self):
        fg.fg_graph_destroy(self.h)

    def info(self):
        st, info = fg.fg_graph_info(self.h)
        fg.check(st)
        return info

    def run(self, kind, srcs, **opts):
        srcs = np.ascontiguousarray(srcs, dtype=np.int32)
        s_d = torch.from_numpy(srcs).to(DEV)
        out = torch.empty((len(srcs), self.g.n), dtype=torch.int32, device=DEV)
        o = fg.fg_default_opts(**dict(dict(watchdog_ms=10000), **opts))
        f = fg.fg_sssp_batch if kind == "sssp" else fg.fg_bfs_batch
        fg.check(f(self.h, s_d, len(srcs), out, None, o))
        st = fg.fg_sync()
        return st, out.cpu().numpy().view(np.uint32)

    def ppr(self, srcs, alpha, eps, **opts):
        srcs = np.ascontiguousarray(srcs, dtype=np.int32)
        s_d = torch.from_numpy(srcs).to(DEV)
        p = torch.empty((len(srcs), self.g.n), dtype=torch.float32, device=DEV)
        r = torch.empty_like(p)
        mass = torch.empty(len(srcs), dtype=torch.float64, device=DEV)
        o = fg.fg_default_opts(**dict(dict(watchdog_ms=10000), **opts))
        fg.check(fg.fg_ppr_batch(self.h, s_d, len(srcs), alpha, eps, p, r, mass, None, o))
        st = fg.fg_sync()
        return st, p.cpu().numpy(), r.cpu().numpy(), mass.cpu().numpy()

    def stats(self):
        st, s = fg.fg_stats(self.h)
        fg.check(st)
        return s


def small_graphs():
    gs = []
    n = 70
    gs.append(inputs.from_edges(n, [(i, i + 1, 3 + i % 5) for i in range(n - 1)], name="path"))
    gs.append(inputs.from_edges(n, [(i, (i + 1) % n, 1 + (7 * i) % 11) for i in range(n)], name="cycle"))
    gs.append(inputs.from_edges(50, [(0, i, i) for i in range(1, 50)], name="star"))
    gs.append(inputs.from_edges(24, [(u, v, 1 + (u * v) % 13) for u in range(24) for v in range(u + 1, 24)],
                                name="K24"))
    full = inputs.grid(30, 41, 0, 0, seed=3)
    full.w = np.full(full.m, 7, dtype=np.int32)
    full.name = "fullgrid"
    gs.append(full)
    gs.append(inputs.grid(45, 60, 3000, 100, seed=5, weights=(100, 10000)))  # disconnected pieces
    gs.append(inputs.rmat(8, 8, seed=1, weights=(1, 255)))
    gs.append(inputs.rmat(11, 16, seed=2, weights=(1, 255)))
    gs.append(inputs.rmat(10, 8, seed=3, directed=True, weights=(1, 255)))
    return gs


GRAPHS = small_graphs()


@pytest.mark.parametrize("gi", range(len(GRAPHS)), ids=[g.name for g in GRAPHS])
@pytest.mark.parametrize("method,S", [(fg.FG_PART_RANGE, 32), (fg.FG_PART_GROW, 64), (fg.FG_PART_AUTO, 0),
                                      (fg.FG_PART_DEGREE, 32)])
def test_sssp_bfs_exact_small(gi, method, S):
    g = GRAPHS[gi]
    dg = DevGraph(g, method, S)
    try:
        for nq in (1, 3, 33):
            srcs = (np.arange(nq) * 7919) % g.n
            st, d = dg.run("sssp", srcs)
            fg.check(st)
            assert np.array_equal(d, oracle.sssp(g, srcs)), (g.name, nq)
            st, lv = dg.run("bfs", srcs)
            fg.check(st)
            assert np.array_equal(lv, oracle.bfs(g, srcs)), (g.name, nq)
    finally:
        dg.close()


OPTS = [
    dict(),
    dict(sched=fg.FG_SCHED_PRIORITY),
    dict(delta=300),
    dict(delta=300, bucket=100, sched=fg.FG_SCHED_PRIORITY, sched_window=600),
    dict(bucket=50),
    dict(yield_edges=8),
    dict(yield_edges=1, delta=100),
    dict(emit_capacity=1),
    dict(emit_capacity=7, yield_edges=3),
    dict(mode=fg.FG_MODE_PLAIN),
    dict(threads_per_vertex=1),
    dict(threads_per_vertex=1, delta=300, sched=fg.FG_SCHED_PRIORITY),
    dict(sched=fg.FG_SCHED_MAXOPS),
    dict(sched=fg.FG_SCHED_RANDOM),
    dict(sched=fg.FG_SCHED_MAXOPS, group=1, yield_edges=4),
    dict(sched=fg.FG_SCHED_RANDOM, group=1, delta=300),
    dict(group=1),
    dict(group=8),
    dict(group=32, sched=fg.FG_SCHED_PRIORITY, sched_window=500),
]


@pytest.mark.parametrize("opts", OPTS, ids=[str(o) for o in OPTS])
def test_options_never_change_results(opts):
    """Scheduling, yield heuristics and buffer capacity change the work, never the answer (Sec. 5.1, App. B.2)."""
    for g, method, S in ((inputs.grid(40, 50, 500, 100, seed=8, weights=(100, 10000)), fg.FG_PART_GROW, 64),
                         (inputs.rmat(10, 8, seed=5, weights=(1, 255)), fg.FG_PART_RANGE, 128)):
        dg = DevGraph(g, method, S)
        try:
            srcs = inputs.sources_uniform(g, 40, 3)
            srcs[5] = srcs[4]  # duplicate source
            bopts = dict(opts)
            if "delta" in bopts and g.w.max() <= 255:
                bopts["delta"] = 30
            st, d = dg.run("sssp", srcs, **bopts)
            fg.check(st)
            assert np.array_equal(d, oracle.sssp(g, srcs))
            if "delta" in bopts:
                bopts["delta"] = 2
                bopts.pop("sched_window", None)
                bopts.pop("bucket", None)
            st, lv = dg.run("bfs", srcs, **bopts)
            fg.check(st)
            assert np.array_equal(lv, oracle.bfs(g, srcs))
        finally:
            dg.close()


def test_rmat14_plain_sssp_workload_exact():
    """64 sources on R-MAT scale 14, buffered and plain forms, bit-exact with Dijkstra."""
    name = "rmat14_plain_sssp"
    g = inputs.workload_graph(name)
    srcs = inputs.workload_sources(name, g)
    ref = oracle.sssp(g, srcs)
    dg = DevGraph(g)
    try:
        st, d = dg.run("sssp", srcs)
        fg.check(st)
        assert np.array_equal(d, ref)
        st, d = dg.run("sssp", srcs, mode=fg.FG_MODE_PLAIN)
        fg.check(st)
        assert np.array_equal(d, ref)
    finally:
        dg.close()


def check_ppr(g, srcs, p, r, mass, alpha, eps, directed=False):
    pi = oracle.ppr_power(g, srcs, alpha)
    deg = np.diff(g.row_ptr).astype(np.float64)
    assert np.all(np.abs(mass - 1.0) <= 1e-5), mass
    assert np.all(np.abs(p.sum(1, dtype=np.float64) + r.sum(1, dtype=np.float64) - mass) <= 1e-6)
    assert np.all(r < eps * np.maximum(deg, 1) * (1 + 1e-6) + 1e-12), "push stopped with an active vertex"
    err = np.abs(p.astype(np.float64) - pi)
    if directed:
        assert np.all(pi - p <= r.sum(1, dtype=np.float64)[:, None] + 1e-6)
    else:
        assert np.all(err <= eps * deg[None, :] + 1e-6), err.max()


@pytest.mark.parametrize("gi", [0, 1, 3, 4, 5, 6, 7, 8], ids=[GRAPHS[i].name for i in [0, 1, 3, 4, 5, 6, 7, 8]])
@pytest.mark.parametrize("method,S", [(fg.FG_PART_RANGE, 32), (fg.FG_PART_GROW, 64), (fg.FG_PART_DEGREE, 32)])
def test_ppr_bound_small(gi, method, S):
    g = GRAPHS[gi]
    dg = DevGraph(g, method, S)
    try:
        srcs = inputs.sources_uniform(g, min(20, g.n // 2), 4)
        for eps in (1e-4, 1e-6):
            st, p, r, mass = dg.ppr(srcs, 0.15, eps)
            fg.check(st)
            check_ppr(g, srcs, p, r, mass, 0.15, eps, directed=g.directed)
    finally:
        dg.close()


@pytest.mark.parametrize("opts", [dict(mode=fg.FG_MODE_PLAIN), dict(yield_edges=16), dict(emit_capacity=4096)],
                         ids=["plain", "yield", "spill"])
def test_ppr_options(opts):
    g = inputs.rmat(10, 8, seed=6)
    dg = DevGraph(g, fg.FG_PART_RANGE, 64)
    try:
        srcs = inputs.sources_logdeg(g, 24, 2)
        st, p, r, mass = dg.ppr(srcs, 0.15, 1e-5, **opts)
        fg.check(st)
        check_ppr(g, srcs, p, r, mass, 0.15, 1e-5)
    finally:
        dg.close()


def test_watchdog_max_rounds_times_out():
    g = inputs.grid(40, 40, 0, 0, seed=1)
    dg = DevGraph(g, fg.FG_PART_GROW, 64)
    try:
        st, _ = dg.run("bfs", [0, 5], max_rounds=1)
        assert st == fg.FG_ERR_TIMEOUT
        st, lv = dg.run("bfs", [0, 5])  # the graph stays usable
        fg.check(st)
        assert np.array_equal(lv, oracle.bfs(g, [0, 5]))
    finally:
        dg.close()


def test_device_side_bad_source_reported_at_sync():
    g = inputs.grid(10, 10, 0, 0, seed=1)
    dg = DevGraph(g, fg.FG_PART_RANGE, 32)
    try:
        st, _ = dg.run("sssp", [0, 100])
        assert st == fg.FG_ERR_INVALID_ARG
        st, d = dg.run("sssp", [0, 99])
        fg.check(st)
        assert np.array_equal(d, oracle.sssp(g, [0, 99]))
    finally:
        dg.close()


def test_host_io_path():
    g = inputs.grid(30, 30, 500, 100, seed=2, weights=(100, 10000))
    dg = DevGraph(g, fg.FG_PART_GROW, 64)
    try:
        srcs = inputs.sources_uniform(g, 9, 1)
        out = np.empty((9, g.n), dtype=np.uint32)
        o = fg.fg_default_opts(host_io=1)
        fg.check(fg.fg_sssp_batch(dg.h, srcs, 9, out, None, o))
        fg.check(fg.fg_sync())
        assert np.array_equal(out, oracle.sssp(g, srcs))
        bad = srcs.copy()
        bad[3] = g.n
        assert fg.fg_sssp_batch(dg.h, bad, 9, out, None, o) == fg.FG_ERR_INVALID_ARG
        p = np.empty((9, g.n), dtype=np.float32)
        r = np.empty((9, g.n), dtype=np.float32)
        mass = np.empty(9, dtype=np.float64)
        fg.check(fg.fg_ppr_batch(dg.h, srcs, 9, 0.15, 1e-5, p, r, mass, None, o))
        fg.check(fg.fg_sync())
        check_ppr(g, srcs, p, r, mass, 0.15, 1e-5)
    finally:
        dg.close()


def test_async_host_io_two_streams():
    # host_io = 2: results land in host buffers at fg_sync; batches alternate between two
    # staging slots, so several batches in flight on two streams must not disturb each other
    g = inputs.grid(40, 40, 500, 100, seed=3, weights=(100, 10000))
    dg = DevGraph(g, fg.FG_PART_GROW, 64)
    try:
        sets = [inputs.sources_uniform(g, 7, 10 + i) for i in range(5)]
        outs = [np.full((7, g.n), 7, dtype=np.uint32) for _ in sets]
        sa, sb = torch.cuda.Stream(), torch.cuda.Stream()
        o = fg.fg_default_opts(host_io=2, watchdog_ms=10000)
        for i, (srcs, out) in enumerate(zip(sets, outs)):
            f = fg.fg_bfs_batch if i % 2 == 0 else fg.fg_sssp_batch
            fg.check(f(dg.h, srcs, 7, out, sa if i % 2 == 0 else sb, o))
        fg.check(fg.fg_sync(sa))
        fg.check(fg.fg_sync(sb))
        for i, (srcs, out) in enumerate(zip(sets, outs)):
            ref = oracle.bfs(g, srcs) if i % 2 == 0 else oracle.sssp(g, srcs)
            assert np.array_equal(out, ref), i
        assert fg.fg_sssp_batch(dg.h, sets[0], 7, outs[0], None, fg.fg_default_opts(host_io=3)) == \
            fg.FG_ERR_INVALID_ARG
    finally:
        dg.close()


def test_query_batch_split():
    g = inputs.rmat(10, 8, seed=9, weights=(1, 255))
    dg = DevGraph(g, fg.FG_PART_RANGE, 64)
    try:
        srcs = inputs.sources_uniform(g, 50, 8)
        st, d = dg.run("sssp", srcs, query_batch=7)
        fg.check(st)
        assert np.array_equal(d, oracle.sssp(g, srcs))
    finally:
        dg.close()
