"""Serving loop (fg_server_*): results in a mixed, overlapping stream equal the results alone.

Requests of all three kinds are submitted in waves while earlier batches are
still on the device. Each SSSP/BFS result must be bit-identical to a batch of
that one source through fg_sssp_batch / fg_bfs_batch (and to the oracle); each
PPR result must meet the push bound against the FP64 oracle and agree with its
stand-alone run within twice that bound (push order may differ), with mass 1.
"""
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_2103_14915_gb300 import fg, inputs

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
ALPHA, EPS = 0.15, 1e-5


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2103_14915_gb300 import build
    build.build()
    fg.load()
    assert torch.cuda.is_available()


@pytest.fixture(scope="module")
def graph():
    g = inputs.grid(48, 64, 500, 100, seed=21, weights=(100, 10000))
    go = fg.fg_default_graph_opts(partition_method=fg.FG_PART_GROW, partition_vertices=256)
    st, h = fg.fg_graph_create_ex(g.n, g.m, g.row_ptr, g.col, g.w, 0, go)
    fg.check(st)
    yield g, h
    fg.fg_graph_destroy(h)


def _alone(h, g, kind, s):
    s_d = torch.tensor([s], dtype=torch.int32, device=DEV)
    o = fg.fg_default_opts(watchdog_ms=10000)
    if kind == fg.FG_QUERY_PPR:
        p = torch.empty((1, g.n), dtype=torch.float32, device=DEV)
        fg.check(fg.fg_ppr_batch(h, s_d, 1, ALPHA, EPS, p, None, None, None, o))
        fg.check(fg.fg_sync())
        return p.cpu().numpy()[0]
    out = torch.empty((1, g.n), dtype=torch.int32, device=DEV)
    f = fg.fg_sssp_batch if kind == fg.FG_QUERY_SSSP else fg.fg_bfs_batch
    fg.check(f(h, s_d, 1, out, None, o))
    fg.check(fg.fg_sync())
    return out.cpu().numpy().view(np.uint32)[0]


class _DeviceRow:
    """A server-owned device row seen through __cuda_array_interface__ (no copy, no ownership)."""

    def __init__(self, ptr, n, typestr):
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": typestr, "data": (ptr, False), "version": 3}


def _row(info, n):
    ppr = info.kind == fg.FG_QUERY_PPR
    t = torch.as_tensor(_DeviceRow(info.result, n, "<f4" if ppr else "<i4"), device=DEV).clone()
    a = t.cpu().numpy()
    return a if ppr else a.view(np.uint32)


def _run_mix(h, g, reqs, lanes, max_batch, waves):
    so = fg.fg_default_server_opts(lanes=lanes, max_batch=max_batch, alpha=ALPHA, eps=EPS)
    for k in range(3):
        so.opts[k].watchdog_ms = 10000
    st, srv = fg.fg_server_create(h, so)
    fg.check(st)
    results, infos = {}, {}
    try:
        ids = {}
        per_wave = (len(reqs) + waves - 1) // waves
        for w in range(waves):
            for i, (kind, s) in enumerate(reqs[w * per_wave:(w + 1) * per_wave]):
                st, rid = fg.fg_server_submit(srv, kind, s)
                fg.check(st)
                ids[rid] = w * per_wave + i
            st, done = fg.fg_server_poll(srv)
            fg.check(st)
            for rid in done:
                st, info = fg.fg_server_info(srv, rid)
                fg.check(st)
                results[ids[rid]] = _row(info, g.n)
                infos[ids[rid]] = (info.status, info.mass, info.batch_size, info.launch_ns, info.done_ns)
                fg.check(fg.fg_server_release(srv, rid))
        t_end = time.time() + 60
        while len(results) < len(reqs):
            assert time.time() < t_end, "server did not complete the requests"
            st, done = fg.fg_server_poll(srv)
            fg.check(st)
            for rid in done:
                st, info = fg.fg_server_info(srv, rid)
                fg.check(st)
                results[ids[rid]] = _row(info, g.n)
                infos[ids[rid]] = (info.status, info.mass, info.batch_size, info.launch_ns, info.done_ns)
                fg.check(fg.fg_server_release(srv, rid))
        # batches overlapped in time when some launch precedes another's completion
        spans = sorted((v[3], v[4]) for v in infos.values())
        overlapped = any(spans[i + 1][0] < spans[i][1] for i in range(len(spans) - 1) if spans[i + 1][0] != spans[i][0])
    finally:
        fg.fg_server_destroy(srv)
    return results, infos, overlapped


def test_mix_equals_alone(graph):
    g, h = graph
    rng = np.random.default_rng(5)
    srcs = inputs.sources_uniform(g, 24, seed=31)
    kinds = rng.integers(0, 3, size=len(srcs))
    reqs = [(int(k), int(s)) for k, s in zip(kinds, srcs)]
    reqs.append(reqs[0])  # the same request twice in the mix
    results, infos, _ = _run_mix(h, g, reqs, lanes=3, max_batch=4, waves=5)
    deg = np.diff(g.row_ptr).astype(np.float64)
    for i, (kind, s) in enumerate(reqs):
        assert infos[i][0] == fg.FG_OK
        alone = _alone(h, g, kind, s)
        if kind == fg.FG_QUERY_PPR:
            pi = oracle.ppr_power(g, [s], ALPHA)[0]
            bound = EPS * deg + 1e-6
            assert np.all(np.abs(results[i].astype(np.float64) - pi) <= bound)
            assert np.all(np.abs(results[i].astype(np.float64) - alone.astype(np.float64)) <= 2 * bound)
            assert abs(infos[i][1] - 1.0) <= 1e-5
        else:
            assert np.array_equal(results[i], alone)
            ref = oracle.sssp(g, [s])[0] if kind == fg.FG_QUERY_SSSP else oracle.bfs(g, [s])[0]
            assert np.array_equal(results[i], ref)


def test_batches_overlap_on_the_device(graph):
    g, h = graph
    srcs = inputs.sources_uniform(g, 48, seed=32)
    reqs = [(k % 2, int(s)) for k, s in enumerate(srcs)]  # SSSP and BFS
    results, infos, overlapped = _run_mix(h, g, reqs, lanes=4, max_batch=6, waves=8)
    assert len(results) == len(reqs)
    assert max(v[2] for v in infos.values()) > 1  # requests were batched
    assert overlapped
    for i, (kind, s) in enumerate(reqs[:6]):
        assert np.array_equal(results[i], _alone(h, g, kind, s))


def test_submit_rejects_bad_requests(graph):
    g, h = graph
    st, srv = fg.fg_server_create(h, fg.fg_default_server_opts(lanes=1, max_batch=2))
    fg.check(st)
    try:
        assert fg.fg_server_submit(srv, 7, 0)[0] == fg.FG_ERR_INVALID_ARG
        assert fg.fg_server_submit(srv, fg.FG_QUERY_BFS, g.n)[0] == fg.FG_ERR_INVALID_ARG
        st, rid = fg.fg_server_submit(srv, fg.FG_QUERY_BFS, 0)
        fg.check(st)
        assert fg.fg_server_release(srv, rid) == fg.FG_ERR_INVALID_ARG  # not completed yet
        st, info = fg.fg_server_info(srv, rid)
        assert info.status == -1
    finally:
        fg.fg_server_destroy(srv)


def test_budget_lowers_batch_size(graph):
    g, h = graph
    info = fg.fg_graph_info(h)[1]
    # device bytes of one PPR request (the most expensive kind) on this relabelled graph:
    # p and r rows, engine estimate/residual/compensation scratch, per-key buffers
    per_q = 20 * g.n + info.num_partitions * 36 + g.n / 8
    so = fg.fg_default_server_opts(lanes=2, max_batch=256, hbm_budget=int(2 * 3 * per_q) + 64)
    st, srv = fg.fg_server_create(h, so)
    fg.check(st)
    try:
        srcs = inputs.sources_uniform(g, 10, seed=33)
        for s in srcs:
            fg.check(fg.fg_server_submit(srv, fg.FG_QUERY_SSSP, int(s))[0])
        sizes, t_end = [], time.time() + 60
        while len(sizes) < len(srcs):
            assert time.time() < t_end
            st, done = fg.fg_server_poll(srv)
            fg.check(st)
            for rid in done:
                sizes.append(fg.fg_server_info(srv, rid)[1].batch_size)
                fg.check(fg.fg_server_release(srv, rid))
        assert max(sizes) == 3  # a full batch of 3 fits each of the 2 lanes, 4 would not
    finally:
        fg.fg_server_destroy(srv)
    st, _ = fg.fg_server_create(h, fg.fg_default_server_opts(lanes=2, hbm_budget=1000))
    assert st == fg.FG_ERR_OOM


def test_destroy_with_batches_in_flight(graph):
    g, h = graph
    st, srv = fg.fg_server_create(h, fg.fg_default_server_opts(lanes=2, max_batch=8))
    fg.check(st)
    for s in inputs.sources_uniform(g, 12, seed=34):
        fg.check(fg.fg_server_submit(srv, fg.FG_QUERY_SSSP, int(s))[0])
    st, _ = fg.fg_server_poll(srv)  # launches both lanes
    fg.check(st)
    assert fg.fg_server_destroy(srv) == fg.FG_OK  # waits for the lanes, then frees
    # the graph and the library stay usable
    s_d = torch.tensor([0], dtype=torch.int32, device=DEV)
    out = torch.empty((1, g.n), dtype=torch.int32, device=DEV)
    fg.check(fg.fg_bfs_batch(h, s_d, 1, out, None, None))
    fg.check(fg.fg_sync())
    assert np.array_equal(out.cpu().numpy().view(np.uint32)[0], oracle.bfs(g, [0])[0])


def test_directed_graph_mix():
    g = inputs.rmat(10, 8, seed=12, directed=True, weights=(1, 255))  # has dangling vertices
    st, h = fg.fg_graph_create_ex(g.n, g.m, g.row_ptr, g.col, g.w, 0, fg.fg_default_graph_opts())
    fg.check(st)
    try:
        srcs = inputs.sources_uniform(g, 9, seed=35)
        reqs = [(k % 3, int(s)) for k, s in enumerate(srcs)]
        results, infos, _ = _run_mix(h, g, reqs, lanes=2, max_batch=3, waves=3)
        for i, (kind, s) in enumerate(reqs):
            assert infos[i][0] == fg.FG_OK
            if kind == fg.FG_QUERY_PPR:
                assert abs(infos[i][1] - 1.0) <= 1e-5  # mass, with dangling vertices returning to the source
                pi = oracle.ppr_power(g, [s], ALPHA)[0]
                assert np.all(results[i].astype(np.float64) <= pi + 1e-6)  # p approaches pi from below
            else:
                ref = oracle.sssp(g, [s])[0] if kind == fg.FG_QUERY_SSSP else oracle.bfs(g, [s])[0]
                assert np.array_equal(results[i], ref)
    finally:
        fg.fg_graph_destroy(h)


# ---- slot-level batching (continuous = 1): SSSP and BFS join running launches ----

def _slot_server(h, slots, group=0, lanes=1, max_rounds=0):
    so = fg.fg_default_server_opts(lanes=lanes, max_batch=4, alpha=ALPHA, eps=EPS, continuous=1, slots=slots)
    for k in range(3):
        so.opts[k].watchdog_ms = 10000
        so.opts[k].group = group
        so.opts[k].max_rounds = max_rounds
    st, srv = fg.fg_server_create(h, so)
    fg.check(st)
    return srv


def _drain(srv, g, want, results, infos, ids, timeout=60):
    t_end = time.time() + timeout
    while len(results) < want:
        assert time.time() < t_end, "server did not complete the requests"
        st, done = fg.fg_server_poll(srv)
        fg.check(st)
        for rid in done:
            st, info = fg.fg_server_info(srv, rid)
            fg.check(st)
            results[ids[rid]] = _row(info, g.n)
            infos[ids[rid]] = (info.status, info.batch_size, info.launch_ns, info.done_ns)
            fg.check(fg.fg_server_release(srv, rid))


def _star_rmat():
    """R-MAT s11 plus a star of 3,000 leaves on vertex 0 (a hub of one chunk
    beside the graph's own high-degree vertices)."""
    base = inputs.rmat(11, 16, seed=41, weights=(1, 255))
    edges = []
    for u in range(base.n):
        for e in range(base.row_ptr[u], base.row_ptr[u + 1]):
            edges.append((u, int(base.col[e]), int(base.w[e])))
    n = base.n + 3000
    edges += [(0, base.n + i, 1 + (i * 29) % 250) for i in range(3000)]
    return inputs.from_edges(n, edges, name="rmat11+star")


@pytest.mark.parametrize("which,group", [("grid", 0), ("rmat_star", 16), ("rmat_star", 8)])
def test_slots_mix_equals_oracle(graph, which, group):
    """More requests than slots, submitted in waves while earlier ones run:
    every slot is reused, and each SSSP / BFS row equals the oracle's; PPR
    requests in the same stream still run on the batch lanes."""
    if which == "grid":
        g, h, own = graph[0], graph[1], False
    else:
        g = _star_rmat()
        st, h = fg.fg_graph_create_ex(g.n, g.m, g.row_ptr, g.col, g.w, 0, fg.fg_default_graph_opts())
        fg.check(st)
        own = True
    slots = 32 if group == 0 else 2 * group
    srv = _slot_server(h, slots, group)
    try:
        rng = np.random.default_rng(7)
        srcs = inputs.sources_uniform(g, 3 * slots + 5, seed=42)
        srcs[0] = 0  # the star's centre
        kinds = rng.choice([0, 1, 0, 1, 2], size=len(srcs))
        reqs = [(int(k), int(s)) for k, s in zip(kinds, srcs)]
        results, infos, ids = {}, {}, {}
        per_wave = 9
        for w in range(0, len(reqs), per_wave):
            for i, (kind, s) in enumerate(reqs[w:w + per_wave]):
                st, rid = fg.fg_server_submit(srv, kind, s)
                fg.check(st)
                ids[rid] = w + i
            st, done = fg.fg_server_poll(srv)
            fg.check(st)
            for rid in done:
                st, info = fg.fg_server_info(srv, rid)
                fg.check(st)
                results[ids[rid]] = _row(info, g.n)
                infos[ids[rid]] = (info.status, info.batch_size, info.launch_ns, info.done_ns)
                fg.check(fg.fg_server_release(srv, rid))
        _drain(srv, g, len(reqs), results, infos, ids)
    finally:
        fg.fg_server_destroy(srv)
    for i, (kind, s) in enumerate(reqs):
        assert infos[i][0] == fg.FG_OK
        if kind == fg.FG_QUERY_PPR:
            pi = oracle.ppr_power(g, [s], ALPHA)[0]
            deg = np.diff(g.row_ptr).astype(np.float64)
            assert np.all(np.abs(results[i].astype(np.float64) - pi) <= EPS * deg + 1e-6)
        else:
            assert infos[i][1] == slots  # batch_size reports the slot count
            ref = oracle.sssp(g, [s])[0] if kind == fg.FG_QUERY_SSSP else oracle.bfs(g, [s])[0]
            assert np.array_equal(results[i], ref), (i, kind, s)
    if own:
        fg.fg_graph_destroy(h)


def test_slots_idle_launch_restarts(graph):
    """A launch ends once it holds no query; a later request starts a new one
    on the state the first left behind (lanes reset on retirement)."""
    g, h = graph
    srv = _slot_server(h, 32)
    try:
        for wave in range(3):
            srcs = inputs.sources_uniform(g, 5, seed=50 + wave)
            results, infos, ids = {}, {}, {}
            for i, s in enumerate(srcs):
                st, rid = fg.fg_server_submit(srv, i % 2, int(s))
                fg.check(st)
                ids[rid] = i
            _drain(srv, g, len(srcs), results, infos, ids)
            for i, s in enumerate(srcs):
                ref = oracle.sssp(g, [s])[0] if i % 2 == 0 else oracle.bfs(g, [s])[0]
                assert np.array_equal(results[i], ref)
            time.sleep(0.2)  # the launch has gone idle and ended
    finally:
        fg.fg_server_destroy(srv)


def test_slots_later_request_finishes_first(graph):
    """A request admitted into a running launch completes without waiting for
    the launch's earlier, longer queries: BFS from the four grid corners is
    submitted and launched first, then BFS from the centre, which needs about
    half their rounds and so completes no later than the last corner."""
    g, h = graph
    # grid 48 x 64: vertex ids row-major; corners and centre
    corners = [0, 63, 47 * 64, 47 * 64 + 63]
    centre = 24 * 64 + 32
    srv = _slot_server(h, 32)
    try:
        ids, results, infos = {}, {}, {}
        for i, s in enumerate(corners):
            st, rid = fg.fg_server_submit(srv, fg.FG_QUERY_BFS, s)
            fg.check(st)
            ids[rid] = i
        st, done = fg.fg_server_poll(srv)  # the launch starts with the corners
        fg.check(st)
        assert not done
        st, rid = fg.fg_server_submit(srv, fg.FG_QUERY_BFS, centre)
        fg.check(st)
        ids[rid] = 4
        _drain(srv, g, 5, results, infos, ids)
    finally:
        fg.fg_server_destroy(srv)
    for i, s in enumerate(corners + [centre]):
        assert np.array_equal(results[i], oracle.bfs(g, [s])[0])
    assert infos[4][3] <= max(infos[i][3] for i in range(4))  # done no later than the last corner


def test_slots_launch_yields_and_resumes(graph):
    """With max_rounds 3 a launch yields every third round with its queries in
    flight and the next launch resumes them (about 100 BFS rounds from a grid
    corner span dozens of launches); requests keep arriving meanwhile."""
    g, h = graph
    srv = _slot_server(h, 32, max_rounds=3)
    try:
        srcs = [0, 47 * 64 + 63] + [int(s) for s in inputs.sources_uniform(g, 10, seed=70)]
        results, infos, ids = {}, {}, {}
        for i, s in enumerate(srcs):
            st, rid = fg.fg_server_submit(srv, i % 2, s)
            fg.check(st)
            ids[rid] = i
            if i % 3 == 2:
                st, done = fg.fg_server_poll(srv)
                fg.check(st)
                for d in done:
                    st, info = fg.fg_server_info(srv, d)
                    results[ids[d]] = _row(info, g.n)
                    infos[ids[d]] = (info.status,)
                    fg.check(fg.fg_server_release(srv, d))
        _drain(srv, g, len(srcs), results, infos, ids)
    finally:
        fg.fg_server_destroy(srv)
    for i, s in enumerate(srcs):
        ref = oracle.sssp(g, [s])[0] if i % 2 == 0 else oracle.bfs(g, [s])[0]
        assert np.array_equal(results[i], ref)


def test_slots_destroy_while_running(graph):
    g, h = graph
    srv = _slot_server(h, 32)
    for s in inputs.sources_uniform(g, 20, seed=60):
        fg.check(fg.fg_server_submit(srv, fg.FG_QUERY_SSSP, int(s))[0])
    st, _ = fg.fg_server_poll(srv)
    fg.check(st)
    t0 = time.time()
    assert fg.fg_server_destroy(srv) == fg.FG_OK  # the launch leaves at its next round boundary
    assert time.time() - t0 < 30
    s_d = torch.tensor([5], dtype=torch.int32, device=DEV)
    out = torch.empty((1, g.n), dtype=torch.int32, device=DEV)
    fg.check(fg.fg_sssp_batch(h, s_d, 1, out, None, None))
    fg.check(fg.fg_sync())
    assert np.array_equal(out.cpu().numpy().view(np.uint32)[0], oracle.sssp(g, [5])[0])


def test_slots_option_checks(graph):
    g, h = graph
    for bad in (dict(continuous=2), dict(continuous=1, slots=0), dict(continuous=1, slots=40)):
        st, _ = fg.fg_server_create(h, fg.fg_default_server_opts(**bad))
        assert st == fg.FG_ERR_INVALID_ARG, bad
    so = fg.fg_default_server_opts(continuous=1, slots=64)
    so.opts[0].group = 16
    st, srv = fg.fg_server_create(h, so)  # 64 is a multiple of 16
    fg.check(st)
    fg.fg_server_destroy(srv)
