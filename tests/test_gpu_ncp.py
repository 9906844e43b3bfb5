"""Parity of the NCP sweep (fg_ncp_sweep) with the oracle's sweep, bit for bit.

Both sides take the same FP32 rows: the sweep order (FP32 keys, ties by id),
the counts, every prefix's conductance (exact int64 cut and volume, one FP64
division) and the profile (minimum over queries per size) must be identical.
The rows never come from the CUDA path: they are the oracle's FP64 forward
push rounded to FP32 (PPR vectors, the application's input) or seeded
generators that reach the sweep's edge cases: many exactly equal keys, fewer
positive entries than `top`, all-zero rows, NaN / negative / subnormal
entries, top = 1 and top = FG_NCP_MAX_TOP, n not a multiple of 4 and rows not
16-byte aligned (scalar loads), identity and relabelled vertex orders, a
directed graph with hubs. The full-size application run (GPU PPR, then the
sweep) is checked by properties that hold at any size.
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


def _graph(g, method=fg.FG_PART_GROW, S=0):
    go = fg.fg_default_graph_opts(partition_method=method, partition_vertices=S)
    st, h = fg.fg_graph_create_ex(g.n, g.m, g.row_ptr, g.col, g.w, 0, go)
    fg.check(st)
    return h


def _sweep(h, p_rows, top, accumulate_into=None):
    p = torch.from_numpy(np.ascontiguousarray(p_rows, dtype=np.float32)).to(DEV)
    nq = p.shape[0]
    order = torch.empty((nq, top), dtype=torch.int32, device=DEV)
    phi = torch.empty((nq, top), dtype=torch.float64, device=DEV)
    count = torch.empty(nq, dtype=torch.int32, device=DEV)
    ncp = accumulate_into if accumulate_into is not None else torch.empty(top, dtype=torch.float64, device=DEV)
    fg.check(fg.fg_ncp_sweep(h, p, nq, top, order, phi, count, ncp, accumulate_into is not None))
    fg.check(fg.fg_sync())
    return order.cpu().numpy(), phi.cpu().numpy(), count.cpu().numpy(), ncp.cpu().numpy()


def _profile(phi, count, top):
    """Minimum over queries per size; +inf where no query reaches that size."""
    prof = np.full(top, np.inf)
    for q in range(phi.shape[0]):
        c = int(count[q])
        prof[:c] = np.minimum(prof[:c], phi[q, :c])
    return prof


def _check(g, h, p_rows, top):
    o, ph, c, prof = _sweep(h, p_rows, top)
    ro, rph, rc = oracle.ncp_sweep(g, p_rows, top)
    assert np.array_equal(c, rc)
    assert np.array_equal(o, ro)
    assert np.array_equal(ph, rph, equal_nan=True)
    assert np.array_equal(prof, _profile(rph, rc, top))
    return c


def _ppr_rows(g, srcs, alpha=0.15, eps=1e-6):
    """The oracle's FP64 forward-push PPR vectors, rounded to FP32."""
    return np.stack([oracle.ppr_push(g, int(s), alpha, eps)[0] for s in srcs]).astype(np.float32)


@pytest.mark.parametrize("method,dims", [(fg.FG_PART_RANGE, (60, 70)), (fg.FG_PART_GROW, (60, 70)),
                                         (fg.FG_PART_GROW, (61, 69))])
def test_ppr_rows_on_a_grid(method, dims):
    # n = 4200 (float4 row loads, a ragged last tile) and n = 4209 (scalar row loads)
    g = inputs.grid(*dims, 300, 50, seed=41)
    h = _graph(g, method, 256)
    try:
        rows = _ppr_rows(g, inputs.sources_uniform(g, 12, seed=42), eps=1e-7)
        c = _check(g, h, rows, 2000)
        assert c.min() > 100  # long sweeps
        _check(g, h, rows, 1)
    finally:
        fg.fg_graph_destroy(h)


def test_ppr_rows_on_a_directed_rmat_with_hubs():
    g = inputs.rmat(13, 16, seed=43, directed=True)
    h = _graph(g, fg.FG_PART_AUTO, 0)
    try:
        rows = _ppr_rows(g, inputs.sources_uniform(g, 16, seed=44), eps=1e-7)
        _check(g, h, rows, fg.FG_NCP_MAX_TOP)
    finally:
        fg.fg_graph_destroy(h)


def test_exact_ties_beyond_the_candidate_buffer():
    # p = 1 everywhere on a grid: ~all keys equal 1/4, far more than fit the buffer;
    # the kept ones must be the smallest ids
    g = inputs.grid(150, 150, 0, 0, seed=45)
    h = _graph(g, fg.FG_PART_GROW, 512)
    try:
        n = g.n
        rows = np.ones((3, n), dtype=np.float32)
        rows[1, ::7] = 2.0  # a few larger keys above the tie
        rows[2, :] = 0.0
        rows[2, 5000:30000] = 0.5
        c = _check(g, h, rows, fg.FG_NCP_MAX_TOP)
        assert list(c) == [fg.FG_NCP_MAX_TOP] * 3
    finally:
        fg.fg_graph_destroy(h)


def test_sparse_zero_and_odd_rows():
    g = inputs.rmat(12, 8, seed=46, weights=(1, 9))
    h = _graph(g, fg.FG_PART_GROW, 128)
    try:
        rng = np.random.default_rng(47)
        n = g.n
        rows = np.zeros((6, n), dtype=np.float32)
        rows[0, rng.choice(n, 37, replace=False)] = rng.random(37).astype(np.float32)  # fewer than top
        # row 1 stays all zero: count 0
        rows[2] = rng.random(n).astype(np.float32)
        rows[2, ::3] = -rows[2, ::3]                      # negatives are not candidates
        rows[2, 1::11] = np.nan                           # NaN is not a candidate
        rows[3, :] = np.float32(1e-45)                    # subnormal: some keys round to zero
        rows[3, ::5] = np.float32(3e-45)
        rows[4] = rng.lognormal(-12, 4, n).astype(np.float32)  # keys over many octaves
        rows[5] = np.float32(1e-3) * rng.integers(1, 4, n).astype(np.float32)  # few distinct values
        c = _check(g, h, rows, 3000)
        assert c[0] == 37 and c[1] == 0
        _check(g, h, rows[:2], 37)
        # rows that start 4 bytes past a 16-byte boundary take the scalar loads
        flat = torch.zeros(rows.size + 1, dtype=torch.float32, device=DEV)
        flat[1:] = torch.from_numpy(rows.ravel()).to(DEV)
        p_off = flat[1:].view(rows.shape)
        assert p_off.data_ptr() % 16 == 4
        nq, top = rows.shape[0], 3000
        order = torch.empty((nq, top), dtype=torch.int32, device=DEV)
        phi = torch.empty((nq, top), dtype=torch.float64, device=DEV)
        count = torch.empty(nq, dtype=torch.int32, device=DEV)
        fg.check(fg.fg_ncp_sweep(h, p_off, nq, top, order, phi, count))
        fg.check(fg.fg_sync())
        ro, rph, rc = oracle.ncp_sweep(g, rows, top)
        assert np.array_equal(count.cpu().numpy(), rc) and np.array_equal(order.cpu().numpy(), ro)
        assert np.array_equal(phi.cpu().numpy(), rph, equal_nan=True)
    finally:
        fg.fg_graph_destroy(h)


def test_rows_split_across_blocks():
    # few rows on a larger graph: each row is split into segments whose survivors are merged
    g = inputs.rmat(16, 8, seed=51)
    h = _graph(g, fg.FG_PART_GROW, 0)
    try:
        rows = _ppr_rows(g, inputs.sources_uniform(g, 8, seed=52), eps=1e-6)
        c = _check(g, h, rows, fg.FG_NCP_MAX_TOP)
        assert c.min() > 1000
        _check(g, h, rows[:1], 777)
    finally:
        fg.fg_graph_destroy(h)
    g = inputs.grid(200, 200, 0, 0, seed=53)  # exact ties across segment boundaries
    h = _graph(g, fg.FG_PART_GROW, 512)
    try:
        rows = np.ones((2, g.n), dtype=np.float32)
        rows[1, 10000:] = 0.25
        _check(g, h, rows, fg.FG_NCP_MAX_TOP)
    finally:
        fg.fg_graph_destroy(h)


def test_hubs_in_the_sweep_set():
    # a star whose centre (9,000 arcs) is swept first: counted by the whole block
    n = 9001
    g = inputs.from_edges(n, [(0, i) for i in range(1, n)])
    h = _graph(g, fg.FG_PART_RANGE, 0)
    try:
        rows = np.full((2, n), 1e-3, dtype=np.float32)
        rows[:, 0] = 50.0
        rows[1, 1::2] = 2e-3
        _check(g, h, rows, fg.FG_NCP_MAX_TOP)
    finally:
        fg.fg_graph_destroy(h)
    # K(70, 5000): 70 hubs of 5,000 arcs in the set, more than the block queue holds
    hubs, leaves = 70, 5000
    g = inputs.from_edges(hubs + leaves, [(i, hubs + j) for i in range(hubs) for j in range(leaves)])
    h = _graph(g, fg.FG_PART_GROW, 512)
    try:
        rng = np.random.default_rng(54)
        rows = rng.random((2, g.n)).astype(np.float32) * np.float32(1e-3)
        rows[:, :hubs] += np.float32(1e4)
        _check(g, h, rows, fg.FG_NCP_MAX_TOP)
    finally:
        fg.fg_graph_destroy(h)


def test_profile_accumulates_over_calls():
    g = inputs.grid(40, 40, 100, 20, seed=48)
    h = _graph(g)
    try:
        rows = _ppr_rows(g, inputs.sources_uniform(g, 10, seed=49))
        top = 700
        _, _, _, whole = _sweep(h, rows, top)
        _, _, _, first = _sweep(h, rows[:4], top)  # without accumulate: this call's rows only
        ncp = torch.from_numpy(first).to(DEV)
        _, _, _, both = _sweep(h, rows[4:], top, accumulate_into=ncp)
        assert np.array_equal(both, whole)
        assert not np.array_equal(first, whole)
    finally:
        fg.fg_graph_destroy(h)


def test_bad_arguments_are_rejected_on_the_host():
    g = inputs.grid(8, 8, 0, 0, seed=50)
    h = _graph(g)
    try:
        p = torch.zeros((1, g.n), dtype=torch.float32, device=DEV)
        cnt = torch.empty(1, dtype=torch.int32, device=DEV)
        assert fg.fg_ncp_sweep(h, p, 1, 0, None, None, cnt) == fg.FG_ERR_INVALID_ARG
        assert fg.fg_ncp_sweep(h, p, 1, fg.FG_NCP_MAX_TOP + 1, None, None, cnt) == fg.FG_ERR_INVALID_ARG
        assert fg.fg_ncp_sweep(h, p, 0, 4, None, None, cnt) == fg.FG_ERR_INVALID_ARG
        assert fg.fg_ncp_sweep(h, p, 1, 4) == fg.FG_ERR_INVALID_ARG  # no output
        assert fg.fg_ncp_sweep(h, None, 1, 4, None, None, cnt) == fg.FG_ERR_INVALID_ARG
        fg.check(fg.fg_ncp_sweep(h, p, 1, 4, None, None, cnt))
        fg.check(fg.fg_sync())
        assert int(cnt[0]) == 0
    finally:
        fg.fg_graph_destroy(h)


@pytest.mark.slow
def test_rmat22_ncp_application():
    """The NCP application at full size: PPRs from 0.01% of the vertices of R-MAT
    scale 22 on the GPU, swept to 4096 vertices (properties: counts, cuts >= 0,
    the profile is the minimum of the rows); and the sweep at the same size on
    the oracle's own PPR rows for four of the seeds, bit for bit."""
    g = inputs.workload_graph("rmat22_ppr")
    h = _graph(g, fg.FG_PART_AUTO, 0)
    try:
        seeds = inputs.ncp_seeds(g)
        assert len(seeds) == round(1e-4 * g.n)
        s_d = torch.from_numpy(seeds).to(DEV)
        nq, top = len(seeds), fg.FG_NCP_MAX_TOP
        p = torch.empty((nq, g.n), dtype=torch.float32, device=DEV)
        fg.check(fg.fg_ppr_batch(h, s_d, nq, 0.15, 1e-7, p, None, None, None, fg.fg_default_opts()))
        order = torch.empty((nq, top), dtype=torch.int32, device=DEV)
        phi = torch.empty((nq, top), dtype=torch.float64, device=DEV)
        count = torch.empty(nq, dtype=torch.int32, device=DEV)
        ncp = torch.empty(top, dtype=torch.float64, device=DEV)
        fg.check(fg.fg_ncp_sweep(h, p, nq, top, order, phi, count, ncp))
        fg.check(fg.fg_sync())
        nnz = (p > 0).sum(dim=1).cpu().numpy()
        cnt = count.cpu().numpy()
        assert np.array_equal(cnt, np.minimum(nnz, top))
        ph = phi.cpu().numpy()
        assert np.array_equal(ncp.cpu().numpy(), _profile(ph, cnt, top))
        assert np.all(ph[~np.isnan(ph)] >= 0)  # undirected: cuts are non-negative
        o = order.cpu().numpy()
        for q in (0, nq // 2, nq - 1):  # each sweep lists distinct vertices with p > 0, largest key first
            c = int(cnt[q])
            assert len(set(o[q, :c].tolist())) == c and np.all(o[q, c:] == -1)
            keys = p[q, o[q, :c]].cpu().numpy() / np.maximum(np.diff(g.row_ptr)[o[q, :c]], 1).astype(np.float32)
            assert np.all(keys > 0) and np.all(np.diff(keys) <= 0)
        rows = _ppr_rows(g, seeds[[0, 1, nq // 2, nq - 1]], eps=1e-7)
        _check(g, h, rows, top)
    finally:
        fg.fg_graph_destroy(h)
