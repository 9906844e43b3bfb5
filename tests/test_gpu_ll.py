"""Parity of landmark labeling (fg_ll_build_labels, fg_ll_query) with the oracle, bit for bit.

Inputs never come from the CUDA path: label construction takes the oracle's
own SSSP rows (uploaded), the query takes the oracle's labels; the
application chain on the GPU (SSSP batch, labels, queries) is compared with
the same chain in the oracle, which agrees exactly because SSSP is exact.
Edge cases: K = 1, K not a multiple of 4 (4-byte loads), misaligned labels,
n not a multiple of the 64-wide tile, unreachable landmarks (two
components), sums past 2^32, pairs with ids outside [0, n), u = v, Q = 0.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_2103_14915_gb300 import fg, inputs

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
U64 = np.iinfo(np.uint64).max


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2103_14915_gb300 import build
    build.build()
    fg.load()
    assert torch.cuda.is_available()


def _labels_gpu(rows):
    K, n = rows.shape
    d = torch.from_numpy(np.ascontiguousarray(rows).view(np.int32)).to(DEV)
    lab = torch.empty((n, K), dtype=torch.int32, device=DEV)
    fg.check(fg.fg_ll_build_labels(d, K, n, lab))
    fg.check(fg.fg_sync())
    return lab


def _query_gpu(lab, n, K, pairs):
    pr = torch.from_numpy(np.ascontiguousarray(pairs, dtype=np.int32)).to(DEV)
    est = torch.empty(len(pairs), dtype=torch.int64, device=DEV)
    fg.check(fg.fg_ll_query(lab, n, K, pr, len(pairs), est))
    fg.check(fg.fg_sync())
    return est.cpu().numpy().view(np.uint64)


@pytest.mark.parametrize("K", [1, 37, 64, 200])
def test_labels_and_queries_match_the_oracle(K):
    g = inputs.grid(45, 71, 300, 50, seed=60, weights=(1, 500))  # n = 3195: a partial tile in both directions
    rng = np.random.default_rng(K)
    lms = rng.choice(g.n, size=K, replace=False).astype(np.int32)
    rows = oracle.sssp(g, lms)
    lab = _labels_gpu(rows)
    ref = oracle.ll_labels(rows)
    assert np.array_equal(lab.cpu().numpy().view(np.uint32), ref)
    pairs = rng.integers(0, g.n, size=(5000, 2)).astype(np.int32)
    pairs[:50, 1] = pairs[:50, 0]          # u = v
    pairs[50:60, 0] = lms[: min(10, K)].repeat(10 // min(10, K) + 1)[:10]  # landmark endpoints
    pairs[60] = (-1, 3)
    pairs[61] = (3, g.n)                   # ids outside [0, n): no estimate
    got = _query_gpu(lab, g.n, K, pairs)
    exp = oracle.ll_query(ref, np.clip(pairs, 0, g.n - 1))
    exp[60] = exp[61] = U64
    assert np.array_equal(got, exp)


def test_unreachable_landmarks_and_wide_sums():
    # synthetic rows (the label code does not care how they were made): vertices 40.. are
    # unreachable from every landmark, and values near 2^32 make sums pass 32 bits
    rng = np.random.default_rng(68)
    K, n = 4, 61
    rows = rng.integers(0, 2**32 - 1, size=(K, n), dtype=np.uint64).astype(np.uint32)
    rows[:, 40:] = 0xFFFFFFFF
    rows[1, 5] = 0xFFFFFFFF  # one landmark misses vertex 5
    rows[:, 0] = 0xFFFFFFFE
    lab = _labels_gpu(rows)
    ref = oracle.ll_labels(rows)
    assert np.array_equal(lab.cpu().numpy().view(np.uint32), ref)
    pairs = np.array([[0, 0], [0, 5], [45, 50], [1, 45], [5, 7], [39, 2]], dtype=np.int32)
    got = _query_gpu(lab, n, K, pairs)
    assert np.array_equal(got, oracle.ll_query(ref, pairs))
    assert got[0] == 2 * 0xFFFFFFFE and got[2] == U64 and got[3] == U64


def test_misaligned_labels_take_the_scalar_loads():
    g = inputs.grid(20, 30, 300, 50, seed=61, weights=(1, 100))
    K = 16
    rows = oracle.sssp(g, inputs.sources_uniform(g, K, seed=62))
    ref = oracle.ll_labels(rows)
    flat = torch.zeros(ref.size + 1, dtype=torch.int32, device=DEV)
    flat[1:] = torch.from_numpy(ref.view(np.int32).ravel()).to(DEV)
    lab = flat[1:].view(g.n, K)
    assert lab.data_ptr() % 16 == 4
    pairs = np.random.default_rng(63).integers(0, g.n, size=(1000, 2)).astype(np.int32)
    assert np.array_equal(_query_gpu(lab, g.n, K, pairs), oracle.ll_query(ref, pairs))


def test_host_checks():
    lab = torch.zeros((4, 4), dtype=torch.int32, device=DEV)
    pr = torch.zeros((1, 2), dtype=torch.int32, device=DEV)
    est = torch.empty(1, dtype=torch.int64, device=DEV)
    assert fg.fg_ll_build_labels(lab, 0, 4, lab) == fg.FG_ERR_INVALID_ARG
    assert fg.fg_ll_build_labels(None, 4, 4, lab) == fg.FG_ERR_INVALID_ARG
    assert fg.fg_ll_query(lab, 4, 4, pr, -1, est) == fg.FG_ERR_INVALID_ARG
    assert fg.fg_ll_query(lab, 4, 4, None, 1, est) == fg.FG_ERR_INVALID_ARG
    assert fg.fg_ll_query(lab, 4, 4, pr, 0, est) == fg.FG_OK  # empty batch: nothing to do


def test_application_chain_on_the_gpu_equals_the_oracle_chain():
    g = inputs.rmat(12, 8, seed=64, weights=(1, 255))
    K = 128
    lms = inputs.sources_uniform(g, K, seed=65)
    st, h = fg.fg_graph_create_ex(g.n, g.m, g.row_ptr, g.col, g.w, 0, fg.fg_default_graph_opts())
    fg.check(st)
    try:
        s_d = torch.from_numpy(lms).to(DEV)
        dist = torch.empty((K, g.n), dtype=torch.int32, device=DEV)
        fg.check(fg.fg_sssp_batch(h, s_d, K, dist, None, None))
        lab = torch.empty((g.n, K), dtype=torch.int32, device=DEV)
        fg.check(fg.fg_ll_build_labels(dist, K, g.n, lab))
        pairs = np.random.default_rng(66).integers(0, g.n, size=(20000, 2)).astype(np.int32)
        got = _query_gpu(lab, g.n, K, pairs)
        ref = oracle.ll_labels(oracle.sssp(g, lms))
        assert np.array_equal(lab.cpu().numpy().view(np.uint32), ref)
        assert np.array_equal(got, oracle.ll_query(ref, pairs))
    finally:
        fg.fg_graph_destroy(h)


@pytest.mark.slow
def test_grid1024_ll_application():
    """LL at the workload's size: 1,024 SSSPs on the 1024 x 1024 grid, labels for
    all 2^20 vertices, 2^20 queries; sampled labels and queries against the
    oracle's labels built from its own SSSP rows."""
    import bench
    g = inputs.workload_graph("grid1024_bfs_sssp")
    lms = inputs.workload_sources("grid1024_bfs_sssp", g)
    K = len(lms)
    st, h = fg.fg_graph_create_ex(g.n, g.m, g.row_ptr, g.col, g.w, 0, fg.fg_default_graph_opts(
        partition_method=fg.FG_PART_GROW))
    fg.check(st)
    try:
        s_d = torch.from_numpy(lms).to(DEV)
        dist = torch.empty((K, g.n), dtype=torch.int32, device=DEV)
        fg.check(fg.fg_sssp_batch(h, s_d, K, dist, None, fg.fg_default_opts(**bench.TUNED_SSSP)))
        lab = torch.empty((g.n, K), dtype=torch.int32, device=DEV)
        fg.check(fg.fg_ll_build_labels(dist, K, g.n, lab))
        del dist
        rng = np.random.default_rng(67)
        pairs = rng.integers(0, g.n, size=(1 << 20, 2)).astype(np.int32)
        got = _query_gpu(lab, g.n, K, pairs)
        ref = oracle.ll_labels(oracle.sssp(g, lms))
        vs = rng.choice(g.n, size=2000, replace=False)
        assert np.array_equal(lab[torch.from_numpy(vs).to(DEV)].cpu().numpy().view(np.uint32), ref[vs])
        sample = rng.choice(len(pairs), size=20000, replace=False)
        assert np.array_equal(got[sample], oracle.ll_query(ref, pairs[sample]))
    finally:
        fg.fg_graph_destroy(h)
