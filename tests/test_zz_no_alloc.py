"""fg_sssp_batch_noalloc (fixed scratch, no allocation) against fg_sssp_batch.

Both are called through the C ABI on the same seeded inputs; distances are
integers, so the comparison is exact. The file name sorts last, so in a full
run it executes on a device that the other GPU tests have already used; it
also passes on its own.
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


def _create(g, method, S):
    go = fg.fg_default_graph_opts(partition_method=method, partition_vertices=S)
    st, h = fg.fg_graph_create_ex(g.n, g.m, g.row_ptr, g.col, g.w, 0, go)
    fg.check(st)
    return h


def _batch(h, g, s_d):
    out = torch.empty((len(s_d), g.n), dtype=torch.int32, device=DEV)
    fg.check(fg.fg_sssp_batch(h, s_d, len(s_d), out, None, fg.fg_default_opts(watchdog_ms=10000)))
    fg.check(fg.fg_sync())
    return out


def _noalloc(h, g, s_d, stream=None):
    out = torch.full((len(s_d), g.n), -7, dtype=torch.int32, device=DEV)  # every entry must be written
    torch.cuda.synchronize()
    fg.check(fg.fg_sssp_batch_noalloc(h, s_d, len(s_d), out, stream))
    return out


CASES = [
    ("rmat11-grow64", lambda: inputs.rmat(11, 16, seed=2, weights=(1, 255)), fg.FG_PART_GROW, 64),
    ("grid-range128", lambda: inputs.grid(48, 40, 500, 100, seed=4, weights=(100, 10000)), fg.FG_PART_RANGE, 128),
    ("rmat10-directed", lambda: inputs.rmat(10, 8, seed=3, directed=True, weights=(1, 255)), fg.FG_PART_AUTO, 0),
]


@pytest.mark.parametrize("name,make,method,S", CASES, ids=[c[0] for c in CASES])
def test_two_calls_in_a_row_match_fg_sssp_batch(name, make, method, S):
    g = make()
    h = _create(g, method, S)
    try:
        a = inputs.sources_uniform(g, 6, seed=11)
        a = np.concatenate([a, a[:1]]).astype(np.int32)  # a duplicate source
        b = inputs.sources_uniform(g, 5, seed=12).astype(np.int32)
        stream = torch.cuda.Stream()
        for srcs, strm in ((a, None), (b, stream)):
            s_d = torch.from_numpy(srcs).to(DEV)
            ref = _batch(h, g, s_d)
            got = _noalloc(h, g, s_d, strm)
            assert torch.equal(got, ref)
        # and against the oracle on the last call's first rows
        exp = oracle.sssp(g, b[:2])
        assert np.array_equal(got.cpu().numpy().view(np.uint32)[:2], exp)
    finally:
        fg.fg_graph_destroy(h)


def test_largest_supported_graph():
    # the road-like 1024 x 1024 grid has exactly FG_NOALLOC_MAX_VERTICES vertices
    g = inputs.grid(1024, 1024, 500, 100, seed=2, weights=(100, 10000))
    assert g.n == fg.FG_NOALLOC_MAX_VERTICES
    h = _create(g, fg.FG_PART_GROW, 1024)
    try:
        s_d = torch.from_numpy(inputs.sources_uniform(g, 2, seed=5).astype(np.int32)).to(DEV)
        assert torch.equal(_noalloc(h, g, s_d), _batch(h, g, s_d))
    finally:
        fg.fg_graph_destroy(h)


def test_rejects_graph_beyond_the_scratch():
    g = inputs.grid(1, fg.FG_NOALLOC_MAX_VERTICES + 1, 0, 0, seed=1)  # a path
    h = _create(g, fg.FG_PART_RANGE, 1024)
    try:
        s_d = torch.zeros(1, dtype=torch.int32, device=DEV)
        out = torch.empty(g.n, dtype=torch.int32, device=DEV)
        assert fg.fg_sssp_batch_noalloc(h, s_d, 1, out) == fg.FG_ERR_UNSUPPORTED
        assert str(fg.FG_NOALLOC_MAX_VERTICES) in fg.fg_last_error()
    finally:
        fg.fg_graph_destroy(h)


def test_device_side_error_then_next_call_is_clean():
    g = inputs.rmat(9, 8, seed=7, weights=(1, 255))
    h = _create(g, fg.FG_PART_RANGE, 64)
    try:
        bad = torch.tensor([0, g.n], dtype=torch.int32, device=DEV)  # second id out of range
        out = torch.empty((2, g.n), dtype=torch.int32, device=DEV)
        assert fg.fg_sssp_batch_noalloc(h, bad, 2, out) == fg.FG_ERR_INVALID_ARG
        s_d = torch.tensor([3, 17], dtype=torch.int32, device=DEV)
        assert torch.equal(_noalloc(h, g, s_d), _batch(h, g, s_d))
    finally:
        fg.fg_graph_destroy(h)


def test_host_side_argument_checks():
    g = inputs.rmat(8, 8, seed=1)
    h = _create(g, fg.FG_PART_RANGE, 64)
    try:
        s_d = torch.zeros(2, dtype=torch.int32, device=DEV)
        out = torch.empty((2, g.n), dtype=torch.int32, device=DEV)
        assert fg.fg_sssp_batch_noalloc(h, s_d, 0, out) == fg.FG_ERR_INVALID_ARG
        assert fg.fg_sssp_batch_noalloc(h, None, 2, out) == fg.FG_ERR_INVALID_ARG
        assert fg.fg_sssp_batch_noalloc(h, s_d, 2, out.data_ptr() + 2) == fg.FG_ERR_INVALID_ARG
    finally:
        fg.fg_graph_destroy(h)


def test_call_after_graph_creation_adds_no_device_memory():
    # graph creation placed the scratch; the call itself must take nothing
    g = inputs.rmat(10, 8, seed=21, weights=(1, 255))
    h = _create(g, fg.FG_PART_RANGE, 64)
    try:
        s_d = torch.from_numpy(inputs.sources_uniform(g, 3, seed=2).astype(np.int32)).to(DEV)
        out = torch.empty((3, g.n), dtype=torch.int32, device=DEV)
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        fg.check(fg.fg_sssp_batch_noalloc(h, s_d, 3, out))
        free1 = torch.cuda.mem_get_info()[0]
        assert free1 == free0
        assert torch.equal(out, _batch(h, g, s_d))
    finally:
        fg.fg_graph_destroy(h)

