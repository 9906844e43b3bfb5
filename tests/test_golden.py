"""Hand-derived fixtures (tests/golden/): the oracle on the CPU and the CUDA path on the GPU
must reproduce values worked out from the definitions, independently of either implementation."""
from pathlib import Path

import numpy as np
import pytest

import oracle
from paper_2103_14915_gb300 import inputs

GOLDEN = Path(__file__).resolve().parent / "golden"
ALPHA = 0.15


def _lines(name):
    for ln in (GOLDEN / name).read_text().splitlines():
        ln = ln.strip()
        if ln and not ln.startswith("#"):
            yield ln.split()


def ppr_cases():
    for f in _lines("ppr_closed_forms.txt"):
        name, n, edges, src = f[0], int(f[1]), f[2], int(f[3])
        pi = np.array([float(x) for x in f[4:]])
        es = [tuple(int(x) for x in e.split("-")) for e in edges.split(",")]
        assert len(pi) == n
        yield name, inputs.from_edges(n, es), src, pi


def hand_graph():
    edges, rows = [], []
    for f in _lines("sssp_bfs_hand.txt"):
        if f[0] == "edge":
            edges.append((int(f[1]), int(f[2]), int(f[3])))
        else:
            rows.append((f[0], int(f[1]), np.array([int(x) for x in f[2:]], dtype=np.uint32)))
    return inputs.from_edges(7, edges), rows


@pytest.mark.parametrize("case", list(ppr_cases()), ids=lambda c: c[0])
def test_oracle_ppr_matches_closed_forms(case):
    name, g, src, pi = case
    got = oracle.ppr_power(g, [src], ALPHA)[0]
    # the power iteration stops at an L1 change below 1e-12, i.e. within ~6e-12 of pi
    assert np.allclose(got, pi, rtol=0, atol=1e-10)


def test_oracle_sssp_bfs_match_hand_values():
    g, rows = hand_graph()
    for kind, src, exp in rows:
        got = oracle.sssp(g, [src])[0] if kind == "sssp" else oracle.bfs(g, [src])[0]
        assert np.array_equal(got, exp), (kind, src)


@pytest.mark.gpu
def test_cuda_path_matches_hand_values():
    torch = pytest.importorskip("torch")
    from paper_2103_14915_gb300 import build, fg
    build.build()
    g, rows = hand_graph()
    st, h = fg.fg_graph_create_ex(g.n, g.m, g.row_ptr, g.col, g.w, 0, fg.fg_default_graph_opts())
    fg.check(st)
    try:
        for kind, src, exp in rows:
            s_d = torch.tensor([src], dtype=torch.int32, device="cuda:0")
            out = torch.empty((1, g.n), dtype=torch.int32, device="cuda:0")
            f = fg.fg_sssp_batch if kind == "sssp" else fg.fg_bfs_batch
            fg.check(f(h, s_d, 1, out, None, None))
            fg.check(fg.fg_sync())
            assert np.array_equal(out.cpu().numpy().view(np.uint32)[0], exp), (kind, src)
        for name, gp, src, pi in ppr_cases():
            st, hp = fg.fg_graph_create_ex(gp.n, gp.m, gp.row_ptr, gp.col, None, 0, fg.fg_default_graph_opts())
            fg.check(st)
            try:
                eps = 1e-7
                s_d = torch.tensor([src], dtype=torch.int32, device="cuda:0")
                p = torch.empty((1, gp.n), dtype=torch.float32, device="cuda:0")
                fg.check(fg.fg_ppr_batch(hp, s_d, 1, ALPHA, eps, p, None, None, None, None))
                fg.check(fg.fg_sync())
                deg = np.diff(gp.row_ptr).astype(np.float64)
                assert np.all(np.abs(p.cpu().numpy()[0].astype(np.float64) - pi) <= eps * deg + 1e-6), name
            finally:
                fg.fg_graph_destroy(hp)
    finally:
        fg.fg_graph_destroy(h)
