"""The applications' and DFS's hand-worked fixtures (tests/golden/apps_hand.txt,
with their derivations) against the oracle on the CPU and the CUDA path on the GPU."""
from fractions import Fraction
from pathlib import Path

import numpy as np
import pytest

import oracle
from paper_2103_14915_gb300 import inputs

FIX = Path(__file__).parent / "golden" / "apps_hand.txt"


def _fixture():
    bc, ll, ncp, dfs = [], [], {}, []
    for line in FIX.read_text().splitlines():
        if not line or line.startswith("#"):
            continue
        f = line.split()
        if f[0] == "bc":
            srcs = list(range(5)) if f[2] == "all" else [int(x) for x in f[2].split(",")]
            bc.append((f[1] == "1", srcs, np.array([float(x) for x in f[3:]])))
        elif f[0] == "ll":
            ll.append((int(f[1]), int(f[2]), int(f[3])))
        elif f[0] == "ncp" and f[1] == "order":
            ncp["order"] = [int(x) for x in f[2:]]
        elif f[0] == "ncp" and f[1] == "phi":
            ncp["phi"] = [float(Fraction(x)) for x in f[2:]]
        elif f[0] == "dfs":
            dfs.append((int(f[1]), [int(x) for x in f[2:]]))
    return bc, ll, ncp, dfs


def _g_bc():
    return inputs.from_edges(5, [(0, 1, 1), (1, 2, 1), (2, 3, 1), (1, 4, 1), (4, 3, 2)])


def _g_ncp():
    return inputs.from_edges(6, [(0, 1), (1, 2), (0, 2), (3, 4), (4, 5), (3, 5), (2, 3)])


P_NCP = np.array([0.5, 0.25, 0.375, 0.0625, 0.0, 0.03125], dtype=np.float32)


def test_oracle_bc_matches_the_hand_values():
    bc, _, _, _ = _fixture()
    g = _g_bc()
    for weighted, srcs, exp in bc:
        got, _, exact = oracle.bc(g, srcs, weighted)
        assert exact and np.array_equal(got, exp)


def test_oracle_ll_matches_the_hand_values():
    _, ll, _, _ = _fixture()
    lab = oracle.ll_labels(oracle.sssp(_g_bc(), [0, 3]))
    pairs = np.array([(u, v) for u, v, _ in ll], dtype=np.int32)
    assert oracle.ll_query(lab, pairs).tolist() == [e for _, _, e in ll]


def test_oracle_ncp_matches_the_hand_values():
    _, _, ncp, _ = _fixture()
    order, phi, count = oracle.ncp_sweep(_g_ncp(), P_NCP[None, :], 6)
    assert count[0] == 5 and order[0, :5].tolist() == ncp["order"]
    assert np.array_equal(phi[0, :5], np.array(ncp["phi"]))


def test_oracle_dfs_matches_the_hand_values():
    _, _, _, dfs = _fixture()
    for s, exp in dfs:
        assert oracle.dfs(_g_bc(), [s])[0].tolist() == exp


@pytest.mark.gpu
def test_cuda_path_matches_the_hand_values():
    torch = pytest.importorskip("torch")
    from paper_2103_14915_gb300 import build, fg
    build.build()
    fg.load()
    dev = "cuda:0"
    bc, ll, ncp, dfs = _fixture()
    g = _g_bc()
    st, h = fg.fg_graph_create_ex(g.n, g.m, g.row_ptr, g.col, g.w, 0, fg.fg_default_graph_opts())
    fg.check(st)
    try:
        for weighted, srcs, exp in bc:
            s_d = torch.tensor(srcs, dtype=torch.int32, device=dev)
            dist = torch.empty((len(srcs), g.n), dtype=torch.int32, device=dev)
            f = fg.fg_sssp_batch if weighted else fg.fg_bfs_batch
            fg.check(f(h, s_d, len(srcs), dist, None, None))
            out = torch.empty(g.n, dtype=torch.float64, device=dev)
            st, _ = fg.fg_bc_accumulate(h, s_d, len(srcs), dist, weighted, out)
            fg.check(st)
            assert np.array_equal(out.cpu().numpy(), exp)
        s_d = torch.tensor([0, 3], dtype=torch.int32, device=dev)
        dist = torch.empty((2, g.n), dtype=torch.int32, device=dev)
        fg.check(fg.fg_sssp_batch(h, s_d, 2, dist, None, None))
        lab = torch.empty((g.n, 2), dtype=torch.int32, device=dev)
        fg.check(fg.fg_ll_build_labels(dist, 2, g.n, lab))
        pairs = torch.tensor([(u, v) for u, v, _ in ll], dtype=torch.int32, device=dev)
        est = torch.empty(len(ll), dtype=torch.int64, device=dev)
        fg.check(fg.fg_ll_query(lab, g.n, 2, pairs, len(ll), est))
        fg.check(fg.fg_sync())
        assert est.cpu().tolist() == [e for _, _, e in ll]
        for src, exp in dfs:
            s1 = torch.tensor([src], dtype=torch.int32, device=dev)
            disc = torch.empty((1, g.n), dtype=torch.int32, device=dev)
            fg.check(fg.fg_dfs_batch(h, s1, 1, disc))
            assert disc[0].cpu().tolist() == exp
    finally:
        fg.fg_graph_destroy(h)
    g = _g_ncp()
    st, h = fg.fg_graph_create_ex(g.n, g.m, g.row_ptr, g.col, g.w, 0, fg.fg_default_graph_opts())
    fg.check(st)
    try:
        p = torch.from_numpy(P_NCP[None, :].copy()).to(dev)
        order = torch.empty((1, 6), dtype=torch.int32, device=dev)
        phi = torch.empty((1, 6), dtype=torch.float64, device=dev)
        cnt = torch.empty(1, dtype=torch.int32, device=dev)
        fg.check(fg.fg_ncp_sweep(h, p, 1, 6, order, phi, cnt))
        fg.check(fg.fg_sync())
        assert int(cnt[0]) == 5 and order[0, :5].cpu().tolist() == ncp["order"]
        assert np.array_equal(phi[0, :5].cpu().numpy(), np.array(ncp["phi"]))
    finally:
        fg.fg_graph_destroy(h)
