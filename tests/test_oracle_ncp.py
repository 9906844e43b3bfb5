"""Pins of the oracle's sweep cut (the NCP step over PPR vectors): brute force over explicit vertex
sets on small graphs, a closed form on two cliques joined by a bridge, zero conductance once the
sweep covers the seed's whole (smaller) component, and a planted mistake."""
import numpy as np
import pytest

import oracle
from paper_2103_14915_gb300 import inputs


def _brute(g, p, top):
    deg = np.diff(g.row_ptr)
    keys = [(np.float32(p[v]) / np.float32(max(int(deg[v]), 1)), v) for v in range(g.n) if p[v] > 0]
    order = [v for _, v in sorted(keys, key=lambda kv: (-kv[0], kv[1]))][:top]
    vol_all = int(deg.sum())
    phis = []
    for k in range(1, len(order) + 1):
        S = set(order[:k])
        cut = sum(1 for u in S for e in range(g.row_ptr[u], g.row_ptr[u + 1]) if int(g.col[e]) not in S)
        vol = sum(int(deg[u]) for u in S)
        den = min(vol, vol_all - vol)
        phis.append(cut / den if den > 0 else 1.0)
    return order, phis


@pytest.mark.parametrize("seed", range(6))
def test_sweep_matches_brute_force(seed):
    rng = np.random.default_rng(seed)
    n = 40
    edges = {(int(a), int(b)) for a, b in rng.integers(0, n, size=(90, 2)) if a != b}
    g = inputs.from_edges(n, sorted(edges))
    p = rng.random(n).astype(np.float32)
    p[rng.random(n) < 0.3] = 0.0          # vertices outside the support
    p[5] = p[6] = p[7]                    # equal keys where degrees agree: ties by id
    for top in (1, 7, n):
        order, phi, cnt = oracle.ncp_sweep(g, p[None, :], top)
        ref_order, ref_phi = _brute(g, p, top)
        assert cnt[0] == len(ref_order)
        assert order[0, :cnt[0]].tolist() == ref_order
        assert np.array_equal(phi[0, :cnt[0]], np.array(ref_phi))


def _two_cliques():
    a = [(i, j) for i in range(5) for j in range(i + 1, 5)]
    b = [(i + 5, j + 5) for i in range(5) for j in range(i + 1, 5)]
    return inputs.from_edges(10, a + b + [(4, 5)])


def test_two_cliques_closed_form():
    # the first clique (with the bridge endpoint) leads the sweep: cut 1, volume 5 * 4 + 1 = 21
    g = _two_cliques()
    p = np.array([0.5, 0.49, 0.48, 0.47, 0.5, 0.01, 0.009, 0.008, 0.007, 0.006], dtype=np.float32)
    order, phi, cnt = oracle.ncp_sweep(g, p[None, :], 10)
    assert cnt[0] == 10 and sorted(order[0, :5].tolist()) == [0, 1, 2, 3, 4]
    assert phi[0, 4] == 1.0 / 21.0
    assert phi[0, 4] == phi[0, :cnt[0] - 1].min()  # the best prefix is the clique


def test_planted_mistake_is_caught():
    g = _two_cliques()
    p = np.linspace(1.0, 0.1, 10).astype(np.float32)
    ok_order, ok_phi, _ = oracle.ncp_sweep(g, p[None, :], 10)
    oracle.set_mutation(6)  # internal arcs counted once
    try:
        _, bad_phi, _ = oracle.ncp_sweep(g, p[None, :], 10)
    finally:
        oracle.set_mutation(0)
    assert not np.array_equal(bad_phi, ok_phi)
    _, ref_phi = _brute(g, p, 10)
    assert np.array_equal(ok_phi[0], np.array(ref_phi))


def test_sweep_reaches_zero_conductance_at_the_seed_component():
    # two components: a 5-cycle with a chord (seeded) and a larger grid; PPR from the
    # cycle never leaves it, so the prefix that covers the cycle has no cut arcs
    cyc = [(i, (i + 1) % 5) for i in range(5)] + [(0, 2)]
    grid = inputs.grid(8, 8, 0, 0, seed=1)
    edges = cyc + [(5 + int(u), 5 + int(grid.col[e])) for u in range(grid.n)
                   for e in range(grid.row_ptr[u], grid.row_ptr[u + 1]) if u < grid.col[e]]
    g = inputs.from_edges(5 + grid.n, edges)
    p = oracle.ppr_push(g, 0, 0.15, 1e-8)[0].astype(np.float32)
    assert np.all(p[5:] == 0) and np.all(p[:5] > 0)
    order, phi, count = oracle.ncp_sweep(g, p[None, :], 64)
    assert count[0] == 5 and sorted(order[0, :5].tolist()) == [0, 1, 2, 3, 4]
    assert phi[0, 4] == 0.0 and np.all(phi[0, :4] > 0.0)
