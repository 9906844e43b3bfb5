"""Seeded synthetic graph inputs, shared by the CPU oracle tests and the CUDA path.

This module draws graphs, weights and source vertices and nothing else: it holds
no arithmetic of the query method. The paper measures on real road and social
graphs (Sec. 6.1, Table 2); the generators here are synthetic stand-ins with the
same structure:

* ``rmat``  -- R-MAT power-law graphs with randomly permuted vertex ids, so that
  equal-size id ranges act as the random equal-vertex partitions the paper uses
  for social graphs (Sec. 6.1, Implementation Details).
* ``grid``  -- a road-like 2-D grid with 5% dropped edges and 1% diagonal shortcuts.
* ``sources_uniform`` / ``sources_logdeg`` -- query sources (uniform among
  non-isolated vertices; or spread evenly over log2-degree buckets for PPR seeds).

The native part (``graphgen.c``) is compiled with gcc by :func:`build`.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import subprocess
import sys
from pathlib import Path

import numpy as np

_HERE = Path(__file__).resolve().parent
_SRC = _HERE / "graphgen.c"
_LIB = _HERE / "_graphgen.so"
_lib = None


def build(force: bool = False) -> Path:
    """Compile graphgen.c into an in-tree shared library (gcc, OpenMP)."""
    if force or not _LIB.exists() or _LIB.stat().st_mtime < _SRC.stat().st_mtime:
        tmp = _LIB.with_suffix(f".{os.getpid()}.tmp")
        cmd = ["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-std=c11", str(_SRC), "-o", str(tmp)]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(str(_LIB))
        p = ctypes.c_void_p
        i32, i64, u32, u64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32, ctypes.c_uint64
        lib.fgg_rmat_edges.argtypes = [ctypes.c_int, ctypes.c_int, u32, u32, u32, u64, p, p]
        lib.fgg_grid_edges.argtypes = [i32, i32, u32, u32, u64, p, p, p]
        lib.fgg_csr_build.argtypes = [i64, i64, p, p, ctypes.c_int, p, p, p]
        lib.fgg_weights.argtypes = [i64, p, p, i32, i32, u64, p]
        lib.fgg_sources_uniform.argtypes = [i64, p, i32, u64, p]
        lib.fgg_sources_logdeg.argtypes = [i64, p, i32, u64, p]
        for f in (lib.fgg_rmat_edges, lib.fgg_grid_edges, lib.fgg_csr_build, lib.fgg_weights,
                  lib.fgg_sources_uniform, lib.fgg_sources_logdeg):
            f.restype = ctypes.c_int
        _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.c_void_p)


@dataclasses.dataclass
class Graph:
    """Host CSR graph: row_ptr int64[n+1], col int32[m], w int32[m] or None."""

    n: int
    row_ptr: np.ndarray
    col: np.ndarray
    w: np.ndarray | None
    directed: bool
    name: str = ""

    @property
    def m(self) -> int:
        return int(self.row_ptr[-1])

    def out_degree(self) -> np.ndarray:
        return np.diff(self.row_ptr)


def csr_from_edges(n: int, src: np.ndarray, dst: np.ndarray, symmetrize: bool) -> tuple[np.ndarray, np.ndarray]:
    """Deduplicated, self-loop-free CSR with sorted adjacency lists."""
    lib = _load()
    src = np.ascontiguousarray(src, dtype=np.uint32)
    dst = np.ascontiguousarray(dst, dtype=np.uint32)
    m = src.shape[0]
    row_ptr = np.empty(n + 1, dtype=np.int64)
    col = np.empty(max(1, (2 if symmetrize else 1) * m), dtype=np.int32)
    mo = ctypes.c_int64(0)
    rc = lib.fgg_csr_build(n, m, _ptr(src), _ptr(dst), int(symmetrize), _ptr(row_ptr), _ptr(col),
                           ctypes.byref(mo))
    if rc != 0:
        raise ValueError(f"fgg_csr_build failed ({rc})")
    return row_ptr, col[: mo.value].copy()


def add_weights(g: Graph, lo: int, hi: int, seed: int) -> Graph:
    lib = _load()
    w = np.empty(max(1, g.m), dtype=np.int32)
    rc = lib.fgg_weights(g.n, _ptr(g.row_ptr), _ptr(g.col), lo, hi, seed, _ptr(w))
    if rc != 0:
        raise ValueError("fgg_weights failed")
    g.w = w[: g.m]
    return g


def rmat(scale: int, edge_factor: int = 16, seed: int = 1, directed: bool = False,
         abc=(5700, 1900, 1900), weights: tuple[int, int] | None = None) -> Graph:
    """R-MAT graph with 2^scale vertices and edge_factor * 2^scale generated edges.

    a/b/c/d default to 0.57/0.19/0.19/0.05 (given per 10000). Undirected graphs
    store both arcs of every edge. Self-loops and duplicates are removed.
    """
    lib = _load()
    n = 1 << scale
    m = edge_factor * n
    src = np.empty(m, dtype=np.uint32)
    dst = np.empty(m, dtype=np.uint32)
    rc = lib.fgg_rmat_edges(scale, edge_factor, abc[0], abc[1], abc[2], seed, _ptr(src), _ptr(dst))
    if rc != 0:
        raise ValueError(f"fgg_rmat_edges failed ({rc})")
    row_ptr, col = csr_from_edges(n, src, dst, symmetrize=not directed)
    del src, dst
    g = Graph(n, row_ptr, col, None, directed, name=f"rmat{scale}_ef{edge_factor}{'_dir' if directed else ''}")
    if weights is not None:
        add_weights(g, weights[0], weights[1], seed ^ 0x5EED)
    return g


def grid(rows: int = 1024, cols: int = 1024, drop_per_10000: int = 500, diag_per_10000: int = 100,
         seed: int = 2, weights: tuple[int, int] | None = None) -> Graph:
    """Road-like undirected grid, id = r*cols + c (5% edges dropped, 1% diagonal shortcuts)."""
    lib = _load()
    n = rows * cols
    cap = 3 * n
    src = np.empty(cap, dtype=np.uint32)
    dst = np.empty(cap, dtype=np.uint32)
    mo = ctypes.c_int64(0)
    rc = lib.fgg_grid_edges(rows, cols, drop_per_10000, diag_per_10000, seed, _ptr(src), _ptr(dst),
                            ctypes.byref(mo))
    if rc != 0:
        raise ValueError("fgg_grid_edges failed")
    row_ptr, col = csr_from_edges(n, src[: mo.value], dst[: mo.value], symmetrize=True)
    g = Graph(n, row_ptr, col, None, False, name=f"grid{rows}x{cols}")
    if weights is not None:
        add_weights(g, weights[0], weights[1], seed ^ 0x5EED)
    return g


def from_edges(n: int, edges, directed: bool = False, weights=None, name: str = "") -> Graph:
    """Small hand-built graph from an edge list [(u, v[, w]), ...].

    With explicit weights, the weight of each arc is the one given for its
    edge (for undirected graphs both arcs take it).
    """
    edges = list(edges)
    src = np.array([e[0] for e in edges], dtype=np.uint32)
    dst = np.array([e[1] for e in edges], dtype=np.uint32)
    row_ptr, col = csr_from_edges(n, src, dst, symmetrize=not directed)
    g = Graph(n, row_ptr, col, None, directed, name=name)
    if edges and len(edges[0]) == 3:
        wmap = {}
        for u, v, w in edges:
            wmap[(u, v)] = w
            if not directed:
                wmap[(v, u)] = w
        w = np.empty(g.m, dtype=np.int32)
        for u in range(n):
            for e in range(g.row_ptr[u], g.row_ptr[u + 1]):
                w[e] = wmap[(u, int(g.col[e]))]
        g.w = w
    elif weights is not None:
        add_weights(g, weights[0], weights[1], 7)
    return g


def sources_uniform(g: Graph, k: int, seed: int) -> np.ndarray:
    """k distinct sources, uniform among vertices with out-degree >= 1."""
    lib = _load()
    out = np.empty(max(1, k), dtype=np.int32)
    rc = lib.fgg_sources_uniform(g.n, _ptr(g.row_ptr), k, seed, _ptr(out))
    if rc != 0:
        raise ValueError("not enough candidate sources")
    return out[:k].copy()


def sources_logdeg(g: Graph, k: int, seed: int) -> np.ndarray:
    """k distinct seeds spread evenly over floor(log2(out-degree)) buckets."""
    lib = _load()
    out = np.empty(max(1, k), dtype=np.int32)
    rc = lib.fgg_sources_logdeg(g.n, _ptr(g.row_ptr), k, seed, _ptr(out))
    if rc != 0:
        raise ValueError("not enough candidate seeds")
    return out[:k].copy()



def ncp_seeds(g: Graph, fraction: float = 1e-4, seed: int = 7) -> np.ndarray:
    """PPR seeds of the NCP application: round(fraction * n) distinct vertices,
    uniform among those with out-degree >= 1 (Sec. 6.1 seeds 0.01% of V)."""
    return sources_uniform(g, max(1, round(fraction * g.n)), seed)

# ---------------------------------------------------------------------------
# The five workloads (sizes from the paper's applications: LL runs 1,024
# SSSPs, BC ~100 sources, NCP thousands of PPRs; Sec. 6.1).
# ---------------------------------------------------------------------------

WORKLOAD_SEEDS = {
    "rmat14_plain_sssp": 14,
    "grid1024_bfs_sssp": 1024,
    "rmat22_ppr": 22,
    "rmat24_sssp": 24,
    "rmat25_serving": 25,
}


def workload_graph(name: str) -> Graph:
    s = WORKLOAD_SEEDS[name]
    if name == "rmat14_plain_sssp":
        return rmat(14, 16, seed=s, weights=(1, 255))
    if name == "grid1024_bfs_sssp":
        return grid(1024, 1024, 500, 100, seed=s, weights=(100, 10000))
    if name == "rmat22_ppr":
        return rmat(22, 16, seed=s)
    if name == "rmat24_sssp":
        return rmat(24, 16, seed=s, weights=(1, 255))
    if name == "rmat25_serving":
        return rmat(25, 24, seed=s, directed=True, weights=(1, 255))
    raise KeyError(name)


def workload_sources(name: str, g: Graph, k: int | None = None, set_index: int = 0) -> np.ndarray:
    base = {"rmat14_plain_sssp": 64, "grid1024_bfs_sssp": 1024, "rmat22_ppr": 4096,
            "rmat24_sssp": 16384, "rmat25_serving": 100000}[name]
    k = base if k is None else k
    seed = 1000 * WORKLOAD_SEEDS[name] + set_index
    if name == "rmat22_ppr":
        return sources_logdeg(g, k, seed)
    return sources_uniform(g, k, seed)
