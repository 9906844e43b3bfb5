"""CPU oracle -- TEST INFRASTRUCTURE ONLY.

Plain, slow reference implementations of the per-source queries of the
fork-processing pattern (Alg. 1, Def. 2.2): Dijkstra SSSP, queue BFS levels,
FP64 power-iteration PPR and an FP64 sequential push, plus implementation-free
certificate checks; and of what is built on them: the NCP sweep, landmark
labels and queries, sampled betweenness centrality (Sec. 1, 6.1), random
walks and DFS (Sec. 3). Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` (which time this oracle and
check sampled outputs against it) may import this package. It shares no code
with the CUDA path and never imports it.

Parity pins (what ties this oracle to something other than itself) live in
``tests/test_oracle.py`` (SSSP, BFS, PPR, certificates),
``tests/test_oracle_ncp.py``, ``test_oracle_ll.py``, ``test_oracle_bc.py``,
``test_oracle_rw.py``, ``test_oracle_dfs.py`` and the hand-worked fixtures of
``tests/golden/``; every function here is pinned there. The PPR sequential
push (``ppr_push``) is order-dependent by design: its per-vertex values are
checked only against the error bound, never element by element.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from pathlib import Path

import numpy as np

_HERE = Path(__file__).resolve().parent
_SRC = _HERE / "oracle.c"
_LIB = _HERE / "_oracle.so"
_lib = None

UNREACHED = np.uint32(0xFFFFFFFF)


def build(force: bool = False) -> Path:
    """Compile oracle.c (gcc -O2, OpenMP over queries) into an in-tree .so."""
    if force or not _LIB.exists() or _LIB.stat().st_mtime < _SRC.stat().st_mtime:
        tmp = _LIB.with_suffix(f".{os.getpid()}.tmp")
        subprocess.run(["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-shared", "-fPIC", "-std=c11", str(_SRC), "-lm",
                        "-o", str(tmp)], check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(str(_LIB))
        p = ctypes.c_void_p
        i32, i64, f64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_double
        lib.orc_set_mutation.argtypes = [ctypes.c_int]
        lib.orc_num_threads.restype = ctypes.c_int
        lib.orc_sssp.argtypes = [i64, p, p, p, i32, p]
        lib.orc_bfs.argtypes = [i64, p, p, i32, p]
        lib.orc_sssp_batch.argtypes = [i64, p, p, p, i32, p, p]
        lib.orc_bfs_batch.argtypes = [i64, p, p, i32, p, p]
        lib.orc_ppr_power.argtypes = [i64, p, p, i32, f64, f64, ctypes.c_int, p]
        lib.orc_ppr_power_batch.argtypes = [i64, p, p, i32, p, f64, f64, ctypes.c_int, p]
        lib.orc_ppr_push.argtypes = [i64, p, p, i32, f64, f64, p, p]
        lib.orc_ppr_push.restype = i64
        lib.orc_sssp_certificate.argtypes = [i64, p, p, p, i32, p]
        lib.orc_bfs_certificate.argtypes = [i64, p, p, i32, p]
        lib.orc_certificate_batch.argtypes = [i64, p, p, p, i32, p, p]
        lib.orc_ncp_sweep_batch.argtypes = [i64, p, p, i32, p, i32, p, p, p]
        lib.orc_ll_query.argtypes = [i64, i32, p, i64, p, p]
        lib.orc_bc_batch.argtypes = [i64, p, p, p, ctypes.c_int, i32, p, p, p]
        lib.orc_splitmix64.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
        lib.orc_splitmix64.restype = ctypes.c_uint64
        lib.orc_rw_batch.argtypes = [i64, p, p, i32, p, i32, ctypes.c_uint64, p]
        lib.orc_dfs_batch.argtypes = [i64, p, p, i32, p, p]
        lib.orc_certificate_batch.restype = i64
        _lib = lib
    return _lib


def _p(a):
    if a is None:
        return None
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.c_void_p)


def _csr(g):
    rp = np.ascontiguousarray(g.row_ptr, dtype=np.int64)
    col = np.ascontiguousarray(g.col, dtype=np.int32)
    w = None if g.w is None else np.ascontiguousarray(g.w, dtype=np.int32)
    return rp, col, w


def num_threads() -> int:
    return int(_load().orc_num_threads())


def set_mutation(k: int) -> None:
    """Plant a known mistake (tests only): 1 ignore weights, 2 skip last arc,
    3 BFS levels start at 1, 4 PPR transposed operand, 5 PPR drops dangling mass,
    6 sweep counts internal arcs once, 7 LL query ignores unreachable landmarks' sentinel,
    8 BC dependency drops the 1 of (1 + delta(w)), 9 random walks draw output k - 1,
    10 DFS scans each vertex's neighbours from the last arc."""
    _load().orc_set_mutation(int(k))


def sssp(g, srcs) -> np.ndarray:
    """Dijkstra distances, query-major uint32[nq, n]; UINT32_MAX = unreachable."""
    lib = _load()
    rp, col, w = _csr(g)
    srcs = np.ascontiguousarray(np.atleast_1d(srcs), dtype=np.int32)
    out = np.empty((srcs.size, g.n), dtype=np.uint32)
    rc = lib.orc_sssp_batch(g.n, _p(rp), _p(col), _p(w), srcs.size, _p(srcs), _p(out))
    if rc != 0:
        raise RuntimeError(f"orc_sssp_batch failed ({rc})")
    return out


def bfs(g, srcs) -> np.ndarray:
    """BFS levels, query-major uint32[nq, n]; UINT32_MAX = unreachable."""
    lib = _load()
    rp, col, _ = _csr(g)
    srcs = np.ascontiguousarray(np.atleast_1d(srcs), dtype=np.int32)
    out = np.empty((srcs.size, g.n), dtype=np.uint32)
    rc = lib.orc_bfs_batch(g.n, _p(rp), _p(col), srcs.size, _p(srcs), _p(out))
    if rc != 0:
        raise RuntimeError(f"orc_bfs_batch failed ({rc})")
    return out


def ppr_power(g, srcs, alpha: float, tol: float = 1e-12, max_iter: int = 100000) -> np.ndarray:
    """FP64 PPR vectors by power iteration, float64[nq, n]."""
    lib = _load()
    rp, col, _ = _csr(g)
    srcs = np.ascontiguousarray(np.atleast_1d(srcs), dtype=np.int32)
    out = np.empty((srcs.size, g.n), dtype=np.float64)
    rc = lib.orc_ppr_power_batch(g.n, _p(rp), _p(col), srcs.size, _p(srcs), alpha, tol, max_iter, _p(out))
    if rc < 0:
        raise RuntimeError(f"orc_ppr_power_batch failed ({rc})")
    return out


def ppr_push(g, src: int, alpha: float, eps: float):
    """FP64 sequential push (largest residual first). Returns (p, r, pushes)."""
    lib = _load()
    rp, col, _ = _csr(g)
    p = np.empty(g.n, dtype=np.float64)
    r = np.empty(g.n, dtype=np.float64)
    k = lib.orc_ppr_push(g.n, _p(rp), _p(col), int(src), alpha, eps, _p(p), _p(r))
    if k < 0:
        raise RuntimeError(f"orc_ppr_push failed ({k})")
    return p, r, int(k)


def sssp_certificate(g, src: int, dist: np.ndarray) -> int:
    lib = _load()
    rp, col, w = _csr(g)
    d = np.ascontiguousarray(dist, dtype=np.uint32)
    return int(lib.orc_sssp_certificate(g.n, _p(rp), _p(col), _p(w), int(src), _p(d)))


def bfs_certificate(g, src: int, level: np.ndarray) -> int:
    lib = _load()
    rp, col, _ = _csr(g)
    d = np.ascontiguousarray(level, dtype=np.uint32)
    return int(lib.orc_bfs_certificate(g.n, _p(rp), _p(col), int(src), _p(d)))


def certificate_batch(g, srcs, out: np.ndarray, weighted: bool) -> int:
    """0 if every query's array passes its certificate, else (code << 20) + first failing query."""
    lib = _load()
    rp, col, w = _csr(g)
    srcs = np.ascontiguousarray(np.atleast_1d(srcs), dtype=np.int32)
    o = np.ascontiguousarray(out, dtype=np.uint32)
    return int(lib.orc_certificate_batch(g.n, _p(rp), _p(col), _p(w) if weighted else None, srcs.size,
                                         _p(srcs), _p(o)))


def reachable_arcs(g, dist_row: np.ndarray) -> int:
    """Arcs whose tail is reachable (the edges a sequential Dijkstra/BFS scans)."""
    deg = np.diff(g.row_ptr)
    return int(deg[dist_row != UNREACHED].sum())


def ncp_sweep(g, p_rows: np.ndarray, top: int):
    """Sweep cuts over PPR vectors (rows of p_rows). Returns (order int32[nq, top],
    phi float64[nq, top], count int32[nq]); entries past count are unused."""
    lib = _load()
    rp, col, _ = _csr(g)
    pr = np.ascontiguousarray(np.atleast_2d(p_rows), dtype=np.float32)
    nq = pr.shape[0]
    order = np.full((nq, top), -1, dtype=np.int32)
    phi = np.full((nq, top), np.nan, dtype=np.float64)
    count = np.zeros(nq, dtype=np.int32)
    r = lib.orc_ncp_sweep_batch(g.n, _p(rp), _p(col), nq, _p(pr), int(top), _p(order), _p(phi), _p(count))
    if r != 0:
        raise RuntimeError(f"orc_ncp_sweep_batch failed ({r})")
    return order, phi, count


def ll_labels(dist_rows: np.ndarray) -> np.ndarray:
    """Label construction of landmark labeling: the batch's distance rows
    (query-major uint32[K, n], row k = d(s_k, .)) as per-vertex labels
    (vertex-major uint32[n, K]): labels[v, k] = d(s_k, v)."""
    return np.ascontiguousarray(np.asarray(dist_rows, dtype=np.uint32).T)


def ll_query(labels: np.ndarray, pairs: np.ndarray) -> np.ndarray:
    """Landmark distance estimates for pairs (int32[Q, 2]): min over landmarks
    reaching both of d(s, u) + d(s, v) (uint64), UINT64_MAX when none does."""
    lib = _load()
    lab = np.ascontiguousarray(labels, dtype=np.uint32)
    pr = np.ascontiguousarray(pairs, dtype=np.int32).reshape(-1, 2)
    out = np.empty(pr.shape[0], dtype=np.uint64)
    r = lib.orc_ll_query(lab.shape[0], lab.shape[1], _p(lab), pr.shape[0], _p(pr), _p(out))
    if r != 0:
        raise ValueError("vertex id out of range")
    return out


def bc(g, srcs, weighted: bool):
    """Betweenness centrality from the sources srcs (Brandes' dependencies summed
    over the sources in order): returns (bc float64[n], sigma_max, exact), exact
    False when some shortest-path count reached 2^53."""
    lib = _load()
    rp, col, w = _csr(g)
    srcs = np.ascontiguousarray(np.atleast_1d(srcs), dtype=np.int32)
    out = np.empty(g.n, dtype=np.float64)
    smax = np.zeros(1, dtype=np.float64)
    r = lib.orc_bc_batch(g.n, _p(rp), _p(col), _p(w) if weighted else None, 1 if weighted else 0, srcs.size,
                         _p(srcs), _p(out), _p(smax))
    if r < 0:
        raise ValueError(f"orc_bc_batch failed ({r})")
    return out, float(smax[0]), r == 0


def splitmix64(seed: int, k: int) -> int:
    """Output number k (>= 1) of the SplitMix64 stream whose state starts at seed."""
    return int(_load().orc_splitmix64(seed & ((1 << 64) - 1), k))


def rw(g, srcs, length: int, seed: int) -> np.ndarray:
    """Random walks: int32[nq, length + 1], -1 after a vertex without out-arcs."""
    lib = _load()
    rp, col, _ = _csr(g)
    srcs = np.ascontiguousarray(np.atleast_1d(srcs), dtype=np.int32)
    out = np.empty((srcs.size, length + 1), dtype=np.int32)
    r = lib.orc_rw_batch(g.n, _p(rp), _p(col), srcs.size, _p(srcs), int(length), seed & ((1 << 64) - 1), _p(out))
    if r != 0:
        raise ValueError("source out of range")
    return out


def dfs(g, srcs) -> np.ndarray:
    """DFS discovery ranks, uint32[nq, n] (UINT32_MAX = not reached)."""
    lib = _load()
    rp, col, _ = _csr(g)
    srcs = np.ascontiguousarray(np.atleast_1d(srcs), dtype=np.int32)
    out = np.empty((srcs.size, g.n), dtype=np.uint32)
    if lib.orc_dfs_batch(g.n, _p(rp), _p(col), srcs.size, _p(srcs), _p(out)) != 0:
        raise ValueError("source out of range or allocation failed")
    return out
