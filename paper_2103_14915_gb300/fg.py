"""Thin ctypes binding of the C ABI in ``include/fg.h`` (argument marshalling only).

Every function has the name of its C entry point and returns the C status code
(``FG_OK`` = 0); :func:`check` turns a code into an exception carrying
``fg_last_error()``. Buffers may be torch tensors (device memory, via
``data_ptr()``), numpy arrays (host memory, for ``host_io`` calls) or raw
integer addresses. Streams are ``torch.cuda.Stream`` objects, raw handles, or
None for the legacy default stream.

The shared library is built in-tree by :func:`paper_2103_14915_gb300.build.build`;
loading fails loudly if it is missing -- there is no fallback path.
"""
from __future__ import annotations

import ctypes
from pathlib import Path

_LIB_PATH = Path(__file__).resolve().parent / "libfg.so"
_lib = None

FG_OK = 0
FG_ERR_INVALID_ARG = 1
FG_ERR_OOM = 2
FG_ERR_CUDA = 3
FG_ERR_TIMEOUT = 4
FG_ERR_BIN_OVERFLOW = 5
FG_ERR_OVERFLOW = 6
FG_ERR_UNSUPPORTED = 7
STATUS_NAMES = {0: "FG_OK", 1: "FG_ERR_INVALID_ARG", 2: "FG_ERR_OOM", 3: "FG_ERR_CUDA", 4: "FG_ERR_TIMEOUT",
                5: "FG_ERR_BIN_OVERFLOW", 6: "FG_ERR_OVERFLOW", 7: "FG_ERR_UNSUPPORTED"}

FG_DEVICE_PTRS = 0x1
FG_PART_AUTO, FG_PART_RANGE, FG_PART_GROW, FG_PART_DEGREE = 0, 1, 2, 3
FG_SCHED_FIFO, FG_SCHED_PRIORITY, FG_SCHED_MAXOPS, FG_SCHED_RANDOM = 0, 1, 2, 3
FG_MODE_BUFFERED, FG_MODE_PLAIN = 0, 1


class fg_graph_opts(ctypes.Structure):
    _fields_ = [("struct_size", ctypes.c_uint32), ("partition_method", ctypes.c_int32),
                ("partition_vertices", ctypes.c_int32)]


class fg_opts(ctypes.Structure):
    _fields_ = [("struct_size", ctypes.c_uint32), ("mode", ctypes.c_int32), ("sched", ctypes.c_int32),
                ("sched_window", ctypes.c_uint32), ("delta", ctypes.c_uint32), ("bucket", ctypes.c_uint32),
                ("yield_edges", ctypes.c_uint64), ("max_rounds", ctypes.c_uint32),
                ("watchdog_ms", ctypes.c_uint32), ("emit_capacity", ctypes.c_uint64),
                ("host_io", ctypes.c_int32), ("query_batch", ctypes.c_int32), ("threads_per_vertex", ctypes.c_int32),
                ("group", ctypes.c_int32), ("group_order", ctypes.c_int32), ("check_staging", ctypes.c_int32)]


class fg_stats_t(ctypes.Structure):
    _fields_ = [(k, ctypes.c_uint64) for k in
                ("rounds", "visits", "edges", "ops", "spills", "yields", "launches", "max_round_ops")] + [
                   ("phase_ns", ctypes.c_uint64 * 6), ("arcs_read", ctypes.c_uint64), ("group", ctypes.c_uint64)]

    PHASES = ("init_tiles", "seed", "scan_a", "scan_b", "scatter", "process")

    def as_dict(self):
        d = {k: int(getattr(self, k)) for k, _ in self._fields_ if k != "phase_ns"}
        d["phase_ms"] = {n: round(self.phase_ns[i] / 1e6, 3) for i, n in enumerate(self.PHASES)}
        return d


FG_QUERY_SSSP, FG_QUERY_BFS, FG_QUERY_PPR = 0, 1, 2


class fg_tune_report(ctypes.Structure):
    _fields_ = [("candidates", ctypes.c_int32), ("best_ms", ctypes.c_float), ("default_ms", ctypes.c_float)]


class fg_server_opts(ctypes.Structure):
    _fields_ = [("struct_size", ctypes.c_uint32), ("lanes", ctypes.c_int32), ("max_batch", ctypes.c_int32),
                ("full_grid", ctypes.c_int32), ("alpha", ctypes.c_float), ("eps", ctypes.c_float),
                ("hbm_budget", ctypes.c_int64), ("opts", fg_opts * 3),
                ("continuous", ctypes.c_int32), ("slots", ctypes.c_int32)]


class fg_request_info(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("source", ctypes.c_int32), ("status", ctypes.c_int32),
                ("batch_size", ctypes.c_int32), ("submit_ns", ctypes.c_int64), ("launch_ns", ctypes.c_int64),
                ("done_ns", ctypes.c_int64), ("result", ctypes.c_void_p), ("residual", ctypes.c_void_p),
                ("mass", ctypes.c_double)]


class fg_bc_info_t(ctypes.Structure):
    _fields_ = [("waves", ctypes.c_int32), ("inexact", ctypes.c_int32), ("sigma_max", ctypes.c_double)]


class fg_graph_info_t(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("m", ctypes.c_int64), ("partition_vertices", ctypes.c_int32),
                ("num_partitions", ctypes.c_int32), ("partition_method", ctypes.c_int32),
                ("weighted", ctypes.c_int32), ("cut_arcs", ctypes.c_int64), ("device_bytes", ctypes.c_int64)]


EXPORTS = ("fg_default_opts", "fg_default_graph_opts", "fg_graph_create", "fg_graph_create_ex",
           "fg_graph_destroy", "fg_graph_info", "fg_sssp_batch", "fg_bfs_batch", "fg_ppr_batch", "fg_sync",
           "fg_last_error", "fg_stats", "fg_partition_plan", "fg_sssp_batch_noalloc", "fg_default_server_opts",
           "fg_server_create", "fg_server_destroy", "fg_server_submit", "fg_server_poll", "fg_server_info",
           "fg_server_release", "fg_tune_opts", "fg_tune_opts_ex", "fg_ncp_sweep", "fg_ll_build_labels",
           "fg_ll_query", "fg_bc_accumulate", "fg_rw_batch", "fg_dfs_batch", "fg_ppr_local_batch")

FG_NOALLOC_MAX_VERTICES = 1 << 20
FG_NCP_MAX_TOP = 4096


def lib_path() -> Path:
    return _LIB_PATH


def load():
    """Load libfg.so (built in-tree). Raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not _LIB_PATH.exists():
        raise RuntimeError(f"{_LIB_PATH} is missing: build it with paper_2103_14915_gb300.build.build()")
    lib = ctypes.CDLL(str(_LIB_PATH))
    vp, i32, i64, u32, f32 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32, ctypes.c_float
    lib.fg_default_opts.argtypes = [ctypes.POINTER(fg_opts)]
    lib.fg_default_opts.restype = None
    lib.fg_default_graph_opts.argtypes = [ctypes.POINTER(fg_graph_opts)]
    lib.fg_default_graph_opts.restype = None
    lib.fg_graph_create.argtypes = [i64, i64, vp, vp, vp, u32, ctypes.POINTER(vp)]
    lib.fg_graph_create_ex.argtypes = [i64, i64, vp, vp, vp, u32, ctypes.POINTER(fg_graph_opts), ctypes.POINTER(vp)]
    lib.fg_graph_destroy.argtypes = [vp]
    lib.fg_graph_info.argtypes = [vp, ctypes.POINTER(fg_graph_info_t)]
    lib.fg_sssp_batch.argtypes = [vp, vp, i32, vp, vp, ctypes.POINTER(fg_opts)]
    lib.fg_bfs_batch.argtypes = [vp, vp, i32, vp, vp, ctypes.POINTER(fg_opts)]
    lib.fg_ppr_batch.argtypes = [vp, vp, i32, f32, f32, vp, vp, vp, vp, ctypes.POINTER(fg_opts)]
    lib.fg_sync.argtypes = [vp]
    lib.fg_last_error.argtypes = []
    lib.fg_last_error.restype = ctypes.c_char_p
    lib.fg_stats.argtypes = [vp, ctypes.POINTER(fg_stats_t)]
    lib.fg_partition_plan.argtypes = [i64, vp, vp, i32, i32, vp]
    lib.fg_sssp_batch_noalloc.argtypes = [vp, vp, i32, vp, vp]
    lib.fg_ncp_sweep.argtypes = [vp, vp, i32, i32, vp, vp, vp, vp, i32, vp]
    lib.fg_ll_build_labels.argtypes = [vp, i32, i64, vp, vp]
    lib.fg_ll_query.argtypes = [vp, i64, i32, vp, i64, vp, vp]
    lib.fg_bc_accumulate.argtypes = [vp, vp, i32, vp, i32, vp, i32, ctypes.POINTER(fg_bc_info_t), vp]
    lib.fg_rw_batch.argtypes = [vp, vp, i32, i32, ctypes.c_uint64, vp, vp]
    lib.fg_dfs_batch.argtypes = [vp, vp, i32, vp, vp]
    lib.fg_ppr_local_batch.argtypes = [vp, vp, i32, f32, f32, i32, vp, vp, vp, vp, vp]
    lib.fg_tune_opts.argtypes = [vp, i32, vp, i32, vp, ctypes.POINTER(fg_opts), ctypes.POINTER(fg_tune_report)]
    lib.fg_tune_opts_ex.argtypes = [vp, i32, vp, i32, f32, f32, vp, ctypes.POINTER(fg_opts),
                                    ctypes.POINTER(fg_tune_report)]
    u64p = ctypes.POINTER(ctypes.c_uint64)
    lib.fg_default_server_opts.argtypes = [ctypes.POINTER(fg_server_opts)]
    lib.fg_default_server_opts.restype = None
    lib.fg_server_create.argtypes = [vp, ctypes.POINTER(fg_server_opts), ctypes.POINTER(vp)]
    lib.fg_server_destroy.argtypes = [vp]
    lib.fg_server_submit.argtypes = [vp, i32, i32, u64p]
    lib.fg_server_poll.argtypes = [vp, vp, i32, ctypes.POINTER(ctypes.c_int32)]
    lib.fg_server_info.argtypes = [vp, ctypes.c_uint64, ctypes.POINTER(fg_request_info)]
    lib.fg_server_release.argtypes = [vp, ctypes.c_uint64]
    for name in ("fg_graph_create", "fg_graph_create_ex", "fg_graph_destroy", "fg_graph_info", "fg_sssp_batch",
                 "fg_bfs_batch", "fg_ppr_batch", "fg_sync", "fg_stats", "fg_partition_plan",
                 "fg_sssp_batch_noalloc", "fg_server_create", "fg_server_destroy", "fg_server_submit",
                 "fg_server_poll", "fg_server_info", "fg_server_release", "fg_tune_opts", "fg_tune_opts_ex",
                 "fg_ncp_sweep", "fg_ll_build_labels", "fg_ll_query"):
        getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


class FGError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


def fg_last_error() -> str:
    return load().fg_last_error().decode()


def check(status: int) -> None:
    if status != FG_OK:
        raise FGError(status, fg_last_error())


def _ptr(x):
    """Address of a torch tensor, numpy array, ctypes object or int (None -> NULL)."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr()
    if hasattr(x, "ctypes"):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return x.ctypes.data
    return ctypes.addressof(x)


def _stream(s):
    if s is None:
        return None
    if isinstance(s, int):
        return s
    return s.cuda_stream


def fg_default_opts(**overrides) -> fg_opts:
    o = fg_opts()
    load().fg_default_opts(ctypes.byref(o))
    for k, v in overrides.items():
        setattr(o, k, v)
    return o


def fg_default_graph_opts(**overrides) -> fg_graph_opts:
    o = fg_graph_opts()
    load().fg_default_graph_opts(ctypes.byref(o))
    for k, v in overrides.items():
        setattr(o, k, v)
    return o


def fg_graph_create(n, m, row_ptr, col, w=None, flags=0):
    """Returns (status, handle)."""
    h = ctypes.c_void_p()
    st = load().fg_graph_create(n, m, _ptr(row_ptr), _ptr(col), _ptr(w), flags, ctypes.byref(h))
    return st, h.value


def fg_graph_create_ex(n, m, row_ptr, col, w=None, flags=0, gopts=None):
    """Returns (status, handle)."""
    h = ctypes.c_void_p()
    st = load().fg_graph_create_ex(n, m, _ptr(row_ptr), _ptr(col), _ptr(w), flags,
                                   ctypes.byref(gopts) if gopts is not None else None, ctypes.byref(h))
    return st, h.value


def fg_graph_destroy(g) -> int:
    return load().fg_graph_destroy(g)


def fg_graph_info(g):
    """Returns (status, fg_graph_info_t)."""
    info = fg_graph_info_t()
    return load().fg_graph_info(g, ctypes.byref(info)), info


def fg_sssp_batch(g, src, nq, dist_out, stream=None, opts=None) -> int:
    return load().fg_sssp_batch(g, _ptr(src), nq, _ptr(dist_out), _stream(stream),
                                ctypes.byref(opts) if opts is not None else None)


def fg_bfs_batch(g, src, nq, level_out, stream=None, opts=None) -> int:
    return load().fg_bfs_batch(g, _ptr(src), nq, _ptr(level_out), _stream(stream),
                               ctypes.byref(opts) if opts is not None else None)


def fg_ppr_batch(g, src, nq, alpha, eps, p_out, r_out=None, mass_out=None, stream=None, opts=None) -> int:
    return load().fg_ppr_batch(g, _ptr(src), nq, alpha, eps, _ptr(p_out), _ptr(r_out), _ptr(mass_out),
                               _stream(stream), ctypes.byref(opts) if opts is not None else None)


def fg_sync(stream=None) -> int:
    return load().fg_sync(_stream(stream))


def fg_stats(g):
    """Returns (status, fg_stats_t)."""
    s = fg_stats_t()
    return load().fg_stats(g, ctypes.byref(s)), s


def fg_partition_plan(n, row_ptr, col, method, partition_vertices, perm_out) -> int:
    return load().fg_partition_plan(n, _ptr(row_ptr), _ptr(col), method, partition_vertices, _ptr(perm_out))


def fg_sssp_batch_noalloc(g, src, nq, dist_out, stream=None) -> int:
    """Synchronous; device pointers only; graph of at most FG_NOALLOC_MAX_VERTICES vertices."""
    return load().fg_sssp_batch_noalloc(g, _ptr(src), nq, _ptr(dist_out), _stream(stream))


def fg_ncp_sweep(g, p, nq, top, order_out=None, phi_out=None, count_out=None, ncp_out=None, accumulate=False,
                 stream=None) -> int:
    """Sweep cuts over PPR rows p (device float[nq, n]); outputs are device tensors or None."""
    return load().fg_ncp_sweep(g, _ptr(p), nq, top, _ptr(order_out), _ptr(phi_out), _ptr(count_out), _ptr(ncp_out),
                               1 if accumulate else 0, _stream(stream))


def fg_ll_build_labels(dist, K, n, labels, stream=None) -> int:
    """Landmark labels: dist uint32[K, n] (query-major) -> labels uint32[n, K] (vertex-major), device tensors."""
    return load().fg_ll_build_labels(_ptr(dist), K, n, _ptr(labels), _stream(stream))


def fg_ll_query(labels, n, K, pairs, Q, est_out, stream=None) -> int:
    """Landmark distance estimates for Q pairs (device int32[Q, 2]) into est_out (device uint64 / int64[Q])."""
    return load().fg_ll_query(_ptr(labels), n, K, _ptr(pairs), Q, _ptr(est_out), _stream(stream))


def fg_bc_accumulate(g, src, nq, dist, weighted, bc, accumulate=False, stream=None):
    """Brandes dependencies of the batch's rows summed into bc (device double[n]); returns (status, fg_bc_info_t)."""
    info = fg_bc_info_t()
    st = load().fg_bc_accumulate(g, _ptr(src), nq, _ptr(dist), 1 if weighted else 0, _ptr(bc), 1 if accumulate else 0,
                                 ctypes.byref(info), _stream(stream))
    return st, info


def fg_rw_batch(g, src, nq, length, seed, paths_out, stream=None) -> int:
    """Random walks into paths_out (device int32[nq, length + 1])."""
    return load().fg_rw_batch(g, _ptr(src), nq, length, seed & ((1 << 64) - 1), _ptr(paths_out), _stream(stream))


def fg_dfs_batch(g, src, nq, disc_out, stream=None) -> int:
    """DFS discovery ranks into disc_out (device uint32 / int32[nq, n]); synchronous."""
    return load().fg_dfs_batch(g, _ptr(src), nq, _ptr(disc_out), _stream(stream))


def fg_ppr_local_batch(g, src, nq, alpha, eps, cap, vert_out, p_out, count_out, mass_out=None, stream=None) -> int:
    """Local PPR with sparse state: per query the support (vertex, estimate) in rows of cap entries; synchronous."""
    return load().fg_ppr_local_batch(g, _ptr(src), nq, alpha, eps, cap, _ptr(vert_out), _ptr(p_out), _ptr(count_out),
                                     _ptr(mass_out), _stream(stream))


def fg_default_server_opts(**overrides) -> fg_server_opts:
    o = fg_server_opts()
    load().fg_default_server_opts(ctypes.byref(o))
    for k, v in overrides.items():
        setattr(o, k, v)
    return o


def fg_server_create(g, opts=None):
    """Returns (status, server handle)."""
    h = ctypes.c_void_p()
    st = load().fg_server_create(g, ctypes.byref(opts) if opts is not None else None, ctypes.byref(h))
    return st, h.value


def fg_server_destroy(s) -> int:
    return load().fg_server_destroy(s)


def fg_server_submit(s, kind, source):
    """Returns (status, request id)."""
    rid = ctypes.c_uint64()
    st = load().fg_server_submit(s, kind, source, ctypes.byref(rid))
    return st, rid.value


def fg_server_poll(s, cap=1024):
    """Returns (status, list of completed request ids)."""
    buf = (ctypes.c_uint64 * max(1, cap))()
    n = ctypes.c_int32()
    st = load().fg_server_poll(s, buf, cap, ctypes.byref(n))
    return st, list(buf[:n.value])


def fg_server_info(s, rid):
    """Returns (status, fg_request_info)."""
    info = fg_request_info()
    return load().fg_server_info(s, rid, ctypes.byref(info)), info


def fg_server_release(s, rid) -> int:
    return load().fg_server_release(s, rid)


def fg_tune_opts(g, kind, src, nq, stream=None):
    """Returns (status, best fg_opts, fg_tune_report)."""
    best = fg_opts()
    rep = fg_tune_report()
    st = load().fg_tune_opts(g, kind, _ptr(src), nq, _stream(stream), ctypes.byref(best), ctypes.byref(rep))
    return st, best, rep


def fg_tune_opts_ex(g, kind, src, nq, alpha, eps, stream=None):
    """As fg_tune_opts, timing PPR candidates at the caller's alpha and eps."""
    best = fg_opts()
    rep = fg_tune_report()
    st = load().fg_tune_opts_ex(g, kind, _ptr(src), nq, alpha, eps, _stream(stream), ctypes.byref(best),
                                ctypes.byref(rep))
    return st, best, rep
