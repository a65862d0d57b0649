"""CPU oracle for Greedy++ group-closeness maximization (arXiv:1710.01144).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this package.  It shares no
code with the CUDA library: its arithmetic lives in ``oracle.c`` (plain
definitions, full BFS everywhere), ``greedypp.c`` (the paper's Greedy++ on
the CPU, pinned to the plain oracle on small graphs) and ``mlp.py`` (float64
reference of the candidate-proposal network).

Conventions (readings of the paper, Sec. 2 and Sec. 4.2):
  * farness f(S) = sum over all vertices u of d(u, S), an int64, with the
    paper's 1/n and group-size normalisations dropped;
  * gain Delta(v|S) = f(S) - f(S + {v}) >= 0 (positive decrease);
  * ties always go to the smallest vertex id.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRCS = [os.path.join(_HERE, "oracle.c"), os.path.join(_HERE, "greedypp.c")]
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile ``liboracle.so`` (gcc, OpenMP) next to its sources."""
    newest = max(os.path.getmtime(s) for s in _SRCS)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < newest:
        tmp = _LIB + ".%d.tmp" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", *_SRCS,
                               "-o", tmp])
        os.replace(tmp, _LIB)
    return _LIB


class _GppStats(ctypes.Structure):
    _fields_ = [("evals", ctypes.c_int64), ("edges", ctypes.c_int64), ("round0_full", ctypes.c_int64)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            vp, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
            lib.or_bfs_multi.restype = i64
            lib.or_bfs_multi.argtypes = [i32, vp, vp, vp, i32, vp]
            lib.or_farness.restype = i64
            lib.or_farness.argtypes = [i32, vp, vp, vp, i32]
            lib.or_gains.restype = ctypes.c_int
            lib.or_gains.argtypes = [i32, vp, vp, vp, i32, vp, i32, vp, i32]
            lib.or_greedy_plain.restype = ctypes.c_int
            lib.or_greedy_plain.argtypes = [i32, vp, vp, i32, vp, vp, vp, i32]
            lib.or_dijkstra_multi.restype = i64
            lib.or_dijkstra_multi.argtypes = [i32, vp, vp, vp, vp, i32, vp]
            lib.or_wfarness.restype = i64
            lib.or_wfarness.argtypes = [i32, vp, vp, vp, vp, i32]
            lib.or_wgains.restype = ctypes.c_int
            lib.or_wgains.argtypes = [i32, vp, vp, vp, vp, i32, vp, i32, vp, i32]
            lib.or_wgreedy_plain.restype = ctypes.c_int
            lib.or_wgreedy_plain.argtypes = [i32, vp, vp, vp, i32, vp, vp, vp, i32]
            lib.or_opt_bruteforce.restype = i64
            lib.or_opt_bruteforce.argtypes = [i32, vp, vp, i32, vp]
            lib.or_gains_bitparallel.restype = ctypes.c_int
            lib.or_gains_bitparallel.argtypes = [i32, vp, vp, vp, i32, vp]
            lib.or_top1_closeness.restype = ctypes.c_int
            lib.or_top1_closeness.argtypes = [i32, vp, vp, i32, vp, vp, vp]
            lib.or_topk_closeness.restype = ctypes.c_int
            lib.or_topk_closeness.argtypes = [i32, vp, vp, i32, i32, vp, vp, vp]
            lib.or_greedypp.restype = ctypes.c_int
            lib.or_greedypp.argtypes = [i32, vp, vp, i32, vp, vp, vp, i32, ctypes.POINTER(_GppStats)]
            lib.or_greedypp_cost_sample.restype = ctypes.c_int
            lib.or_greedypp_cost_sample.argtypes = [i32, vp, vp, i32, i64, i32, vp, i32, i32, vp]
            _lib = lib
    return _lib


def _csr(row_ptr, col_idx):
    rp = np.ascontiguousarray(row_ptr, dtype=np.int32)
    ci = np.ascontiguousarray(col_idx, dtype=np.int32)
    if ci.size == 0:
        ci = np.zeros(1, dtype=np.int32)
    return rp, ci, rp.size - 1


def _i32(a):
    a = np.ascontiguousarray(a, dtype=np.int32)
    return a if a.size else np.zeros(1, dtype=np.int32)


def default_threads() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:  # pragma: no cover
        return os.cpu_count() or 1


def bfs(row_ptr, col_idx, sources):
    """Distances from the nearest source (-1 where unreachable)."""
    rp, ci, n = _csr(row_ptr, col_idx)
    src = np.atleast_1d(np.asarray(sources, dtype=np.int32))
    d = np.empty(n, dtype=np.int32)
    r = _load().or_bfs_multi(n, rp.ctypes.data, ci.ctypes.data, _i32(src).ctypes.data, src.size,
                             d.ctypes.data)
    if r < 0:
        raise ValueError("bad source")
    return d


def farness(row_ptr, col_idx, S) -> int:
    """f(S) = sum_u d(u, S) (int); raises on an empty group or unreachable vertex."""
    rp, ci, n = _csr(row_ptr, col_idx)
    s = np.asarray(S, dtype=np.int32)
    f = _load().or_farness(n, rp.ctypes.data, ci.ctypes.data, _i32(s).ctypes.data, s.size)
    if f < 0:
        raise ValueError("farness undefined (empty group, bad id or disconnected graph)")
    return int(f)


def gains(row_ptr, col_idx, S, cand, threads: int | None = None):
    """Delta(v|S) for each candidate by a full BFS from v (int64 array)."""
    rp, ci, n = _csr(row_ptr, col_idx)
    s = np.asarray(S, dtype=np.int32)
    c = np.asarray(cand, dtype=np.int32)
    out = np.zeros(max(c.size, 1), dtype=np.int64)
    rc = _load().or_gains(n, rp.ctypes.data, ci.ctypes.data, _i32(s).ctypes.data, s.size,
                          _i32(c).ctypes.data, c.size, out.ctypes.data, threads or default_threads())
    if rc:
        raise ValueError("bad group or candidate")
    return out[:c.size]


def greedy_plain(row_ptr, col_idx, k: int, threads: int | None = None):
    """Plain greedy: returns (group, farness_trace, gain_trace) as numpy arrays."""
    rp, ci, n = _csr(row_ptr, col_idx)
    g = np.empty(k, dtype=np.int32)
    ft = np.empty(k, dtype=np.int64)
    gt = np.empty(k, dtype=np.int64)
    rc = _load().or_greedy_plain(n, rp.ctypes.data, ci.ctypes.data, k, g.ctypes.data,
                                 ft.ctypes.data, gt.ctypes.data, threads or default_threads())
    if rc:
        raise ValueError("bad k or disconnected graph")
    return g, ft, gt


def dijkstra(row_ptr, col_idx, weights, src):
    """Weighted distances from the sources (int64 array, -1 where unreachable)."""
    rp, ci, n = _csr(row_ptr, col_idx)
    w = _i32(np.asarray(weights, dtype=np.int32))
    s = np.atleast_1d(np.asarray(src, dtype=np.int32))
    d = np.zeros(max(n, 1), dtype=np.int64)
    r = _load().or_dijkstra_multi(n, rp.ctypes.data, ci.ctypes.data, w.ctypes.data, _i32(s).ctypes.data, s.size,
                                  d.ctypes.data)
    if r < 0:
        raise ValueError("bad source id or a weight below 1")
    return d[:n]


def wfarness(row_ptr, col_idx, weights, S) -> int:
    """Weighted f(S) = sum_u d_w(u, S) (int); raises if undefined."""
    rp, ci, n = _csr(row_ptr, col_idx)
    w = _i32(np.asarray(weights, dtype=np.int32))
    s = np.asarray(S, dtype=np.int32)
    f = _load().or_wfarness(n, rp.ctypes.data, ci.ctypes.data, w.ctypes.data, _i32(s).ctypes.data, s.size)
    if f < 0:
        raise ValueError("weighted farness undefined (empty group, bad id, bad weight or disconnected graph)")
    return int(f)


def wgains(row_ptr, col_idx, weights, S, cand, threads: int | None = None):
    """Weighted Delta(v|S) for each candidate by a full Dijkstra from v."""
    rp, ci, n = _csr(row_ptr, col_idx)
    w = _i32(np.asarray(weights, dtype=np.int32))
    s = np.asarray(S, dtype=np.int32)
    c = np.asarray(cand, dtype=np.int32)
    out = np.zeros(max(c.size, 1), dtype=np.int64)
    rc = _load().or_wgains(n, rp.ctypes.data, ci.ctypes.data, w.ctypes.data, _i32(s).ctypes.data, s.size,
                           _i32(c).ctypes.data, c.size, out.ctypes.data, threads or default_threads())
    if rc:
        raise ValueError("bad group or candidate")
    return out[:c.size]


def wgreedy_plain(row_ptr, col_idx, weights, k: int, threads: int | None = None):
    """Plain weighted greedy (Dijkstra for every SSSP): (group, farness_trace, gain_trace)."""
    rp, ci, n = _csr(row_ptr, col_idx)
    w = _i32(np.asarray(weights, dtype=np.int32))
    g = np.empty(k, dtype=np.int32)
    ft = np.empty(k, dtype=np.int64)
    gt = np.empty(k, dtype=np.int64)
    rc = _load().or_wgreedy_plain(n, rp.ctypes.data, ci.ctypes.data, w.ctypes.data, k, g.ctypes.data,
                                  ft.ctypes.data, gt.ctypes.data, threads or default_threads())
    if rc:
        raise ValueError("bad k or disconnected graph")
    return g, ft, gt


def opt_bruteforce(row_ptr, col_idx, k: int):
    """(min farness over all k-subsets, lexicographically first optimal set)."""
    rp, ci, n = _csr(row_ptr, col_idx)
    g = np.empty(k, dtype=np.int32)
    f = _load().or_opt_bruteforce(n, rp.ctypes.data, ci.ctypes.data, k, g.ctypes.data)
    if f < 0:
        raise ValueError("bad k, n > 24 or disconnected graph")
    return int(f), g


def gains_bitparallel(row_ptr, col_idx, S):
    """Theorem 1 gains for every vertex (int64 array of length n)."""
    rp, ci, n = _csr(row_ptr, col_idx)
    s = np.asarray(S, dtype=np.int32)
    out = np.zeros(max(n, 1), dtype=np.int64)
    rc = _load().or_gains_bitparallel(n, rp.ctypes.data, ci.ctypes.data, _i32(s).ctypes.data, s.size,
                                      out.ctypes.data)
    if rc:
        raise ValueError("bad group or n too large")
    return out[:n]


def top1_closeness(row_ptr, col_idx, threads: int | None = None):
    """(s0, f({s0}), number of BFSs that ran to completion)."""
    rp, ci, n = _csr(row_ptr, col_idx)
    s0, f0, full = ctypes.c_int32(), ctypes.c_int64(), ctypes.c_int64()
    rc = _load().or_top1_closeness(n, rp.ctypes.data, ci.ctypes.data, threads or default_threads(),
                                   ctypes.addressof(s0), ctypes.addressof(f0), ctypes.addressof(full))
    if rc:
        raise ValueError("disconnected graph")
    return s0.value, f0.value, full.value


def topk_closeness(row_ptr, col_idx, k: int, threads: int | None = None):
    """Top-k closeness (Sec. 3.1, Algorithm 3): (ids, farness values) of the k
    vertices of smallest farness, ordered by (farness, id); plus the number of
    BFSs that ran to completion."""
    rp, ci, n = _csr(row_ptr, col_idx)
    ids = np.zeros(k, dtype=np.int32)
    f = np.zeros(k, dtype=np.int64)
    full = ctypes.c_int64()
    rc = _load().or_topk_closeness(n, rp.ctypes.data, ci.ctypes.data, k, threads or default_threads(),
                                   ids.ctypes.data, f.ctypes.data, ctypes.addressof(full))
    if rc:
        raise ValueError("disconnected graph or k outside [1, n]" if rc == -1 else "allocation failed")
    return ids, f, full.value


def greedypp(row_ptr, col_idx, k: int, threads: int | None = None):
    """CPU Greedy++: returns (group, farness_trace, gain_trace, stats dict)."""
    rp, ci, n = _csr(row_ptr, col_idx)
    g = np.empty(k, dtype=np.int32)
    ft = np.empty(k, dtype=np.int64)
    gt = np.empty(k, dtype=np.int64)
    st = _GppStats()
    rc = _load().or_greedypp(n, rp.ctypes.data, ci.ctypes.data, k, g.ctypes.data, ft.ctypes.data,
                             gt.ctypes.data, threads or default_threads(), ctypes.byref(st))
    if rc:
        raise ValueError("bad k or disconnected graph")
    return g, ft, gt, {"evals": st.evals, "edges": st.edges, "round0_full": st.round0_full}


def greedypp_cost_sample(row_ptr, col_idx, s0: int, f_best: int, cand, threads: int | None = None):
    """Wall seconds of CPU Greedy++'s two dominant steps on the vertices `cand`:
    (round-0 BFScut against the fixed threshold (f_best, s0), round-1 pruned
    SSSP against S = {s0}, entries scanned by the latter).  Used only to time
    the oracle on a bounded sample of a large workload."""
    rp, ci, n = _csr(row_ptr, col_idx)
    c = _i32(cand)
    out = np.zeros(3, dtype=np.float64)
    rc = _load().or_greedypp_cost_sample(n, rp.ctypes.data, ci.ctypes.data, int(s0), int(f_best), int(s0),
                                         c.ctypes.data, int(np.size(cand)), threads or default_threads(),
                                         out.ctypes.data)
    if rc:
        raise MemoryError("oracle cost sample failed")
    return float(out[0]), float(out[1]), float(out[2])
