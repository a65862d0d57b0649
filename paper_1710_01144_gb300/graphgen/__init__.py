"""Seeded synthetic graphs shaped like the paper's workloads (Sec. 6 uses real
social and road networks; these generators stand in for them).

Every function returns ``(row_ptr, col_idx)`` as numpy int32 arrays: the CSR of
a simple undirected graph (sorted neighbour lists, no self-loops, no duplicate
edges) restricted to its largest connected component, ids compacted in their
original order.  The generators live in ``graphgen.c`` and hold none of the
group-closeness arithmetic; both the CPU oracle's tests and the GPU path draw
their inputs from here.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "graphgen.c")
_LIB = os.path.join(_HERE, "libgraphgen.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile ``libgraphgen.so`` next to its source (plain gcc, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".%d.tmp" % os.getpid()
        subprocess.check_call(
            ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
             _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            vp = ctypes.c_void_p
            lib.gg_barabasi_albert.restype = vp
            lib.gg_barabasi_albert.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_uint64]
            lib.gg_rmat.restype = vp
            lib.gg_rmat.argtypes = [ctypes.c_int32, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                    ctypes.c_double, ctypes.c_uint64, ctypes.c_int32]
            lib.gg_grid_road.restype = vp
            lib.gg_grid_road.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_double,
                                         ctypes.c_double, ctypes.c_uint64]
            lib.gg_n.restype = ctypes.c_int32
            lib.gg_n.argtypes = [vp]
            lib.gg_nnz.restype = ctypes.c_int64
            lib.gg_nnz.argtypes = [vp]
            lib.gg_n_raw.restype = ctypes.c_int32
            lib.gg_n_raw.argtypes = [vp]
            lib.gg_copy.restype = None
            lib.gg_copy.argtypes = [vp, vp, vp]
            lib.gg_free.restype = None
            lib.gg_free.argtypes = [vp]
            i32p = ctypes.POINTER(ctypes.c_int32)
            lib.gg_batch_params.restype = None
            lib.gg_batch_params.argtypes = [
                ctypes.c_uint64, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_double,
                ctypes.c_double, ctypes.c_int32, ctypes.c_int32, i32p, i32p,
                ctypes.POINTER(ctypes.c_double), i32p, ctypes.POINTER(ctypes.c_uint64)]
            _lib = lib
    return _lib


def _take(h):
    lib = _load()
    if not h:
        raise MemoryError("graph generation failed (allocation or int32 CSR limit)")
    try:
        n, nnz = lib.gg_n(h), lib.gg_nnz(h)
        rp = np.empty(n + 1, dtype=np.int32)
        ci = np.empty(max(nnz, 1), dtype=np.int32)
        lib.gg_copy(h, rp.ctypes.data, ci.ctypes.data)
        return rp, ci[:nnz]
    finally:
        lib.gg_free(h)


def barabasi_albert(n: int, m: int, seed: int = 1):
    """Preferential attachment: clique on m+1 vertices, then each new vertex
    joins m distinct earlier vertices drawn from the edge-endpoint list."""
    return _take(_load().gg_barabasi_albert(n, m, seed))


def rmat(scale: int, edge_factor: float = 16.0, a: float = 0.57, b: float = 0.19, c: float = 0.19,
         seed: int = 1, n_keep: int = 0):
    """R-MAT: edge_factor * 2**scale sampled pairs by recursive quadrant
    descent; symmetrised, deduplicated, self-loops dropped, LCC kept."""
    return _take(_load().gg_rmat(scale, edge_factor, a, b, c, seed, n_keep))


def grid_road(rows: int, cols: int, p_del: float = 0.2, diag_frac: float = 0.01, seed: int = 1):
    """Road-like graph: 4-neighbour grid, each edge deleted with p_del, plus
    diag_frac * (grid edge count) random diagonal shortcuts; LCC kept."""
    return _take(_load().gg_grid_road(rows, cols, p_del, diag_frac, seed))


@dataclass
class BatchItem:
    family: str
    n_target: int
    avg_deg: float
    k: int
    seed: int


def batch_params(count: int = 256, seed: int = 1, n_lo: int = 10_000, n_hi: int = 500_000,
                 deg_lo: float = 4.0, deg_hi: float = 32.0, k_lo: int = 5, k_hi: int = 50):
    """Parameters of a mixed serving-style batch: family by coin flip, n
    log-uniform in [n_lo, n_hi], average degree uniform, k uniform integer."""
    lib = _load()
    out = []
    for i in range(count):
        fam, n, k = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        deg, gs = ctypes.c_double(), ctypes.c_uint64()
        lib.gg_batch_params(seed, i, n_lo, n_hi, deg_lo, deg_hi, k_lo, k_hi, ctypes.byref(fam),
                            ctypes.byref(n), ctypes.byref(deg), ctypes.byref(k), ctypes.byref(gs))
        out.append(BatchItem("ba" if fam.value == 0 else "rmat", n.value, deg.value, k.value, gs.value))
    return out


def batch_graph(item: BatchItem):
    """Materialise one graph of a mixed batch (BA with m = round(deg/2); R-MAT
    at scale ceil(log2 n) with edge factor deg/2, pairs outside [0, n) dropped)."""
    if item.family == "ba":
        return barabasi_albert(item.n_target, max(1, int(round(item.avg_deg / 2))), item.seed)
    scale = max(1, int(np.ceil(np.log2(item.n_target))))
    # edge factor is relative to 2**scale; rescale so the kept vertex range sees deg/2 pairs per vertex
    ef = (item.avg_deg / 2.0) * item.n_target / float(1 << scale)
    return rmat(scale, ef, seed=item.seed, n_keep=item.n_target)


# Named workloads (the five evaluation configurations, by what they are).
def edge_weights(row_ptr, col_idx, w_max: int = 16, seed: int = 1):
    """Seeded positive integer weights in [1, w_max] for every adjacency entry,
    the same in both rows of an edge: a splitmix64 hash of (min(u, w),
    max(u, w), seed).  int32 array aligned with col_idx."""
    rp = np.asarray(row_ptr, dtype=np.int64)
    ci = np.asarray(col_idx, dtype=np.int64)
    u = np.repeat(np.arange(rp.size - 1, dtype=np.int64), np.diff(rp))
    a, b = np.minimum(u, ci).astype(np.uint64), np.maximum(u, ci).astype(np.uint64)
    with np.errstate(over="ignore"):
        x = (a * np.uint64(0x9E3779B97F4A7C15)) ^ (b + np.uint64(seed) * np.uint64(0xD1B54A32D192ED03))
        x = (x ^ (x >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        x = (x ^ (x >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        x = x ^ (x >> np.uint64(31))
    return (x % np.uint64(w_max)).astype(np.int32) + np.int32(1)


def ba_n2000_m5(seed: int = 1):
    return barabasi_albert(2000, 5, seed)


def rmat_s20_ef16(seed: int = 1):
    return rmat(20, 16.0, seed=seed)


def road_grid_2048(seed: int = 1):
    return grid_road(2048, 2048, 0.2, 0.01, seed)


def rmat_s24_ef16(seed: int = 1):
    return rmat(24, 16.0, seed=seed)
