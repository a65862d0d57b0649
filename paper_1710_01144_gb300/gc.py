"""Thin ctypes binding of ``libgc.so`` (C ABI in include/gc.h).

Argument marshalling only: every step of the path runs in the library's CUDA
kernels.  There is no CPU fallback -- if the library is missing or no GPU is
present, the calls raise.  PyTorch is used for device memory and the current
stream when tensors are passed.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libgc.so")

GC_OK = 0
GC_EINVAL = -1
GC_EDISCONNECTED = -2
GC_ERANGE = -3
GC_ENOMEM = -4
GC_ECUDA = -5
GC_ETIMEOUT = -6
GC_EINTERNAL = -7
GC_DEVICE_PTRS = 0x1
GC_ADOPT = 0x2
GC_VALIDATE = 0x4
GC_OPT_NO_EXPAND_BOUND = 0x1
GC_OPT_CAPTURE = 0x2
GC_OPT_FULL_ADJACENCY = 0x4
GC_OPT_NO_ROUND1_BOUND = 0x8
GC_OPT_R0_FULL_LEVELS = 0x10
GC_OPT_R0_NO_PROBE = 0x40
GC_OPT_NO_CLAIM_LOG = 0x20

# every entry point declared in include/gc.h
EXPORTS = ("gc_opts_default", "gc_load_csr", "gc_free", "gc_num_vertices", "gc_num_entries",
           "gc_group_farness", "gc_marginal_gains", "gc_marginal_gains_device", "gc_greedy",
           "gc_last_error", "gc_marginal_gains_static", "gc_mlp_create", "gc_mlp_free", "gc_mlp_set_params",
           "gc_mlp_get_params", "gc_mlp_forward", "gc_mlp_grad", "gc_mlp_adam_step", "gc_mlp_train",
           "gc_candidate_features", "gc_set_proposal", "gc_set_recorder", "gc_recorded", "gc_batch_load",
           "gc_batch_free", "gc_batch_vertices", "gc_batch_greedy", "gc_gain_upper_bounds", "gc_greedy_batch",
           "gc_top_closeness", "gc_greedy_bits", "gc_set_weights", "gc_greedy_weighted", "gc_set_gain_lanes")
MLP_IN, MLP_HIDDEN, MLP_PARAMS = 8, 64, 4801


class GcError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__("%s (code %d)" % (msg, code))
        self.code = code


class Opts(ctypes.Structure):
    _fields_ = [("eval_per_step", ctypes.c_int32), ("use_proposal", ctypes.c_int32),
                ("max_ctas", ctypes.c_int32), ("timeout_ms", ctypes.c_int32),
                ("step_lanes", ctypes.c_int32), ("step_mode", ctypes.c_int32),
                ("active_target", ctypes.c_int32), ("round1_heavy", ctypes.c_int32),
                ("flags", ctypes.c_uint32), ("step_form", ctypes.c_int32),
                ("local_update_max_gain", ctypes.c_int32), ("lazy_ctas", ctypes.c_int32),
                ("batch_grid_min_n", ctypes.c_int32), ("round0_lanes", ctypes.c_int32),
                ("timeout_us", ctypes.c_int32), ("claim_log_cap", ctypes.c_int32)]


class Stats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in (
        "rounds", "steps", "evals", "batches", "edges_scalar", "edges_union", "levels", "frontier",
        "pushes", "lanes", "round0_evals")] + [
        ("ms_round0", ctypes.c_double), ("ms_round1", ctypes.c_double), ("ms_total", ctypes.c_double), ("ms_gain_kernel", ctypes.c_double),
        ("ms_lazy_select", ctypes.c_double), ("ms_lazy_gain", ctypes.c_double), ("ms_lazy_update", ctypes.c_double),
        ("gain_launches", ctypes.c_int64), ("kernel_launches", ctypes.c_int64), ("graph_replay", ctypes.c_int64),
        ("gain64_launches", ctypes.c_int64), ("ms_gain64", ctypes.c_double)] + [(n, ctypes.c_int64) for n in (
        "gain64_frontier", "gain64_edges", "gain64_pushes", "gain64_lanes",
        "lazy_frontier", "lazy_edges", "lazy_pushes", "lazy_lanes", "lazy_launches")] + [
        ("ms_lazy_kernel", ctypes.c_double)] + [(n, ctypes.c_int64) for n in (
        "lazy_upd_frontier", "lazy_upd_edges", "lazy_upd_relabels", "lazy_sel_scanned")] + [
        ("ms_round0_wide", ctypes.c_double), ("r0_batches", ctypes.c_int64), ("r0_levels", ctypes.c_int64),
        ("r0_td_edges", ctypes.c_int64), ("ms_r0_select", ctypes.c_double), ("ms_r0_topdown", ctypes.c_double),
        ("ms_r0_bottomup", ctypes.c_double), ("ms_r0_clear", ctypes.c_double), ("r0_bu_rows", ctypes.c_int64),
        ("r0_bu_scanned", ctypes.c_int64), ("r0_bu_gathers", ctypes.c_int64), ("r0_width", ctypes.c_int64),
        ("r0_dense_clears", ctypes.c_int64), ("lazy_log_picks", ctypes.c_int64), ("lazy_upd_log", ctypes.c_int64),
        ("lazy_log_entries", ctypes.c_int64), ("r0_probes", ctypes.c_int64), ("r0_probe_cut", ctypes.c_int64),
        ("r0_bu_vertices", ctypes.c_int64), ("r0_bu_visreads", ctypes.c_int64)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


_lock = threading.Lock()
_lib = None


def load(path: str = LIB_PATH):
    """Load libgc.so; raises if it has not been built (no fallback)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise RuntimeError("libgc.so is not built (run paper_1710_01144_gb300.build.build())")
        lib = ctypes.CDLL(path)
        vp, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
        lib.gc_opts_default.argtypes = [ctypes.POINTER(Opts)]
        lib.gc_load_csr.argtypes = [i32, vp, vp, ctypes.c_uint32, vp, ctypes.POINTER(vp)]
        lib.gc_free.argtypes = [vp]
        lib.gc_num_vertices.argtypes = [vp]
        lib.gc_num_vertices.restype = i64
        lib.gc_num_entries.argtypes = [vp]
        lib.gc_num_entries.restype = i64
        lib.gc_group_farness.argtypes = [vp, vp, i32, vp]
        lib.gc_marginal_gains.argtypes = [vp, vp, i32, vp, i32, vp, ctypes.POINTER(Stats)]
        lib.gc_marginal_gains_device.argtypes = [vp, vp, i32, vp, i32, vp]
        lib.gc_set_gain_lanes.argtypes = [vp, i32]
        lib.gc_greedy.argtypes = [vp, i32, ctypes.POINTER(Opts), vp, vp, ctypes.POINTER(Stats)]
        lib.gc_gain_upper_bounds.argtypes = [vp, vp, i32, vp]
        lib.gc_marginal_gains_static.argtypes = [i32, vp, vp, vp, i32, vp, i32, vp, vp]
        lib.gc_mlp_create.argtypes = [i32, vp, ctypes.POINTER(vp)]
        lib.gc_mlp_free.argtypes = [vp]
        lib.gc_mlp_set_params.argtypes = [vp, vp]
        lib.gc_mlp_get_params.argtypes = [vp, vp]
        lib.gc_mlp_forward.argtypes = [vp, vp, i32, vp]
        lib.gc_mlp_grad.argtypes = [vp, vp, vp, i32, vp, ctypes.POINTER(ctypes.c_double)]
        lib.gc_mlp_adam_step.argtypes = [vp, vp, vp, i32, ctypes.c_float]
        lib.gc_mlp_train.argtypes = [vp, vp, vp, i32, i32, i32, ctypes.c_float, ctypes.c_uint64,
                                     ctypes.POINTER(ctypes.c_double)]
        lib.gc_candidate_features.argtypes = [vp, vp, vp, vp, vp, vp, vp, i32, i32, i64, vp, vp]
        lib.gc_set_proposal.argtypes = [vp, vp, i32]
        lib.gc_set_recorder.argtypes = [vp, vp, vp, i32]
        lib.gc_recorded.argtypes = [vp]
        lib.gc_recorded.restype = i64
        lib.gc_batch_load.argtypes = [i32, vp, vp, vp, ctypes.c_uint32, vp, ctypes.POINTER(vp)]
        lib.gc_batch_free.argtypes = [vp]
        lib.gc_batch_vertices.argtypes = [vp]
        lib.gc_batch_vertices.restype = i64
        lib.gc_batch_greedy.argtypes = [vp, vp, ctypes.POINTER(Opts), vp, vp, ctypes.POINTER(Stats)]
        lib.gc_greedy_batch.argtypes = [vp, vp, i32, ctypes.POINTER(Opts), vp, vp, ctypes.POINTER(Stats)]
        lib.gc_top_closeness.argtypes = [vp, i32, ctypes.POINTER(Opts), vp, vp, ctypes.POINTER(Stats)]
        lib.gc_greedy_bits.argtypes = [vp, i32, ctypes.POINTER(Opts), vp, vp, ctypes.POINTER(Stats)]
        lib.gc_set_weights.argtypes = [vp, vp, ctypes.c_uint32]
        lib.gc_greedy_weighted.argtypes = [vp, i32, ctypes.POINTER(Opts), vp, vp, ctypes.POINTER(Stats)]
        lib.gc_last_error.restype = ctypes.c_char_p
        for name in EXPORTS:
            if name not in ("gc_num_vertices", "gc_num_entries", "gc_last_error", "gc_recorded",
                            "gc_batch_vertices"):
                getattr(lib, name).restype = ctypes.c_int
        _lib = lib
        return lib


def _check(rc: int):
    if rc != GC_OK:
        raise GcError(rc, load().gc_last_error().decode())


def _current_stream() -> int:
    import torch

    return int(torch.cuda.current_stream().cuda_stream)


def _i32(a):
    a = np.ascontiguousarray(a, dtype=np.int32)
    return a if a.size else np.zeros(1, dtype=np.int32)


class Graph:
    """A graph resident on the current CUDA device.

    ``row_ptr``/``col_idx`` are numpy int32 arrays (host, copied) or int32 CUDA
    tensors (device; ``adopt=True`` uses them in place, keep them alive)."""

    def __init__(self, row_ptr, col_idx, validate: bool = False, adopt: bool = False, stream=None):
        lib = load()
        self._keep = None
        flags = GC_VALIDATE if validate else 0
        if hasattr(row_ptr, "data_ptr"):
            flags |= GC_DEVICE_PTRS | (GC_ADOPT if adopt else 0)
            n = row_ptr.numel() - 1
            rp_p, ci_p = row_ptr.data_ptr(), col_idx.data_ptr()
            if adopt:
                self._keep = (row_ptr, col_idx)
        else:
            rp = np.ascontiguousarray(row_ptr, dtype=np.int32)
            ci = _i32(col_idx)
            n = rp.size - 1
            rp_p, ci_p = rp.ctypes.data, ci.ctypes.data
        self.stream = _current_stream() if stream is None else int(stream)
        h = ctypes.c_void_p()
        _check(lib.gc_load_csr(n, rp_p, ci_p, flags, self.stream, ctypes.byref(h)))
        self._h = h
        self.n = int(lib.gc_num_vertices(h))
        self.nnz = int(lib.gc_num_entries(h))

    def close(self):
        if getattr(self, "_h", None):
            load().gc_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def farness(self, S) -> int:
        s = _i32(S)
        out = ctypes.c_int64()
        _check(load().gc_group_farness(self._h, s.ctypes.data, int(np.size(S)), ctypes.byref(out)))
        return out.value

    def gains(self, S, cand, stats: bool = False):
        s = _i32(S)
        c = np.ascontiguousarray(cand, dtype=np.int32)
        out = np.zeros(max(c.size, 1), dtype=np.int64)
        st = Stats()
        _check(load().gc_marginal_gains(self._h, s.ctypes.data, int(np.size(S)), _i32(c).ctypes.data,
                                        c.size, out.ctypes.data, ctypes.byref(st)))
        return (out[:c.size], st.as_dict()) if stats else out[:c.size]

    def set_gain_lanes(self, lanes: int):
        """Candidates per batch (64, 128 or 256) of the CTA-batched gain kernel."""
        _check(load().gc_set_gain_lanes(self._h, int(lanes)))

    def gains_device(self, S_dev, cand_dev, out_dev):
        """Asynchronous gains on the handle's stream; all three are CUDA tensors."""
        _check(load().gc_marginal_gains_device(self._h, S_dev.data_ptr(), S_dev.numel(), cand_dev.data_ptr(),
                                               cand_dev.numel(), out_dev.data_ptr()))

    def upper_bounds(self, S):
        """Two-hop upper bounds on Delta(v|S) for every vertex (-1 for members)."""
        s = _i32(S)
        out = np.zeros(self.n, dtype=np.int64)
        _check(load().gc_gain_upper_bounds(self._h, s.ctypes.data, int(np.size(S)), out.ctypes.data))
        return out

    def set_proposal(self, mlp, fill: int = 0):
        """Use `mlp` (an Mlp, or None to disable) for part of every batch."""
        self._prop = mlp
        _check(load().gc_set_proposal(self._h, mlp._h if mlp is not None else None, fill))

    def set_recorder(self, X_dev, y_dev):
        """Record (features, log1p gain) of host-driven lazy steps into CUDA tensors
        X_dev [cap, 8] and y_dev [cap] (float32); None disables."""
        if X_dev is None:
            _check(load().gc_set_recorder(self._h, None, None, 0))
            self._rec = None
            return
        self._rec = (X_dev, y_dev)
        _check(load().gc_set_recorder(self._h, X_dev.data_ptr(), y_dev.data_ptr(), int(y_dev.numel())))

    def recorded(self) -> int:
        return int(load().gc_recorded(self._h))

    def greedy(self, k: int, eval_per_step: int = 0, max_ctas: int = 0, timeout_ms: int = 0,
               use_proposal: bool = False, step_lanes: int = 0, step_mode: int = 0,
               active_target: int = 0, round1_heavy: int = 0, expand_bound: bool = True,
               step_form: int = 0, local_update_max_gain: int = 0, lazy_ctas: int = 0,
               pruned_adjacency: bool = True, round1_bound: bool = True, timeout_us: int = 0,
               round0_lanes: int = 0, r0_full_levels: bool = False, r0_probe: bool = True, claim_log: bool = True,
               claim_log_cap: int = 0):
        o = Opts()
        load().gc_opts_default(ctypes.byref(o))
        o.eval_per_step, o.max_ctas, o.use_proposal = eval_per_step, max_ctas, int(use_proposal)
        o.step_lanes, o.step_mode, o.active_target = step_lanes, step_mode, active_target
        o.round1_heavy = round1_heavy
        o.flags = ((0 if expand_bound else GC_OPT_NO_EXPAND_BOUND) | (0 if pruned_adjacency else GC_OPT_FULL_ADJACENCY)
                   | (0 if round1_bound else GC_OPT_NO_ROUND1_BOUND) | (GC_OPT_R0_FULL_LEVELS if r0_full_levels else 0)
                   | (0 if r0_probe else GC_OPT_R0_NO_PROBE)
                   | (0 if claim_log else GC_OPT_NO_CLAIM_LOG))
        o.step_form, o.local_update_max_gain = step_form, local_update_max_gain
        o.lazy_ctas = lazy_ctas
        if timeout_ms:
            o.timeout_ms = timeout_ms
        o.timeout_us = timeout_us
        o.round0_lanes = round0_lanes
        o.claim_log_cap = claim_log_cap
        grp = np.zeros(max(int(k), 1), dtype=np.int32)
        f = ctypes.c_int64()
        st = Stats()
        _check(load().gc_greedy(self._h, int(k), ctypes.byref(o), grp.ctypes.data, ctypes.byref(f),
                                ctypes.byref(st)))
        return grp[:k], f.value, st.as_dict()

    def set_weights(self, weights, validate: bool = False):
        """gc_set_weights: positive int32 edge weights aligned with col_idx
        (numpy, copied; or an int32 CUDA tensor)."""
        flags = GC_VALIDATE if validate else 0
        if hasattr(weights, "data_ptr"):
            _check(load().gc_set_weights(self._h, weights.data_ptr(), flags | GC_DEVICE_PTRS))
        else:
            w = _i32(np.asarray(weights, dtype=np.int32))
            _check(load().gc_set_weights(self._h, w.ctypes.data, flags))

    def greedy_weighted(self, k: int):
        """gc_greedy_weighted: (group, farness, stats) with weighted distances."""
        o = Opts()
        load().gc_opts_default(ctypes.byref(o))
        grp = np.zeros(max(int(k), 1), dtype=np.int32)
        f = ctypes.c_int64()
        st = Stats()
        _check(load().gc_greedy_weighted(self._h, int(k), ctypes.byref(o), grp.ctypes.data, ctypes.byref(f),
                                         ctypes.byref(st)))
        return grp[:k], f.value, st.as_dict()

    def greedy_bits(self, k: int, timeout_us: int = 0):
        """gc_greedy_bits (bitGreedy++, every vertex scored every round):
        (group, farness, stats)."""
        o = Opts()
        load().gc_opts_default(ctypes.byref(o))
        o.timeout_us = timeout_us
        grp = np.zeros(max(int(k), 1), dtype=np.int32)
        f = ctypes.c_int64()
        st = Stats()
        _check(load().gc_greedy_bits(self._h, int(k), ctypes.byref(o), grp.ctypes.data, ctypes.byref(f),
                                     ctypes.byref(st)))
        return grp[:k], f.value, st.as_dict()

    def top_closeness(self, k: int, round0_lanes: int = 0, max_ctas: int = 0, r0_full_levels: bool = False,
                      r0_probe: bool = True):
        """gc_top_closeness: (ids, farness values, stats) of the k vertices of
        smallest farness, ordered by (farness, id)."""
        o = Opts()
        load().gc_opts_default(ctypes.byref(o))
        o.round0_lanes, o.max_ctas = round0_lanes, max_ctas
        o.flags = (GC_OPT_R0_FULL_LEVELS if r0_full_levels else 0) | (0 if r0_probe else GC_OPT_R0_NO_PROBE)
        ids = np.zeros(max(int(k), 1), dtype=np.int32)
        f = np.zeros(max(int(k), 1), dtype=np.int64)
        st = Stats()
        _check(load().gc_top_closeness(self._h, int(k), ctypes.byref(o), ids.ctypes.data, f.ctypes.data,
                                       ctypes.byref(st)))
        return ids[:k], f[:k], st.as_dict()


def gains_static(row_ptr_dev, col_idx_dev, S_dev, cand_dev, out_dev, stream=None):
    """gc_marginal_gains_static on CUDA tensors: no device allocation by the
    library (its scratch is a fixed array); asynchronous on ``stream``."""
    st = _current_stream() if stream is None else int(stream)
    _check(load().gc_marginal_gains_static(row_ptr_dev.numel() - 1, row_ptr_dev.data_ptr(), col_idx_dev.data_ptr(),
                                           S_dev.data_ptr(), S_dev.numel(), cand_dev.data_ptr(), cand_dev.numel(),
                                           out_dev.data_ptr(), st))


class Mlp:
    """The proposal network (8 -> 64 -> 64 -> 1, float32) on the current device."""

    def __init__(self, max_batch: int = 4096, stream=None):
        self.stream = _current_stream() if stream is None else int(stream)
        h = ctypes.c_void_p()
        _check(load().gc_mlp_create(max_batch, self.stream, ctypes.byref(h)))
        self._h = h
        self.max_batch = max_batch

    def close(self):
        if getattr(self, "_h", None):
            load().gc_mlp_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, p):
        p = np.ascontiguousarray(p, dtype=np.float32)
        assert p.size == MLP_PARAMS
        _check(load().gc_mlp_set_params(self._h, p.ctypes.data))

    def get_params(self):
        p = np.empty(MLP_PARAMS, dtype=np.float32)
        _check(load().gc_mlp_get_params(self._h, p.ctypes.data))
        return p

    def forward(self, X_dev, out_dev):
        _check(load().gc_mlp_forward(self._h, X_dev.data_ptr(), int(X_dev.shape[0]), out_dev.data_ptr()))

    def grad(self, X_dev, y_dev):
        g = np.empty(MLP_PARAMS, dtype=np.float32)
        loss = ctypes.c_double()
        _check(load().gc_mlp_grad(self._h, X_dev.data_ptr(), y_dev.data_ptr(), int(X_dev.shape[0]), g.ctypes.data,
                                  ctypes.byref(loss)))
        return g, loss.value

    def adam_step(self, X_dev, y_dev, lr: float):
        _check(load().gc_mlp_adam_step(self._h, X_dev.data_ptr(), y_dev.data_ptr(), int(X_dev.shape[0]), lr))

    def train(self, X_dev, y_dev, epochs: int = 20, batch: int = 1024, lr: float = 1e-3, seed: int = 1) -> float:
        loss = ctypes.c_double()
        _check(load().gc_mlp_train(self._h, X_dev.data_ptr(), y_dev.data_ptr(), int(X_dev.shape[0]), epochs, batch,
                                   lr, seed, ctypes.byref(loss)))
        return loss.value


def candidate_features(row_ptr, dS, ub, stamp, two_hop, mx, cand, rnd, prev_gain, X_out, stream=None):
    """gc_candidate_features on CUDA tensors (asynchronous)."""
    st = _current_stream() if stream is None else int(stream)
    _check(load().gc_candidate_features(row_ptr.data_ptr(), dS.data_ptr(), ub.data_ptr(), stamp.data_ptr(),
                                        two_hop.data_ptr(), mx.data_ptr() if mx is not None else None,
                                        cand.data_ptr(), int(cand.numel()), int(rnd), int(prev_gain),
                                        X_out.data_ptr(), st))


class Batch:
    """Many graphs solved together by one persistent kernel (gc_batch_*)."""

    def __init__(self, graphs, stream=None):
        lib = load()
        self._keep = [(np.ascontiguousarray(rp, dtype=np.int32), _i32(ci)) for rp, ci in graphs]
        cnt = len(self._keep)
        rps = (ctypes.c_void_p * cnt)(*[rp.ctypes.data for rp, _ in self._keep])
        cis = (ctypes.c_void_p * cnt)(*[ci.ctypes.data for _, ci in self._keep])
        self.ns = np.array([rp.size - 1 for rp, _ in self._keep], dtype=np.int32)
        self.stream = _current_stream() if stream is None else int(stream)
        h = ctypes.c_void_p()
        _check(lib.gc_batch_load(cnt, rps, cis, self.ns.ctypes.data, 0, self.stream, ctypes.byref(h)))
        self._h = h
        self.count = cnt

    def close(self):
        if getattr(self, "_h", None):
            load().gc_batch_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def greedy(self, ks, active_target: int = 0, lanes: int = 0, capture: bool = False, timeout_ms: int = 0,
               grid_min_n: int = 0, round1_bound: bool = True):
        ks = np.ascontiguousarray(ks, dtype=np.int32)
        o = Opts()
        load().gc_opts_default(ctypes.byref(o))
        o.active_target, o.step_lanes = active_target, lanes
        o.batch_grid_min_n = grid_min_n
        o.flags = (GC_OPT_CAPTURE if capture else 0) | (0 if round1_bound else GC_OPT_NO_ROUND1_BOUND)
        if timeout_ms:
            o.timeout_ms = timeout_ms
        groups = np.zeros(max(int(ks.sum()), 1), dtype=np.int32)
        far = np.zeros(self.count, dtype=np.int64)
        st = Stats()
        _check(load().gc_batch_greedy(self._h, ks.ctypes.data, ctypes.byref(o), groups.ctypes.data, far.ctypes.data,
                                      ctypes.byref(st)))
        out, pos = [], 0
        for k in ks:
            out.append(groups[pos:pos + k].copy())
            pos += k
        return out, far, st.as_dict()


def greedy_batch(graphs, ks, active_target: int = 0, lanes: int = 0, timeout_ms: int = 0):
    """gc_greedy_batch over existing Graph handles: (groups, farness, stats)."""
    lib = load()
    cnt = len(graphs)
    ks = np.ascontiguousarray(ks, dtype=np.int32)
    hs = (ctypes.c_void_p * cnt)(*[G._h.value for G in graphs])
    outs = [np.zeros(max(int(k), 1), dtype=np.int32) for k in ks]
    optr = (ctypes.c_void_p * cnt)(*[o.ctypes.data for o in outs])
    far = np.zeros(cnt, dtype=np.int64)
    o = Opts()
    lib.gc_opts_default(ctypes.byref(o))
    o.active_target, o.step_lanes = active_target, lanes
    if timeout_ms:
        o.timeout_ms = timeout_ms
    st = Stats()
    _check(lib.gc_greedy_batch(hs, ks.ctypes.data, cnt, ctypes.byref(o), optr, far.ctypes.data, ctypes.byref(st)))
    return [out[:k] for out, k in zip(outs, ks)], far, st.as_dict()
