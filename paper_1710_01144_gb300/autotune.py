"""Autotuner for the launch parameters of the batched and single-graph solvers.

The parameters only change work and speed, never the groups (every candidate
setting is checked to return the same groups as the first one).  Results are
cached in a JSON file keyed by a signature of the workload.

Batched solver (`gc_batch_greedy`):
    lanes  -- candidates per round-1 batch (the candidate-batch width of one
              64-bit lane word: 16, 32 or 64)
    A      -- per-graph candidate-list capacity of the lazy rounds
Single-graph solver (`gc_greedy`):
    active_target -- candidate-list size of the persistent lazy kernel
    round1_heavy  -- highest-degree round-1 candidates evaluated grid-wide
Gain evaluation (`gc_marginal_gains`):
    gain_lanes    -- candidates per CTA batch of the bit-parallel pruned BFS
                     (64, 128 or 256: one, two or four 64-bit words per vertex)
"""
from __future__ import annotations

import hashlib
import json
import os
import time

import numpy as np

DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "gcgb300", "autotune.json")

BATCH_SPACE = [{"lanes": l, "A": a} for l in (16, 32, 64) for a in (256, 1024, 4096)]
SINGLE_SPACE = [{"active_target": a, "round1_heavy": h} for a in (512, 2048, 8192) for h in (256, 1024, 4096)]
GAIN_LANES_SPACE = (64, 128, 256)


def _load(path):
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(path, data):
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = path + ".%d.tmp" % os.getpid()
    with open(tmp, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def signature(kind: str, sizes, ks) -> str:
    h = hashlib.sha256()
    h.update(kind.encode())
    h.update(np.asarray(sizes, dtype=np.int64).tobytes())
    h.update(np.asarray(ks, dtype=np.int64).tobytes())
    return kind + ":" + h.hexdigest()[:20]


def _time(fn, reps):
    import torch

    best = float("inf")
    out = None
    for _ in range(reps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        out = fn()
        torch.cuda.synchronize()
        best = min(best, (time.perf_counter() - t0) * 1e3)
    return best, out


def tune_batch(batch, ks, sizes, reps: int = 2, cache: str | None = DEFAULT_CACHE, space=None, log=None):
    """Best {lanes, A} for gc_batch_greedy on this batch (cached)."""
    key = signature("batch", sizes, ks)
    data = _load(cache) if cache else {}
    if key in data:
        return data[key]["best"], data[key]
    results, ref = [], None
    for cfg in space or BATCH_SPACE:
        ms, (groups, far, _) = _time(lambda: batch.greedy(ks, active_target=cfg["A"], lanes=cfg["lanes"]), reps)
        if ref is None:
            ref = (groups, far)
        elif not (all(np.array_equal(a, b) for a, b in zip(groups, ref[0])) and np.array_equal(far, ref[1])):
            raise RuntimeError("autotune: setting %s changed a group" % cfg)
        results.append(dict(cfg, ms=ms))
        if log:
            log("batch %s: %.2f ms" % (cfg, ms))
    best = min(results, key=lambda r: r["ms"])
    entry = {"best": {"lanes": best["lanes"], "A": best["A"]}, "trials": results}
    if cache:
        data[key] = entry
        _store(cache, data)
    return entry["best"], entry


def tune_single(graph, k: int, reps: int = 2, cache: str | None = DEFAULT_CACHE, space=None, log=None):
    """Best {active_target, round1_heavy} for gc_greedy on this graph (cached)."""
    key = signature("single", [graph.n, graph.nnz], [k])
    data = _load(cache) if cache else {}
    if key in data:
        return data[key]["best"], data[key]
    results, ref = [], None
    for cfg in space or SINGLE_SPACE:
        ms, (grp, f, _) = _time(lambda: graph.greedy(k, **cfg), reps)
        if ref is None:
            ref = (grp, f)
        elif not (np.array_equal(grp, ref[0]) and f == ref[1]):
            raise RuntimeError("autotune: setting %s changed the group" % cfg)
        results.append(dict(cfg, ms=ms))
        if log:
            log("single %s: %.2f ms" % (cfg, ms))
    best = min(results, key=lambda r: r["ms"])
    entry = {"best": {kk: best[kk] for kk in ("active_target", "round1_heavy")}, "trials": results}
    if cache:
        data[key] = entry
        _store(cache, data)
    return entry["best"], entry


def tune_gain_lanes(graph, S, cand, reps: int = 3, cache: str | None = DEFAULT_CACHE, space=None, log=None):
    """Best candidates-per-batch width for gc_marginal_gains of this many
    candidates against a group of this size on this graph (cached), by the
    gain kernel's device time; every width must return the same gains.  The
    handle is left at the winning width."""
    key = signature("gains", [graph.n, graph.nnz], [int(np.size(S)), int(np.size(cand))])
    data = _load(cache) if cache else {}
    if key not in data:
        results, ref = [], None
        for lanes in space or GAIN_LANES_SPACE:
            graph.set_gain_lanes(lanes)
            graph.gains(S, cand)  # warm-up (allocates a wide kernel's workspace)
            best, got = float("inf"), None
            for _ in range(reps):
                got, st = graph.gains(S, cand, stats=True)
                best = min(best, st["ms_gain_kernel"])
            if ref is None:
                ref = got
            elif not np.array_equal(got, ref):
                raise RuntimeError("autotune: gain_lanes %d changed a gain" % lanes)
            results.append({"gain_lanes": lanes, "ms": best})
            if log:
                log("gains lanes %d: %.2f ms" % (lanes, best))
        win = min(results, key=lambda r: r["ms"])
        data[key] = {"best": {"gain_lanes": win["gain_lanes"]}, "trials": results}
        if cache:
            _store(cache, data)
    graph.set_gain_lanes(data[key]["best"]["gain_lanes"])
    return data[key]["best"], data[key]
