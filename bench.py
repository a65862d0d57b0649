"""Benchmark: time to a size-k Greedy++ group on the GPU (plus pruned-BFS GTEPS).

Workload (one step): the whole hot path -- round 0 (top-1 closeness), d_S,
and k-1 lazy rounds of exact pruned-BFS gains -- on a seeded R-MAT graph of
scale 24 (edge factor 16, a=.57 b=.19 c=.19, seed 1, largest connected
component: 8.86M vertices, 521M adjacency entries), k = 50.  --scale/--k pick
another R-MAT size (scale 20, k = 100 is the earlier headline and is reported
as an extra).

value = size-k groups per second over all ranks (each rank solves its own
replica; no collective on the data path), with the CSR resident in HBM.
e2e   = the same through the public API from pinned host buffers: load the
        CSR (H2D), run, read the group back (D2H), free.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gc|reference]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "time to size-k group and pruned-BFS GTEPS, learned+batched vs plain GPU greedy"
WORKLOAD = "rmat_s24_ef16_lcc_k50"
L2_FLUSH_BYTES = 512 << 20


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="gc", choices=["gc", "reference"])
    p.add_argument("--k", type=int, default=50)
    p.add_argument("--scale", type=int, default=24)
    p.add_argument("--e2e-steps", type=int, default=0, help="0 = same as --steps")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-extras", action="store_true",
                   help="skip the plain-vs-learned+batched comparison legs")
    p.add_argument("--batch-graphs", type=int, default=256,
                   help="graphs of the mixed batched workload (0 = skip)")
    return p.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(x: float, device="cpu") -> float:
    """The largest value of x over the ranks of the default process group
    (x itself without one); every rank gets it."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(world: int, ms_per_step: float) -> float:
    """Whole-job throughput: each of `world` replicas solves one group per
    step, and a step takes ms_per_step (the slowest rank's time)."""
    return world * 1000.0 / ms_per_step


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:  # pragma: no cover
        return os.cpu_count() or 1


def workload_graph(scale: int):
    from paper_1710_01144_gb300 import graphgen

    return graphgen.rmat(scale, 16.0, 0.57, 0.19, 0.19, seed=1)


def config_dict(args, n, nnz, l2_note):
    return {"workload": "rmat_s%d_ef16_lcc_k%d" % (args.scale, args.k),
            "graph": "R-MAT scale %d, edge factor 16, (a,b,c)=(.57,.19,.19), seed 1, "
                     "symmetrised, deduplicated, largest component" % args.scale,
            "n": int(n), "nnz": int(nnz), "k": args.k, "l2": l2_note,
            "parallelism": "replicas (one independent solve per GPU)"}


# ------------------------------------------------------------------ clocks --
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str | None):
        self.gpu_id = gpu_id
        self.proc = None
        self.lines = []

    def start(self):
        cmd = ["nvidia-smi", "--query-gpu=" + self.Q, "--format=csv,noheader,nounits", "-lms", "100"]
        if self.gpu_id:
            cmd += ["-i", self.gpu_id]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# sources of each profiled kernel: a committed DRAM figure (profiles/) is used
# only while they are unchanged
KERNEL_SOURCES = {
    "k_round0_wide": ("gc_round0.cu", "gc_device.cuh", "gc_internal.cuh"),
    "k_gains64": ("gc_gain.cu", "gc_cta.cuh", "gc_device.cuh", "gc_internal.cuh"),
    "k_lazy_rounds": ("gc_lazy.cu", "gc_lazy.cuh", "gc_grid.cuh", "gc_cta.cuh", "gc_mlp.cuh", "gc_device.cuh",
                      "gc_internal.cuh"),
}
TRAFFIC_FILES = {
    "k_round0_wide": os.path.join(ROOT, "profiles", "dram_traffic_round0_wide_rmat.txt"),
    "k_gains64": os.path.join(ROOT, "profiles", "dram_traffic_rmat_s20_k100.txt"),
    "k_lazy_rounds": os.path.join(ROOT, "profiles", "dram_traffic_lazy_rounds_rmat_s24.txt"),
}


def kernel_hash(kernel: str) -> str:
    h = hashlib.sha256()
    for name in KERNEL_SOURCES[kernel]:
        with open(os.path.join(ROOT, "paper_1710_01144_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def profiled_traffic(kernel: str, workload: str):
    """DRAM bytes (read + write) per launch of `kernel` from the committed ncu
    summary, scaled to `workload` where the summary gives a per-workload figure,
    if the summary was taken on the current sources (None otherwise)."""
    path = TRAFFIC_FILES.get(kernel)
    if not path or not os.path.exists(path):
        return None
    kv = {}
    for line in open(path):
        if "=" in line and not line.lstrip().startswith("#"):
            a, b = line.split("=", 1)
            kv[a.strip()] = b.strip()
    if kv.get(kernel + ".source_sha256_16") != kernel_hash(kernel):
        return None
    for key in (kernel + "." + workload + ".dram_bytes_per_launch", kernel + ".dram_bytes_per_launch"):
        try:
            return float(kv[key])
        except (KeyError, ValueError):
            continue
    return None


def lazy_kernel_bytes(t) -> float:
    """Algorithmic bytes of the persistent lazy kernel: its gain phases (the
    model below), the claim log (16 B per entry written by the gain phases and
    per entry read by a d_S update), its relabel-BFS d_S updates (row pointers
    8 B per frontier entry, 4 B per adjacency entry) and every update's lowered
    labels (4 B each), and its selection passes (list id, bound and stamp: 16 B
    per active-list entry read)."""
    return (algorithmic_bytes(t["lazy_frontier"], t["lazy_edges"], t["lazy_pushes"], t["lazy_lanes"]) +
            16.0 * t.get("lazy_log_entries", 0) + 16.0 * t.get("lazy_upd_log", 0) +
            8.0 * t["lazy_upd_frontier"] + 4.0 * t["lazy_upd_edges"] + 4.0 * t["lazy_upd_relabels"] +
            16.0 * t["lazy_sel_scanned"])


def algorithmic_bytes(frontier, edges, pushes, lanes) -> float:
    """Bytes the 64-lane pruned BFS must move: per frontier entry the row
    pointers (8 B) and its lane word (8 B); 4 B per adjacency entry scanned;
    per vertex entering a next frontier its d_S value (4 B) and a visited and a
    next-level lane word (2 x 8 B); 8 B per candidate gain written."""
    return 16.0 * frontier + 4.0 * edges + 20.0 * pushes + 8.0 * lanes


def round0_kernel_bytes(t, n) -> float:
    """Algorithmic bytes of the wide round-0 kernel (bottom-up bit-parallel
    BFScut, B = r0_width lanes, B/8 bytes per lane word): in the bottom-up
    passes, the row pointers (8 B) of every vertex they visit and the visited
    word (B/8 B) of every vertex whose row they consider (the far-vertex probe
    stages visit only part of the vertices); 4 B per adjacency entry read; per
    vertex whose claim is written, its visited and claim words (2 B/8 B) and
    the later clear of the claim word (B/8 B); per top-down adjacency entry 4 B
    plus the 8-byte visited word it sets and its later clear (20 B: a
    count-only batch sets no distance-1 claim word; the first-pass batches,
    where nearly every top-down entry lies, are count-only, and the second word
    that full batches set is not counted); per batch that wrote bottom-up
    levels the dense clear of the visited words (n B/8 B).
    Gathered frontier words are not counted: each re-reads a word already
    counted when it was written (most hit L2)."""
    wb = t["r0_width"] / 8.0 if t["r0_width"] else 0.0
    return (8.0 * t["r0_bu_vertices"] + wb * t["r0_bu_visreads"] + 4.0 * t["r0_bu_scanned"] +
            3.0 * wb * t["r0_bu_rows"] + 20.0 * t["r0_td_edges"] + t["r0_dense_clears"] * n * wb)


def golden_for(scale: int, k: int):
    """(s0, f({s0})) and the group from the committed oracle answer for this
    workload, if there is one (tests/golden/)."""
    path = os.path.join(ROOT, "tests", "golden", "rmat%d_ef16_k%d.txt" % (scale, k))
    if not os.path.exists(path):
        return None
    out = {}
    for line in open(path):
        if line.startswith("#") or not line.strip():
            continue
        key, _, val = line.partition(" ")
        out[key] = val.split()
    return out


# --------------------------------------------------------------- gc arm ----
def run_gc(args):
    import torch

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_1710_01144_gb300 import build as gcbuild
    from paper_1710_01144_gb300 import gc

    gcbuild.build()
    rp, ci = workload_graph(args.scale)
    n, nnz = rp.size - 1, ci.size
    G = gc.Graph(rp, ci, validate=True)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()

    def barrier():
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        grp0, f0, _ = G.greedy(args.k)
    barrier()
    props = torch.cuda.get_device_properties(local)
    uuid = getattr(props, "uuid", None)
    clk = ClockSampler(("GPU-" + str(uuid)) if uuid is not None else None)
    clk.start()
    times, stats = [], []
    barrier()
    for _ in range(args.steps):
        flush.fill_(1)  # evict L2 between steps (outside the timed window)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        grp, f, st = G.greedy(args.k)
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
        stats.append(st)
        assert np.array_equal(grp, grp0) and f == f0, "non-deterministic group"
    barrier()
    clocks = clk.stop()
    t_step = max_over_ranks(sum(times) / len(times), "cuda")

    # e2e: public API from pinned host buffers, copies inside the timed region
    trp = torch.from_numpy(rp).pin_memory()
    tci = torch.from_numpy(ci).pin_memory()
    hrp, hci = trp.numpy(), tci.numpy()
    e2e_steps = args.e2e_steps or args.steps
    G.close()
    with gc.Graph(hrp, hci) as Gw:  # warm the allocator path once
        Gw.greedy(args.k)
    barrier()
    e2e_t, e2e_parts = [], []
    for _ in range(e2e_steps):
        flush.fill_(1)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        with gc.Graph(hrp, hci) as Ge:
            t1 = time.perf_counter()
            g_e, f_e, _ = Ge.greedy(args.k)
            t2 = time.perf_counter()
        t3 = time.perf_counter()
        e2e_t.append((t3 - t0) * 1e3)
        e2e_parts.append(((t1 - t0) * 1e3, (t2 - t1) * 1e3, (t3 - t2) * 1e3))
        assert np.array_equal(g_e, grp0) and f_e == f0
    barrier()
    t_e2e = max_over_ranks(sum(e2e_t) / len(e2e_t), "cuda")

    if rank == 0:
        tot = {k: sum(s[k] for s in stats) for k in stats[0]}
        tot["r0_width"] = stats[0]["r0_width"]  # a width, not a count
        peak, peak_kind = measured_peaks()
        workload = "rmat_s%d_ef16_lcc_k%d" % (args.scale, args.k)

        def roof(name, bytes_alg, ms, launches):
            achieved = bytes_alg / (ms * 1e-3) / 1e9 if ms > 0 else 0.0
            return {"kernel": name, "bound": "hbm", "achieved": achieved, "peak": peak, "peak_kind": peak_kind,
                    "unit": "GB/s", "frac": achieved / peak, "traffic": profiled_traffic(name, workload),
                    "algorithmic_bytes_per_launch": bytes_alg / max(launches, 1),
                    "avg_launch_ms": ms / max(launches, 1), "launches": launches,
                    "share_of_step": ms / sum(times)}

        # every kernel family with its own timing, the largest device-time share first
        roofs = []
        if tot["r0_batches"] > 0:
            roofs.append(roof("k_round0_wide", round0_kernel_bytes(tot, n), tot["ms_round0_wide"], args.steps))
        if tot["lazy_launches"] > 0:
            roofs.append(roof("k_lazy_rounds", lazy_kernel_bytes(tot), tot["ms_lazy_kernel"], tot["lazy_launches"]))
        if tot["gain64_launches"] > 0:
            roofs.append(roof("k_gains64", algorithmic_bytes(tot["gain64_frontier"], tot["gain64_edges"],
                                                             tot["gain64_pushes"], tot["gain64_lanes"]),
                              tot["ms_gain64"], tot["gain64_launches"]))
        roofs.sort(key=lambda r: -r["share_of_step"])
        per = lambda k: tot[k] / args.steps
        line = {
            "metric": METRIC,
            "value": job_value(ws, t_step),
            "unit": "size-%d groups/s" % args.k,
            "n_gpus": ws,
            "steps": args.steps,
            "warmup": args.warmup,
            "ms_per_step": t_step,
            "time_to_group_ms": t_step,
            "time_to_group_without_round0_ms": t_step - per("ms_round0"),
            "higher_is_better": True,
            "scaling": "weak",
            "vs_baseline": None,
            "dtype": "int64",
            "data": "synthetic (seeded R-MAT generator)",
            "config": config_dict(args, n, nnz, "flushed between steps (512 MiB write outside the timed window)"),
            "gteps_scalar": tot["edges_scalar"] / (sum(times) * 1e-3) / 1e9,
            "gteps_union": tot["edges_union"] / (sum(times) * 1e-3) / 1e9,
            "work_per_step": dict({k: tot[k] // args.steps for k in
                                   ("evals", "steps", "batches", "edges_scalar", "edges_union", "levels",
                                    "round0_evals", "gain_launches", "kernel_launches", "r0_batches", "r0_levels",
                                    "r0_bu_scanned", "r0_bu_gathers", "r0_td_edges", "r0_probes", "r0_probe_cut",
                                    "r0_bu_vertices", "r0_bu_visreads")}, r0_width=tot["r0_width"]),
            "ms_round0": per("ms_round0"),
            "ms_round1": per("ms_round1"),
            "ms_phases": {k: per(k) for k in ("ms_round0_wide", "ms_r0_topdown", "ms_r0_bottomup", "ms_r0_clear",
                                              "ms_lazy_kernel", "ms_lazy_select", "ms_lazy_gain", "ms_lazy_update")},
            "group_farness": int(f0),
            "group_prefix": [int(x) for x in grp0[:10]],
            "roofline": roofs[0] if roofs else None,
            "roofline_other_kernels": roofs[1:],
            "e2e": {"value": job_value(ws, t_e2e), "unit": "size-%d groups/s" % args.k,
                    "ms_per_step": t_e2e,
                    "h2d_bytes_per_step": int(rp.nbytes + ci.nbytes),
                    "d2h_bytes_per_step": int(4 * args.k + 8),
                    "ms_load_greedy_free": [round(float(np.mean([p[i] for p in e2e_parts])), 2) for i in range(3)]},
            "gpu_launches": int(tot["kernel_launches"]),
            "clocks": clocks,
        }
        gold = golden_for(args.scale, args.k)
        if gold:
            line["same_group_as_oracle_golden"] = bool(
                [int(x) for x in gold["group"]] == [int(x) for x in grp0] and int(gold["farness"][-1]) == f0)
        if ws == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(rp, ci, args, grp0, f0)
        if not args.no_extras:
            line["comparison"] = comparison_legs(gc, rp, ci, args, grp0, f0)
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()


def _best_ms(fn, reps):
    import torch

    best, out = float("inf"), None
    for _ in range(reps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        out = fn()
        torch.cuda.synchronize()
        best = min(best, (time.perf_counter() - t0) * 1e3)
    return best, out


def comparison_legs(gc, rp, ci, args, grp0, f0):
    """Plain GPU lazy greedy (the library's default path with the proposal
    off) against the learned proposal and the batched form, same GPU, same
    groups; plus the earlier R-MAT scale-20, k = 100 workload."""
    from paper_1710_01144_gb300 import graphgen, proposal

    out = {}
    with gc.Graph(rp, ci) as G:
        ms, (g, f, st0) = _best_ms(lambda: G.greedy(args.k), 3)
        assert np.array_equal(g, grp0) and f == f0
        out["plain_gpu_lazy_ms"] = ms
        out["plain_steps"] = st0["steps"]
        out["plain_evals"] = st0["evals"]
        # learned proposal trained on this family's exact gains (other seeds, scales 18-20)
        t0 = time.perf_counter()
        train = [graphgen.rmat(sc, 16.0, seed=s) for sc, s in ((18, 2), (19, 3), (20, 4))]
        net, (m, l0, l1) = proposal.train(train, k=min(args.k, 50))
        out["proposal"] = {"train_graphs": "R-MAT scales 18, 19, 20, ef 16, seeds 2, 3, 4", "samples": m,
                           "loss_initial": l0, "loss_final": l1, "train_s": time.perf_counter() - t0}
        G.set_proposal(net, 0)  # round 1's first batch (the lazy fill cannot remove a required evaluation)
        ms, (g, f, st) = _best_ms(lambda: G.greedy(args.k, use_proposal=True), 3)
        assert np.array_equal(g, grp0) and f == f0
        out["learned_ms"] = ms
        out["learned_steps"] = st["steps"]
        out["learned_evals"] = st["evals"]
        G.set_proposal(None)
        net.close()
    out["speedup_learned_vs_plain"] = out["plain_gpu_lazy_ms"] / out["learned_ms"]
    rp20, ci20 = graphgen.rmat_s20_ef16() if (args.scale != 20) else (rp, ci)
    with gc.Graph(rp20, ci20) as G20:
        g20, _, _ = G20.greedy(100)
        ms, _ = _best_ms(lambda: G20.greedy(100), 5)
        out["rmat_s20_ef16_lcc_k100_ms"] = ms
        out["gain_lanes_rmat_s20"] = gain_lanes_leg(G20, int(g20[0]))
    if args.batch_graphs > 0:
        out["mixed_batch"] = mixed_batch_leg(gc, args.batch_graphs)
    return out


def gain_lanes_leg(G, s0):
    """Round 1 without bounds as one gc_marginal_gains call: the gain of every
    vertex for S = {s0}, at 64, 128 and 256 candidates per CTA batch (identical
    results), with the kernel's device time and its byte model per width."""
    n = G.n
    allv = np.arange(n, dtype=np.int32)
    res, ref = {}, None
    for lanes in (64, 128, 256):
        G.set_gain_lanes(lanes)
        G.gains([s0], allv)  # warm-up (and the wide kernel's workspace)
        best = None
        for _ in range(3):
            g, st = G.gains([s0], allv, stats=True)
            if best is None or st["ms_gain_kernel"] < best["ms_gain_kernel"]:
                best = st
        if ref is None:
            ref = g
        assert np.array_equal(g, ref), "gains differ between lane widths"
        w = lanes // 64
        # per frontier entry: row pointers and its W claim words; per adjacency
        # entry 4 B; per push: d_S, visited and claim words; 8 B per gain
        bytes_alg = ((8.0 + 8.0 * w) * best["frontier"] + 4.0 * best["edges_union"]
                     + (4.0 + 16.0 * w) * best["pushes"] + 8.0 * n)
        res[str(lanes)] = {"ms_gain_kernel": best["ms_gain_kernel"], "batches": best["batches"],
                           "edges_union": best["edges_union"], "edges_scalar": best["edges_scalar"],
                           "gteps_scalar": best["edges_scalar"] / (best["ms_gain_kernel"] * 1e6),
                           "achieved_gbs": bytes_alg / (best["ms_gain_kernel"] * 1e6)}
    G.set_gain_lanes(64)
    res["fastest"] = min((k for k in res), key=lambda k: res[k]["ms_gain_kernel"])
    return res


def mixed_batch_leg(gc, count):
    """The serving-style workload: `count` BA/R-MAT graphs, n log-uniform in
    [1e4, 5e5], degree 4-32, k in 5-50, solved (a) in one persistent launch
    replayed from a captured CUDA graph with autotuned lanes/list size and (b)
    one graph at a time through gc_greedy; groups must be identical."""
    from paper_1710_01144_gb300 import autotune, graphgen

    items = graphgen.batch_params(count, seed=1)
    graphs = [graphgen.batch_graph(it) for it in items]
    ks = np.array([min(it.k, rp.size - 1) for it, (rp, _) in zip(items, graphs)], dtype=np.int32)
    sizes = [rp.size - 1 for rp, _ in graphs]
    res = {"graphs": count, "vertices": int(sum(sizes)), "entries": int(sum(ci.size for _, ci in graphs)),
           "sum_k": int(ks.sum())}
    with gc.Batch(graphs) as B:
        space = [{"lanes": 64, "A": 4096}, {"lanes": 32, "A": 1024}]
        best, entry = autotune.tune_batch(B, ks, sizes, reps=1, space=space)
        res["autotuned"] = best
        res["autotune_trials"] = entry.get("trials")
        # first call records the CUDA graph, the timed call replays it
        B.greedy(ks, active_target=best["A"], lanes=best["lanes"], capture=True)
        ms, (groups, far, st) = _best_ms(
            lambda: B.greedy(ks, active_target=best["A"], lanes=best["lanes"], capture=True), 1)
        res["batched_ms"] = ms
        res["graph_replay"] = bool(st["graph_replay"])
        res["iterations"] = int(st["steps"])
    seq = 0.0
    same = True
    for i, ((rp, ci), k) in enumerate(zip(graphs, ks)):
        with gc.Graph(rp, ci) as G:
            ms, (g, f, _) = _best_ms(lambda: G.greedy(int(k)), 1)
        seq += ms
        same = same and np.array_equal(g, groups[i]) and f == far[i]
    res["sequential_gc_greedy_ms"] = seq
    res["groups_identical"] = bool(same)
    res["speedup_batched_vs_sequential"] = seq / res["batched_ms"]
    return res


def oracle_sample_seconds(rp, ci, args, m, seed, cores):
    """Estimated wall seconds of the CPU oracle (CPU Greedy++, as it stands) on
    the whole workload, from a bounded sample: its two dominant steps -- the
    round-0 BFScut (Sec. 3.1, Algorithm 3) and the round-1 pruned SSSP
    (Sec. 4.1) -- timed on m seeded random vertices and scaled by n / m.  The
    cut uses the final best farness from the start (the real run starts from a
    looser one), and the lazy rounds >= 2 are left out, so the estimate is
    below the oracle's true time."""
    import oracle

    n = rp.size - 1
    gold = golden_for(args.scale, args.k)
    if gold:  # the oracle's own answer, stored once (tests/golden/)
        s0, f_s0 = int(gold["group"][0]), int(gold["farness"][0])
    elif args.scale <= 22:
        s0, f_s0, _ = oracle.top1_closeness(rp, ci, threads=cores)
    else:  # the oracle's top-1 search alone takes tens of minutes here
        return None
    rng = np.random.default_rng(seed)
    cand = rng.choice(n, size=min(m, n), replace=False).astype(np.int32)
    t0 = time.perf_counter()
    t_cut, t_gain, scanned = oracle.greedypp_cost_sample(rp, ci, s0, f_s0, cand, threads=cores)
    wall = time.perf_counter() - t0
    return (t_cut + t_gain) * n / cand.size, wall, cand.size


def cpu_baseline(rp, ci, args, grp_gpu, f_gpu):
    """The CPU oracle on the host cores.  Where the whole oracle run finishes in
    seconds (scale <= 20) it is timed in full; otherwise a bounded sample of it
    is timed and scaled to the workload (oracle_sample_seconds)."""
    import oracle

    cores = host_cores()
    unit = "size-%d groups/s" % args.k
    if args.scale <= 20:
        t0 = time.perf_counter()
        grp, ft, _, st = oracle.greedypp(rp, ci, args.k, threads=cores)
        dt = time.perf_counter() - t0
        return {"value": 1.0 / dt, "unit": unit, "cores": cores, "kind": "oracle",
                "sample": "full workload, one run: CPU Greedy++ (BFScut top-1 closeness, pruned SSSP, "
                          "lazy bounds; OpenMP) k=%d on the same graph" % args.k,
                "seconds": dt, "same_group_as_gpu": bool(np.array_equal(grp, grp_gpu) and ft[-1] == f_gpu)}
    m = 20000
    r = oracle_sample_seconds(rp, ci, args, m, 1, cores)
    if r is None:
        return {"value": None, "unit": unit, "cores": cores, "kind": "oracle",
                "sample": "not run: no stored oracle answer for this workload in tests/golden/"}
    est, wall, used = r
    return {"value": 1.0 / est, "unit": unit, "cores": cores, "kind": "oracle",
            "sample": ("bounded sample: CPU Greedy++'s round-0 BFScut (against the final best farness) and "
                       "round-1 pruned SSSP on %d seeded random vertices of the same graph, scaled by n/%d; "
                       "later lazy rounds left out; the estimate (%.0f s for the whole workload) is below "
                       "the oracle's true time" % (used, used, est)),
            "sample_wall_s": wall, "estimated_workload_s": est}


# -------------------------------------------------------- reference arm ----
def run_reference(args):
    """The CPU oracle (CPU Greedy++) on the host cores, on the same workload,
    metric and unit; under torchrun only rank 0 runs.  At scale <= 20 each step
    is the whole oracle run; above it each step is a bounded sample of the
    oracle's work (see oracle_sample_seconds), scaled to the workload."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle

    rp, ci = workload_graph(args.scale)
    cores = host_cores()
    unit = "size-%d groups/s" % args.k
    if args.scale <= 20:
        for _ in range(args.warmup):
            oracle.greedypp(rp, ci, args.k, threads=cores)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            grp, ft, _, st = oracle.greedypp(rp, ci, args.k, threads=cores)
        dt = (time.perf_counter() - t0) / args.steps
        sample = "full workload per step: CPU Greedy++ k=%d" % args.k
        farness = int(ft[-1])
    else:
        m = 2000
        if oracle_sample_seconds(rp, ci, args, 1, 99, cores) is None:
            print(json.dumps({"impl": "reference", "unavailable": "no stored oracle answer for this workload "
                              "(tests/golden/); the oracle's own top-1 search takes tens of minutes"}), flush=True)
            return
        for i in range(args.warmup):
            oracle_sample_seconds(rp, ci, args, m, 100 + i, cores)
        ests = [oracle_sample_seconds(rp, ci, args, m, 1 + i, cores)[0] for i in range(args.steps)]
        dt = sum(ests) / len(ests)
        sample = ("bounded sample per step: CPU Greedy++'s round-0 BFScut and round-1 pruned SSSP on %d seeded "
                  "random vertices, scaled by n/%d (an estimate below the oracle's true time)" % (m, m))
        gold = golden_for(args.scale, args.k)
        farness = int(gold["farness"][-1]) if gold else None
    v = 1.0 / dt
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": unit, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3, "time_to_group_ms": dt * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
        "data": "synthetic (seeded R-MAT generator)",
        "config": config_dict(args, rp.size - 1, ci.size, "n/a (CPU)"),
        "cpu_baseline": {"value": v, "unit": unit, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": v, "unit": unit, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "group_farness": farness,
    }), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gc(args)


if __name__ == "__main__":
    main()
