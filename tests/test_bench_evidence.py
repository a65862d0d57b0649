"""Host logic behind the bench line's roofline objects, on the CPU: the byte
models add up their work counters as their docstrings state, and a committed
DRAM figure is used only while the sources of its kernel are the ones it was
captured on (the test checks that rule, not that the figures are current)."""
import importlib.util
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_ev", os.path.join(ROOT, "bench.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


def test_round0_byte_model():
    b = _bench()
    t = {"r0_width": 256, "r0_bu_vertices": 10, "r0_bu_visreads": 7, "r0_bu_scanned": 100, "r0_bu_rows": 3,
         "r0_td_edges": 5, "r0_dense_clears": 2}
    wb = 256 / 8
    n = 1000
    want = 8 * 10 + wb * 7 + 4 * 100 + 3 * wb * 3 + 20 * 5 + 2 * n * wb
    assert b.round0_kernel_bytes(t, n) == want
    t["r0_width"] = 0  # the kernel did not run: only the width-free terms
    assert b.round0_kernel_bytes(t, n) == 8 * 10 + 4 * 100 + 20 * 5


def test_gain_byte_model():
    b = _bench()
    assert b.algorithmic_bytes(frontier=2, edges=10, pushes=3, lanes=64) == 16 * 2 + 4 * 10 + 20 * 3 + 8 * 64


def test_committed_traffic_follows_the_source_hash(monkeypatch):
    b = _bench()
    for kernel, workload in (("k_round0_wide", "rmat_s24_ef16_lcc_k50"), ("k_lazy_rounds", "rmat_s24_ef16_lcc_k50")):
        captured = None
        for line in open(b.TRAFFIC_FILES[kernel]):
            if line.startswith(kernel + ".source_sha256_16"):
                captured = line.split("=", 1)[1].strip()
        got = b.profiled_traffic(kernel, workload)
        if captured == b.kernel_hash(kernel):  # the figure describes these sources
            assert got is not None and got > 0, kernel
        else:
            assert got is None, kernel
        assert b.profiled_traffic(kernel, "no_such_workload") is None
        monkeypatch.setattr(b, "kernel_hash", lambda k: "0" * 16)  # the sources changed since the capture
        assert b.profiled_traffic(kernel, workload) is None
        monkeypatch.undo()
    assert b.profiled_traffic("k_unknown", "rmat_s24_ef16_lcc_k50") is None
