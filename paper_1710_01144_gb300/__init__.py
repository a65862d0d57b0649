"""GB300-native Greedy++ group-closeness maximization (arXiv:1710.01144).

The hot path (pruned-BFS marginal gains, distance-to-group maintenance, the
lazy greedy loop) runs in hand-written CUDA kernels behind the C ABI declared
in ``include/gc.h``; ``paper_1710_01144_gb300.gc`` is the thin ctypes binding.
Importing this package loads nothing; the CUDA library is loaded on first use
of ``paper_1710_01144_gb300.gc``.
"""
