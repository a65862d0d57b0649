"""Writes tests/golden/batch256_groups.txt: the Greedy++ group and farness of
each graph of the seeded 256-graph mixed workload (BA and R-MAT graphs, n
log-uniform in [1e4, 5e5], average degree 4-32, k in 5-50), computed by the
CPU oracle only (oracle.greedypp: Algorithm 2 with the pruned SSSP of Sec. 4.1
and the lazy bounds of Sec. 4.2, ties to the smallest id).  The whole mix takes
the oracle minutes, too long to rerun inside every GPU test; each graph is
identified by its size and a SHA-256 of its CSR.

Usage: python tests/golden/make_batch256.py [threads]
"""
import hashlib
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1710_01144_gb300 import graphgen  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "batch256_groups.txt")


def csr_sha256(rp, ci) -> str:
    h = hashlib.sha256()
    h.update(rp.astype("<i4").tobytes())
    h.update(ci.astype("<i4").tobytes())
    return h.hexdigest()


def main():
    threads = int(sys.argv[1]) if len(sys.argv) > 1 else oracle.default_threads()
    items = graphgen.batch_params(256, seed=1)
    t0 = time.time()
    lines = []
    for i, it in enumerate(items):
        rp, ci = graphgen.batch_graph(it)
        k = min(it.k, rp.size - 1)
        grp, ft, _, _ = oracle.greedypp(rp, ci, k, threads=threads)
        lines.append("graph %d %s n %d nnz %d k %d sha256 %s farness %d group %s" % (
            i, it.family, rp.size - 1, ci.size, k, csr_sha256(rp, ci)[:32], int(ft[-1]),
            " ".join(str(int(v)) for v in grp)))
    dt = time.time() - t0
    with open(OUT, "w") as f:
        f.write("# Greedy++ (CPU oracle, oracle.greedypp) on each graph of the 256-graph mixed\n")
        f.write("# workload (graphgen.batch_params(256, seed=1)).  Algorithm 2 with the pruned SSSP\n")
        f.write("# of Sec. 4.1 and the lazy bounds of Sec. 4.2, ties to the smallest id.  Written by\n")
        f.write("# make_batch256.py; oracle time %.1f s on %d host threads (informational).\n" % (dt, threads))
        f.write("\n".join(lines) + "\n")
    print("wrote", OUT, "in %.1f s" % dt)


if __name__ == "__main__":
    main()
