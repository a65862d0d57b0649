"""Writes tests/golden/rmat24_ef16_k50.txt: the Greedy++ group of size 50 on the
seeded R-MAT scale-24 graph, computed by the CPU oracle only.

Parity for this workload cannot rerun the CPU oracle inside a GPU test (its
top-1 closeness search alone takes hours on the host cores), so the oracle's
answer is stored here once.  Greedy++ itself is Algorithm 2 with the pruned
SSSP of Sec. 4.1 and the lazy bounds of Sec. 4.2 (smallest id on ties); the
stored group is what oracle.greedypp returns.  The graph is identified by its
size and a SHA-256 of its CSR arrays, so a change of the generator shows up as
a mismatch instead of a silently different workload.

Usage: python tests/golden/make_rmat24_k50.py [threads]
"""
import hashlib
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1710_01144_gb300 import graphgen  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "rmat24_ef16_k50.txt")
K = 50


def csr_sha256(rp, ci) -> str:
    h = hashlib.sha256()
    h.update(rp.astype("<i4").tobytes())
    h.update(ci.astype("<i4").tobytes())
    return h.hexdigest()


def main():
    threads = int(sys.argv[1]) if len(sys.argv) > 1 else oracle.default_threads()
    rp, ci = graphgen.rmat_s24_ef16()
    t0 = time.time()
    grp, ft, gt, st = oracle.greedypp(rp, ci, K, threads=threads)
    dt = time.time() - t0
    with open(OUT, "w") as f:
        f.write("# Greedy++ (CPU oracle, oracle.greedypp) on R-MAT scale 24, edge factor 16,\n")
        f.write("# (a,b,c) = (.57,.19,.19), seed 1, symmetrised, deduplicated, largest component;\n")
        f.write("# k = %d.  Algorithm 2 with the pruned SSSP of Sec. 4.1 and the lazy bounds of\n" % K)
        f.write("# Sec. 4.2, ties to the smallest id.  Written by make_rmat24_k50.py.\n")
        f.write("# oracle time %.1f s on %d host threads (informational)\n" % (dt, threads))
        f.write("n %d\n" % (rp.size - 1))
        f.write("nnz %d\n" % ci.size)
        f.write("sha256 %s\n" % csr_sha256(rp, ci))
        f.write("group %s\n" % " ".join(str(int(v)) for v in grp))
        f.write("farness %s\n" % " ".join(str(int(v)) for v in ft))
    print("wrote", OUT, "in %.1f s" % dt)


if __name__ == "__main__":
    main()
