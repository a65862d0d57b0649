"""Tiny named graphs as int32 CSR (inputs only: no distances, no gains).

Used by the oracle pins and by the GPU parity tests alike.
"""
import numpy as np


def csr_from_edges(n, edges):
    """Simple undirected graph from an edge list (duplicates/self-loops dropped)."""
    adj = [set() for _ in range(n)]
    for a, b in edges:
        if a != b:
            adj[a].add(b)
            adj[b].add(a)
    rp = np.zeros(n + 1, dtype=np.int32)
    for i in range(n):
        rp[i + 1] = rp[i] + len(adj[i])
    ci = np.array([w for i in range(n) for w in sorted(adj[i])], dtype=np.int32)
    return rp, ci


def path(n):
    return csr_from_edges(n, [(i, i + 1) for i in range(n - 1)])


def cycle(n):
    return csr_from_edges(n, [(i, (i + 1) % n) for i in range(n)])


def star(n):
    """Centre 0, leaves 1..n-1."""
    return csr_from_edges(n, [(0, i) for i in range(1, n)])


def complete(n):
    return csr_from_edges(n, [(i, j) for i in range(n) for j in range(i + 1, n)])


def grid(a, b):
    """a rows x b columns, row-major ids."""
    e = []
    for i in range(a):
        for j in range(b):
            v = i * b + j
            if j + 1 < b:
                e.append((v, v + 1))
            if i + 1 < a:
                e.append((v, v + b))
    return csr_from_edges(a * b, e)


def gnp_connected(n, p, seed):
    """Erdos-Renyi G(n,p) plus a random spanning path so it is connected."""
    rng = np.random.default_rng(seed)
    e = [(i, j) for i in range(n) for j in range(i + 1, n) if rng.random() < p]
    perm = rng.permutation(n)
    e += [(int(perm[i]), int(perm[i + 1])) for i in range(n - 1)]
    return csr_from_edges(n, e)


def tree_random(n, seed):
    rng = np.random.default_rng(seed)
    return csr_from_edges(n, [(i, int(rng.integers(0, i))) for i in range(1, n)])


def caterpillar(n_spine, legs):
    """Path of n_spine vertices, each with `legs` pendant leaves (many ties)."""
    e = [(i, i + 1) for i in range(n_spine - 1)]
    nxt = n_spine
    for i in range(n_spine):
        for _ in range(legs):
            e.append((i, nxt))
            nxt += 1
    return csr_from_edges(nxt, e)


def disjoint_union(*graphs):
    """Disconnected union (for the error paths)."""
    edges, off = [], 0
    for rp, ci in graphs:
        n = rp.size - 1
        for u in range(n):
            for k in range(rp[u], rp[u + 1]):
                edges.append((u + off, int(ci[k]) + off))
        off += n
    return csr_from_edges(off, edges)
