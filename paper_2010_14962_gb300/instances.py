"""Seeded synthetic QAOA instances (inputs only; no part of the method).

The paper evaluates on 3-regular QAOA: edges placed at random on a given
vertex set, disconnected graphs discarded (Sec. IV.A).  This module draws
such graphs (configuration model, rejecting self-loops, multi-edges and
disconnected graphs), the layer angles gamma_l, beta_l ~ U[0, pi), measured
bitstrings x and cut-count choices.  Both the CUDA path and the oracle take
their inputs from here; nothing here evaluates a gate, a tensor or an
amplitude.

All draws use numpy's PCG64 generator seeded with explicit integers, so the
same seed gives the same instance on every machine.
"""
from __future__ import annotations

import dataclasses

import numpy as np


def _connected(n: int, edges: np.ndarray) -> bool:
    parent = list(range(n))

    def find(a):
        while parent[a] != a:
            parent[a] = parent[parent[a]]
            a = parent[a]
        return a

    for a, b in edges:
        ra, rb = find(int(a)), find(int(b))
        if ra != rb:
            parent[ra] = rb
    root = find(0)
    return all(find(i) == root for i in range(n))


def random_regular_graph(n: int, degree: int = 3, seed: int = 0) -> np.ndarray:
    """Edges (m x 2, int32, each row i < j, rows sorted) of a connected simple
    `degree`-regular graph on n vertices."""
    if (n * degree) % 2 or degree >= n:
        raise ValueError("n * degree must be even and degree < n")
    rng = np.random.Generator(np.random.PCG64(seed))
    while True:
        stubs = np.repeat(np.arange(n), degree)
        rng.shuffle(stubs)
        pairs = stubs.reshape(-1, 2)
        a = np.minimum(pairs[:, 0], pairs[:, 1])
        b = np.maximum(pairs[:, 0], pairs[:, 1])
        if np.any(a == b):
            continue
        e = np.stack([a, b], axis=1)
        if len({(int(x), int(y)) for x, y in e}) != len(e):
            continue
        if not _connected(n, e):
            continue
        order = np.lexsort((e[:, 1], e[:, 0]))
        return np.ascontiguousarray(e[order].astype(np.int32))


def angles(p: int, seed: int = 0):
    """gamma, beta of shape (p,), each uniform in [0, pi)."""
    rng = np.random.Generator(np.random.PCG64(seed + 0x5EED))
    g = rng.uniform(0.0, np.pi, size=p)
    b = rng.uniform(0.0, np.pi, size=p)
    return g, b


def bitstrings(n: int, count: int, seed: int = 0) -> np.ndarray:
    """count x n uint8 array of uniformly random bits."""
    rng = np.random.Generator(np.random.PCG64(seed + 0xB175))
    return rng.integers(0, 2, size=(count, n), dtype=np.uint8)


@dataclasses.dataclass
class Instance:
    n: int
    p: int
    edges: np.ndarray
    gamma: np.ndarray
    beta: np.ndarray
    seed: int


def qaoa_instance(n: int, p: int, seed: int) -> Instance:
    e = random_regular_graph(n, 3, seed)
    g, b = angles(p, seed)
    return Instance(n, p, e, g, b, seed)


# The five synthetic workloads (sizes, depths, cut counts, seeds).
WORKLOADS = {
    "qaoa16_p1_k2": dict(n=16, p=1, k=2, seed=1),
    "qaoa40_p2_k10": dict(n=40, p=2, k=10, seed=2),
    "qaoa80_p1_k16": dict(n=80, p=1, k=16, seed=3, bitstrings=8),
    "uneven64": dict(jobs=64, n_range=(30, 100), p_choices=(1, 2), k_range=(6, 18), seed=4),
    "qaoa120_p1_k22": dict(n=120, p=1, k=22, seed=5),
}


def uneven_jobs(jobs: int = 64, n_range=(30, 100), p_choices=(1, 2), k_range=(6, 18), seed: int = 4,
                p2_n_max: int = 0):
    """Job list for the uneven batch: (n even, p, k, instance seed), n uniform
    in n_range, p from p_choices, k (the job's cut count) uniform in k_range.
    p2_n_max > 0 caps n of the depth-2 jobs (smaller test batches)."""
    rng = np.random.Generator(np.random.PCG64(seed + 0xBA7C))
    out = []
    for j in range(jobs):
        p = int(rng.choice(p_choices))
        hi = n_range[1] if p == 1 or p2_n_max <= 0 else min(n_range[1], p2_n_max)
        n = int(rng.integers(n_range[0] // 2, hi // 2 + 1)) * 2
        k = int(rng.integers(k_range[0], k_range[1] + 1))
        out.append(dict(n=n, p=p, k=k, seed=1000 + seed * 100 + j))
    return out
