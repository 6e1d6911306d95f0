"""Shared helpers for the tests (no method arithmetic here)."""
from __future__ import annotations

import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def read_golden(name: str):
    """Non-comment lines of a golden fixture, split into tokens."""
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            rows.append(line.split())
    return rows


def tiny_hypergraph(rng: np.random.Generator, n: int, m: int, lo: int = 1, hi: int = None):
    """Random small hypergraph as (edge_ptr, members) with unsorted members."""
    hi = n if hi is None else min(hi, n)
    sizes = rng.integers(lo, hi + 1, size=m)
    ptr = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(sizes, out=ptr[1:])
    mem = np.concatenate([rng.permutation(n)[:s] for s in sizes]).astype(np.int32) if m else np.zeros(0, np.int32)
    return ptr, mem


def dense_incidence(n: int, m: int, edge_ptr, members) -> np.ndarray:
    """H by explicit loops over the member lists."""
    H = np.zeros((n, m))
    for e in range(m):
        for i in range(int(edge_ptr[e]), int(edge_ptr[e + 1])):
            H[int(members[i]), e] = 1.0
    return H
