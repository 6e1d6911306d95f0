"""Seeded synthetic inputs for adaptive hypergraph learning.

This module is the one piece of code shared by the CPU oracle (``oracle/``) and the
CUDA library's tests and benchmark.  It draws random hypergraphs, tag matrices and
tessellation boundaries; it holds none of the method's arithmetic (no degrees, no
operator, no solver).  Every draw is a function of an integer seed only.

The workloads stand in for the paper's Flickr image-tagging hypergraph (Section 4,
Table 1), which is not available: only the object counts of that dataset are known,
so the hypergraphs here are random, with hyperedge-size distributions chosen per
workload (uniform, truncated power law, or a mixture) and members drawn uniformly
without replacement.

Notation follows the library: n vertices, m hyperedges (the paper's Section 2 uses
m for vertices and n for hyperedges), c right-hand-side (tag) columns.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

__all__ = [
    "Workload",
    "WORKLOADS",
    "powerlaw_mean",
    "powerlaw_exponent_for_mean",
    "draw_sizes",
    "random_hypergraph",
    "binary_tags",
    "blocks_rescaled",
    "blocks_sequential",
    "make_hypergraph",
]


@dataclasses.dataclass(frozen=True)
class Workload:
    """One synthetic workload: hypergraph shape, tag matrix and method parameters."""

    name: str
    n: int                      # vertices
    m: int                      # hyperedges
    sizes: tuple                # ("uniform", lo, hi) | ("powerlaw", a, lo, hi) | ("mixture", ...)
    c: int                      # tag columns (right-hand sides)
    rho: float                  # Bernoulli density of the 0/1 tag matrix Y
    lam: float                  # ranking regulariser (theta in Eq. 3)
    mu: float = 0.0             # weight regulariser (kappa in Eq. 4)
    eta: float = 1e-2           # projected-gradient step size on w
    outer: int = 1              # adaptive outer iterations
    tol: float = 1e-10          # relative residual target of the solve
    blocks: tuple | None = None # ("rescaled", count, lo, hi) | ("sequential", lo, hi)
    k: int = 0                  # rSVD target rank
    p: int = 0                  # rSVD oversampling
    q: int = 0                  # rSVD subspace iterations


# The exponent of the largest workload is chosen so that the mean hyperedge size is
# 10, which gives the stated ~20M incidence nonzeros for m = 2M hyperedges.
WORKLOADS = {
    "small_fp64": Workload(
        "small_fp64", n=2_000, m=3_000, sizes=("uniform", 2, 20), c=10, rho=0.05,
        lam=1.0, mu=0.0, eta=1e-2, outer=5, tol=1e-10),
    "mixed_cg": Workload(
        "mixed_cg", n=50_000, m=80_000, sizes=("powerlaw", 2.5, 2, 500), c=100, rho=0.02,
        lam=0.5, outer=1, tol=1e-8),
    "batched_rsvd": Workload(
        "batched_rsvd", n=120_000, m=200_000, sizes=("powerlaw", 2.5, 2, 500), c=256,
        rho=0.01, lam=0.5, outer=1, tol=1e-8, blocks=("rescaled", 64, 512, 4096),
        k=64, p=10, q=2),
    "adjoint": Workload(
        "adjoint", n=200_000, m=400_000,
        sizes=("mixture", 0.6, ("uniform", 2, 5), ("powerlaw", 2.5, 6, 1000)), c=256,
        rho=0.01, lam=1.0, mu=1e-3, outer=1, tol=1e-10),
    "full_adaptive": Workload(
        "full_adaptive", n=1_000_000, m=2_000_000, sizes=("powerlaw", "mean=10", 2, 2000),
        c=512, rho=0.005, lam=0.5, mu=0.0, eta=2e-13, outer=20, tol=1e-6,
        blocks=("sequential", 1024, 8192), k=64, p=10, q=2),
}


def powerlaw_mean(a: float, lo: int, hi: int) -> float:
    """Mean of the discrete law P(s) proportional to s**-a on lo..hi."""
    s = np.arange(lo, hi + 1, dtype=np.float64)
    pmf = s ** (-a)
    return float((s * pmf).sum() / pmf.sum())


def powerlaw_exponent_for_mean(mean: float, lo: int, hi: int) -> float:
    """Exponent a whose truncated discrete power law on lo..hi has the given mean."""
    a_lo, a_hi = 0.0, 10.0  # the mean falls as a grows
    for _ in range(200):
        mid = 0.5 * (a_lo + a_hi)
        if powerlaw_mean(mid, lo, hi) > mean:
            a_lo = mid
        else:
            a_hi = mid
    return 0.5 * (a_lo + a_hi)


def _powerlaw_draw(rng: np.random.Generator, count: int, a: float, lo: int, hi: int):
    s = np.arange(lo, hi + 1, dtype=np.float64)
    cdf = np.cumsum(s ** (-a))
    cdf /= cdf[-1]
    u = rng.random(count)
    idx = np.searchsorted(cdf, u, side="right")
    return (lo + np.minimum(idx, hi - lo)).astype(np.int64)


def draw_sizes(rng: np.random.Generator, m: int, spec) -> np.ndarray:
    """Hyperedge sizes for m hyperedges from a size specification."""
    kind = spec[0]
    if kind == "uniform":
        _, lo, hi = spec
        return rng.integers(lo, hi + 1, size=m, dtype=np.int64)
    if kind == "powerlaw":
        _, a, lo, hi = spec
        if isinstance(a, str):  # "mean=<x>": solve the exponent for that mean
            a = powerlaw_exponent_for_mean(float(a.split("=")[1]), lo, hi)
        return _powerlaw_draw(rng, m, float(a), lo, hi)
    if kind == "mixture":
        _, frac, first, second = spec
        pick = rng.random(m) < frac
        out = np.empty(m, dtype=np.int64)
        out[pick] = draw_sizes(rng, int(pick.sum()), first)
        out[~pick] = draw_sizes(rng, int((~pick).sum()), second)
        return out
    raise ValueError(f"unknown size spec {spec!r}")


def random_hypergraph(n: int, sizes: np.ndarray, rng: np.random.Generator):
    """Members of each hyperedge drawn uniformly without replacement from 0..n-1.

    Returns ``(edge_ptr int64[m+1], members int32[nnz])``.  Members are left in a
    random order inside each hyperedge, so consumers must sort them themselves.
    Sampling: draw with replacement, then redraw every repeated member of a
    hyperedge until none remain.  The procedure commutes with relabelling the
    vertices, so every subset of a given size is equally likely.
    """
    sizes = np.asarray(sizes, dtype=np.int64)
    if (sizes > n).any():
        raise ValueError("a hyperedge cannot have more members than there are vertices")
    m = sizes.size
    edge_ptr = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(sizes, out=edge_ptr[1:])
    nnz = int(edge_ptr[-1])
    edge_of = np.repeat(np.arange(m, dtype=np.int64), sizes)
    members = rng.integers(0, n, size=nnz, dtype=np.int64)
    while True:
        order = np.lexsort((members, edge_of))
        e_sorted = edge_of[order]
        v_sorted = members[order]
        dup = np.zeros(nnz, dtype=bool)
        dup[1:] = (e_sorted[1:] == e_sorted[:-1]) & (v_sorted[1:] == v_sorted[:-1])
        if not dup.any():
            break
        pos = order[dup]
        members[pos] = rng.integers(0, n, size=pos.size, dtype=np.int64)
    # shuffle inside each hyperedge (the edge order itself is kept)
    key = rng.random(nnz)
    order = np.lexsort((key, edge_of))
    members = members[order]
    return edge_ptr, members.astype(np.int32)


def binary_tags(n: int, c: int, rho: float, rng: np.random.Generator,
                dtype=np.float64, chunk_rows: int = 65_536) -> np.ndarray:
    """n x c matrix of independent Bernoulli(rho) 0/1 entries (row-major)."""
    out = np.empty((n, c), dtype=dtype)
    for r0 in range(0, n, chunk_rows):
        r1 = min(n, r0 + chunk_rows)
        out[r0:r1] = (rng.random((r1 - r0, c), dtype=np.float32) < rho)
    return out


def blocks_rescaled(n: int, count: int, lo: int, hi: int, rng: np.random.Generator):
    """Block boundaries: ``count`` sizes drawn from U{lo..hi}, rescaled to sum to n.

    Sizes are scaled by n / sum, floored and clamped to [lo, hi]; the remainder is
    spread one by one round-robin over blocks that still have room.
    Returns ``block_ptr int64[count+1]``.
    """
    raw = rng.integers(lo, hi + 1, size=count).astype(np.float64)
    sz = np.clip(np.floor(raw * (n / raw.sum())), lo, hi).astype(np.int64)
    rem = n - int(sz.sum())
    i = 0
    guard = 0
    while rem != 0:
        step = 1 if rem > 0 else -1
        cand = sz[i] + step
        if lo <= cand <= hi:
            sz[i] = cand
            rem -= step
            guard = 0
        else:
            guard += 1
            if guard > count:
                raise ValueError("cannot fit n into the requested block size range")
        i = (i + 1) % count
    ptr = np.zeros(count + 1, dtype=np.int64)
    np.cumsum(sz, out=ptr[1:])
    return ptr


def blocks_sequential(n: int, lo: int, hi: int, rng: np.random.Generator):
    """Block boundaries: sizes from U{lo..hi} drawn until they cover n vertices.

    The last block is cut at n; a final piece shorter than lo is merged into the
    block before it.  Returns ``block_ptr int64[count+1]``.
    """
    sizes = []
    total = 0
    while total < n:
        s = int(rng.integers(lo, hi + 1))
        s = min(s, n - total)
        sizes.append(s)
        total += s
    if len(sizes) > 1 and sizes[-1] < lo:
        last = sizes.pop()
        sizes[-1] += last
    ptr = np.zeros(len(sizes) + 1, dtype=np.int64)
    np.cumsum(np.asarray(sizes, dtype=np.int64), out=ptr[1:])
    return ptr


def make_hypergraph(wl: Workload, seed: int = 0, n: int | None = None,
                    m: int | None = None, c: int | None = None,
                    tags_dtype=np.float64):
    """Draw the hypergraph, the tag matrix and (if any) the blocks of a workload.

    ``n``, ``m`` and ``c`` override the workload's sizes (same distributions), which
    is how the tests get small cases of every workload's shape.
    Returns a dict with edge_ptr, members, Y, w0 (uniform 1/m), block_ptr.
    """
    n = wl.n if n is None else n
    m = wl.m if m is None else m
    c = wl.c if c is None else c
    rng = np.random.default_rng(np.random.SeedSequence([seed, n, m, c]))
    spec = wl.sizes
    if spec[0] == "powerlaw" or spec[0] == "uniform":
        hi = spec[-1]
        if hi > n:
            spec = spec[:-1] + (n,)
    sizes = draw_sizes(rng, m, spec)
    sizes = np.minimum(sizes, n)
    edge_ptr, members = random_hypergraph(n, sizes, rng)
    Y = binary_tags(n, c, wl.rho, rng, dtype=tags_dtype)
    w0 = np.full(m, 1.0 / m)
    block_ptr = None
    if wl.blocks is not None:
        # smaller cases keep the workload's block-size law, scaled by n / wl.n
        scale = n / wl.n
        if wl.blocks[0] == "rescaled":
            _, count, lo, hi = wl.blocks
            count = min(count, n)
            lo_s = max(1, int(round(lo * scale)))
            hi_s = max(lo_s, int(round(hi * scale)))
            lo_s = min(lo_s, n // count)
            hi_s = max(hi_s, -(-n // count))
            block_ptr = blocks_rescaled(n, count, lo_s, hi_s, rng)
        else:
            _, lo, hi = wl.blocks
            lo_s = max(1, min(n, int(round(lo * scale))))
            hi_s = max(lo_s, min(n, int(round(hi * scale))))
            block_ptr = blocks_sequential(n, lo_s, hi_s, rng)
    return {"n": n, "m": m, "c": c, "edge_ptr": edge_ptr, "members": members, "Y": Y,
            "w0": w0, "block_ptr": block_ptr, "lam": wl.lam, "mu": wl.mu, "eta": wl.eta}


def describe_sizes(wl: Workload) -> str:
    """Human-readable size law of a workload (with the solved exponent, if any)."""
    spec = wl.sizes
    if spec[0] == "powerlaw" and isinstance(spec[1], str):
        a = powerlaw_exponent_for_mean(float(spec[1].split("=")[1]), spec[2], spec[3])
        return f"powerlaw(a={a:.4f}, {spec[2]}..{spec[3]})"
    return repr(spec)


def _selfcheck():  # pragma: no cover - manual use
    wl = WORKLOADS["small_fp64"]
    d = make_hypergraph(wl, 0)
    print(d["edge_ptr"][-1], d["Y"].sum(), math.fsum(d["w0"]))
