"""Oracle: the incidence matrix H and its two compressed layouts (Section 2).

H(v, e) = 1 if vertex v belongs to hyperedge e and 0 otherwise (Section 2).  The
hyperedge-major layout (CSC of H: hyperedge -> sorted members) and the vertex-major
layout (CSR of H: vertex -> sorted hyperedges) are plain sorts of the (v, e) pairs.
The hyperedge degree de(e) = sum_v H(v, e) is the member count (Section 2).

Errors follow the library's status names: a vertex id outside [0, n) is INDEX_RANGE,
a vertex listed twice in one hyperedge is DUPLICATE_MEMBER (H is 0/1), an empty
hyperedge is EMPTY_EDGE (De^-1 is undefined), a malformed pointer array is
INVALID_ARG.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


class IncidenceError(ValueError):
    """Raised with ``.code`` in {INVALID_ARG, INDEX_RANGE, DUPLICATE_MEMBER, EMPTY_EDGE}."""

    def __init__(self, code: str, msg: str):
        super().__init__(f"{code}: {msg}")
        self.code = code


def build_incidence(n: int, m: int, edge_ptr, members):
    """CSC and CSR of H from hyperedge member lists, plus de.

    Returns a dict with csc_ptr int64[m+1], csc_idx int32[nnz] (members of each
    hyperedge in ascending order), csr_ptr int64[n+1], csr_idx int32[nnz] (hyperedges
    of each vertex in ascending order) and de int32[m].
    """
    edge_ptr = np.asarray(edge_ptr, dtype=np.int64)
    members = np.asarray(members)
    if n < 0 or m < 0 or edge_ptr.shape != (m + 1,):
        raise IncidenceError("INVALID_ARG", "edge_ptr must have m+1 entries")
    if edge_ptr[0] != 0 or np.any(np.diff(edge_ptr) < 0) or edge_ptr[-1] != members.size:
        raise IncidenceError("INVALID_ARG", "edge_ptr must start at 0, not decrease, end at nnz")
    sizes = np.diff(edge_ptr)
    if m > 0 and np.any(sizes == 0):
        raise IncidenceError("EMPTY_EDGE", f"hyperedge {int(np.argmax(sizes == 0))} is empty")
    members = members.astype(np.int64)
    if members.size and (members.min() < 0 or members.max() >= n):
        raise IncidenceError("INDEX_RANGE", "a member id lies outside [0, n)")
    edge_of = np.repeat(np.arange(m, dtype=np.int64), sizes)

    # hyperedge-major: sort pairs by (edge, vertex)
    order = np.lexsort((members, edge_of))
    csc_idx = members[order]
    e_sorted = edge_of[order]
    if csc_idx.size > 1:
        same = (e_sorted[1:] == e_sorted[:-1]) & (csc_idx[1:] == csc_idx[:-1])
        if same.any():
            raise IncidenceError("DUPLICATE_MEMBER", "a vertex appears twice in one hyperedge")

    # vertex-major: sort pairs by (vertex, edge); pointers from the vertex counts
    order_v = np.lexsort((edge_of, members))
    csr_idx = edge_of[order_v]
    counts = np.bincount(members, minlength=n) if members.size else np.zeros(n, np.int64)
    csr_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=csr_ptr[1:])

    return {
        "n": n, "m": m, "nnz": int(members.size),
        "csc_ptr": edge_ptr.copy(), "csc_idx": csc_idx.astype(np.int32),
        "csr_ptr": csr_ptr, "csr_idx": csr_idx.astype(np.int32),
        "de": sizes.astype(np.int32),
    }


def incidence_matrix(g) -> sp.csr_matrix:
    """H as an n x m scipy sparse matrix (float64 ones)."""
    n, m = g["n"], g["m"]
    data = np.ones(g["nnz"], dtype=np.float64)
    return sp.csc_matrix((data, g["csc_idx"].astype(np.int64), g["csc_ptr"]), shape=(n, m)).tocsr()
