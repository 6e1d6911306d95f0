"""Pins of the oracle's incidence construction (Section 2: H(v, e) = 1 iff v in e)."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle.incidence import IncidenceError, build_incidence, incidence_matrix
from tests._util import dense_incidence, tiny_hypergraph
import synth


@pytest.mark.parametrize("seed", range(5))
def test_matches_dense_brute_force(seed):
    rng = np.random.default_rng(seed)
    n, m = 9, 7
    ptr, mem = tiny_hypergraph(rng, n, m)
    g = build_incidence(n, m, ptr, mem)
    assert np.array_equal(incidence_matrix(g).toarray(), dense_incidence(n, m, ptr, mem))
    # each CSC segment ascending, each CSR segment ascending
    for e in range(m):
        seg = g["csc_idx"][g["csc_ptr"][e]:g["csc_ptr"][e + 1]]
        assert np.all(np.diff(seg) > 0)
    for v in range(n):
        seg = g["csr_idx"][g["csr_ptr"][v]:g["csr_ptr"][v + 1]]
        assert np.all(np.diff(seg) > 0)
    assert np.array_equal(g["de"], np.diff(ptr))


def test_matches_scipy_transpose():
    wl = synth.WORKLOADS["small_fp64"]
    d = synth.make_hypergraph(wl, 3)
    n, m = d["n"], d["m"]
    g = build_incidence(n, m, d["edge_ptr"], d["members"])
    A = sp.csc_matrix((np.ones(d["members"].size), d["members"].astype(np.int64), d["edge_ptr"]),
                      shape=(n, m))
    A.sort_indices()
    R = A.tocsr()
    R.sort_indices()
    assert np.array_equal(A.indptr, g["csc_ptr"])
    assert np.array_equal(A.indices, g["csc_idx"])
    assert np.array_equal(R.indptr, g["csr_ptr"])
    assert np.array_equal(R.indices, g["csr_idx"])


def test_isolated_vertex_allowed():
    g = build_incidence(4, 1, [0, 2], [2, 0])
    assert list(g["csr_ptr"]) == [0, 1, 1, 2, 2]
    assert list(g["csc_idx"]) == [0, 2]


@pytest.mark.parametrize("ptr,mem,code", [
    ([0, 2, 2], [0, 1], "EMPTY_EDGE"),
    ([0, 2], [0, 5], "INDEX_RANGE"),
    ([0, 2], [-1, 0], "INDEX_RANGE"),
    ([0, 3], [1, 2, 1], "DUPLICATE_MEMBER"),
    ([1, 2], [0, 1], "INVALID_ARG"),
    ([0, 3], [0, 1], "INVALID_ARG"),
])
def test_errors(ptr, mem, code):
    m = len(ptr) - 1
    with pytest.raises(IncidenceError) as ei:
        build_incidence(3, m, ptr, mem)
    assert ei.value.code == code


def test_generator_draws_valid_hypergraphs():
    for name, wl in synth.WORKLOADS.items():
        d = synth.make_hypergraph(wl, 1, n=3000, m=4000, c=4)
        g = build_incidence(d["n"], d["m"], d["edge_ptr"], d["members"])  # raises if invalid
        assert g["nnz"] == d["members"].size
        if d["block_ptr"] is not None:
            bp = d["block_ptr"]
            assert bp[0] == 0 and bp[-1] == d["n"] and np.all(np.diff(bp) > 0)


def test_paper_vertex_counts_sum_to_query_length():
    # Table 1 object counts concatenate into the query vector of length 5867 (Section 4).
    assert 1292 + 440 + 1644 + 125 + 2366 == 5867
