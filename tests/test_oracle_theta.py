"""Pins of the oracle's operator Theta (Eq. 1) and Laplacian Delta = I - Theta."""
import itertools

import networkx as nx
import numpy as np
import pytest

from oracle.core import degrees, system_dense, theta_apply, theta_dense
from oracle.incidence import build_incidence, incidence_matrix
from tests._util import read_golden, tiny_hypergraph


def _H(n, m, ptr, mem):
    return incidence_matrix(build_incidence(n, m, ptr, mem))


def brute_theta(n, m, ptr, mem, w):
    """Theta_uv = sum_e H(u,e) H(v,e) w_e / (de_e sqrt(dv_u dv_v)) by explicit loops."""
    members = [set(int(x) for x in mem[ptr[e]:ptr[e + 1]]) for e in range(m)]
    dv = [sum(w[e] for e in range(m) if v in members[e]) for v in range(n)]
    T = np.zeros((n, n))
    for u in range(n):
        for v in range(n):
            acc = 0.0
            for e in range(m):
                if u in members[e] and v in members[e]:
                    acc += w[e] / len(members[e])
            if dv[u] > 0 and dv[v] > 0:
                T[u, v] = acc / np.sqrt(dv[u] * dv[v])
    return T


@pytest.mark.parametrize("seed", range(6))
def test_brute_force(seed):
    rng = np.random.default_rng(100 + seed)
    n, m = int(rng.integers(3, 12)), int(rng.integers(1, 9))
    ptr, mem = tiny_hypergraph(rng, n, m)
    w = rng.random(m) + 0.05
    H = _H(n, m, ptr, mem)
    B = brute_theta(n, m, ptr, mem, w)
    assert np.allclose(theta_dense(H, w), B, rtol=1e-13, atol=1e-15)
    X = rng.standard_normal((n, 3))
    assert np.allclose(theta_apply(H, w, X), B @ X, rtol=1e-12, atol=1e-14)
    a, b = 1.7, -0.3
    assert np.allclose(theta_apply(H, w, X, a, b), a * X + b * (B @ X), rtol=1e-12, atol=1e-14)


def test_golden_three_vertex_path():
    rows = read_golden("path3_theta.txt")
    n, m = int(rows[0][0]), int(rows[0][1])
    ptr = np.array([int(x) for x in rows[1]])
    mem = np.array([int(x) for x in rows[2]])
    w = np.array([float(x) for x in rows[3]])
    expect = np.array([[float(x) for x in r] for r in rows[4:4 + n]])
    eig = np.array([float(x) for x in rows[4 + n]])
    Th = theta_dense(_H(n, m, ptr, mem), w)
    assert np.allclose(Th, expect, rtol=0, atol=1e-15)
    assert np.allclose(np.linalg.eigvalsh(Th), eig, atol=1e-14)


@pytest.mark.parametrize("seed", range(4))
def test_invariants(seed):
    rng = np.random.default_rng(200 + seed)
    n, m = 40, 60
    ptr, mem = tiny_hypergraph(rng, n, m, 2, 8)
    w = rng.random(m)
    w /= w.sum()
    H = _H(n, m, ptr, mem)
    dv, _, s, _ = degrees(H, w)
    Th = theta_dense(H, w)
    assert np.allclose(Th, Th.T, atol=1e-15)
    ev = np.linalg.eigvalsh(Th)
    assert ev.min() > -1e-12 and ev.max() < 1 + 1e-12
    # Delta Dv^1/2 1 = 0 on the support
    sq = np.sqrt(dv)
    assert np.allclose(Th @ sq, sq, atol=1e-13)
    lam = 0.5
    evM = np.linalg.eigvalsh(system_dense(H, w, lam))
    assert evM.min() > lam - 1e-12 and evM.max() < 1 + lam + 1e-12


def test_zero_weight_isolates_vertex():
    # vertex 3 only in hyperedge 1, whose weight is zero -> dv_3 = 0, s_3 = 0
    ptr = [0, 3, 5]
    mem = [0, 1, 2, 3, 2]
    H = _H(4, 2, ptr, mem)
    w = np.array([1.0, 0.0])
    Th = theta_dense(H, w)
    assert np.all(Th[3] == 0) and np.all(Th[:, 3] == 0)
    dv, *_ = degrees(H, w)
    assert dv[3] == 0
    assert np.allclose(Th @ np.sqrt(dv), np.sqrt(dv), atol=1e-15)


def test_two_uniform_is_half_normalised_graph_laplacian():
    # every hyperedge of size 2: Delta = (1/2) (I - D^-1/2 A_w D^-1/2), the normalised
    # Laplacian of the weighted graph (networkx), since Theta_uu = 1/2.
    rng = np.random.default_rng(7)
    n = 15
    pairs = [p for p in itertools.combinations(range(n), 2) if rng.random() < 0.35]
    m = len(pairs)
    ptr = np.arange(0, 2 * m + 1, 2)
    mem = np.array([x for p in pairs for x in p])
    w = rng.random(m) + 0.1
    G = nx.Graph()
    G.add_nodes_from(range(n))
    for (u, v), we in zip(pairs, w):
        G.add_edge(u, v, weight=we)
    L = nx.normalized_laplacian_matrix(G, nodelist=range(n), weight="weight").toarray()
    H = _H(n, m, ptr, mem)
    Delta = np.eye(n) - theta_dense(H, w)
    connected = np.array([G.degree(v) > 0 for v in range(n)])
    idx = np.where(connected)[0]
    assert np.allclose(Delta[np.ix_(idx, idx)], 0.5 * L[np.ix_(idx, idx)], atol=1e-14)


def test_single_edge_rank_one():
    n = 7
    H = _H(n, 1, [0, n], list(range(n)))
    Th = theta_dense(H, np.array([0.3]))
    assert np.allclose(Th, np.ones((n, n)) / n, atol=1e-15)


def test_regular_uniform_closed_form():
    # all 3-subsets of 6 vertices: k = 3, each vertex in d = 10 hyperedges; uniform w
    n, k = 6, 3
    edges = list(itertools.combinations(range(n), k))
    m = len(edges)
    ptr = np.arange(0, k * m + 1, k)
    mem = np.array([x for e in edges for x in e])
    H = _H(n, m, ptr, mem)
    Hd = H.toarray()
    d = 10
    Th = theta_dense(H, np.full(m, 1.0 / m))
    assert np.allclose(Th, Hd @ Hd.T / (k * d), atol=1e-15)


def test_paper_form_equivalence():
    # X = I - Theta/(1+theta) (Section 2); M = (1+lam) I - Theta = (1+lam) X
    rng = np.random.default_rng(3)
    ptr, mem = tiny_hypergraph(rng, 10, 8)
    H = _H(10, 8, ptr, mem)
    w = rng.random(8) + 0.1
    lam = 0.7
    X = np.eye(10) - theta_dense(H, w) / (1 + lam)
    assert np.allclose(system_dense(H, w, lam), (1 + lam) * X, atol=1e-15)


def test_theta_rows_matches_the_sparse_operator():
    """Row-by-row evaluation of Eq. 1 (for checking sampled outputs of large graphs)
    against the factor-by-factor sparse operator, including a zero-degree vertex."""
    import numpy as np
    from oracle.core import incidence_lists, theta_apply, theta_rows
    from oracle.incidence import build_incidence, incidence_matrix
    from tests._util import tiny_hypergraph
    rng = np.random.default_rng(5)
    n, m = 40, 30
    ptr, mem = tiny_hypergraph(rng, n, m, 2, 7)
    H = incidence_matrix(build_incidence(n, m, ptr, mem))
    w = rng.random(m) + 0.1
    w[np.asarray(H[3].nonzero()[1])] = 0.0  # vertex 3 loses all weight
    X = rng.standard_normal((n, 5))
    lists = incidence_lists(n, m, ptr, mem)
    rows = np.array([0, 3, 7, 39])
    Z = theta_rows(lists, w, lambda u: X[np.asarray(u)], rows, 1.5, -1.0)
    ref = theta_apply(H, w, X, 1.5, -1.0)[rows]
    assert np.allclose(Z, ref, rtol=1e-13, atol=1e-14)


@pytest.mark.parametrize("seed", range(4))
def test_split_by_hyperedge_size_is_eq1(seed):
    """The GPU operator splits Eq. 1 by hyperedge size: hyperedges of more than three
    members go through the intermediate t_e H^T s X, the others become vertex-to-vertex
    terms -- per member u of such a hyperedge, t_e s_v X[v] for its other members v plus
    the diagonal s_u^2 t_e X[u].  Written out here with explicit loops, the two parts add
    up to the oracle's Theta X (any split threshold, sizes one to six, a vertex in no
    hyperedge)."""
    rng = np.random.default_rng(300 + seed)
    n, m, c = 40, 60, 3
    sizes = rng.integers(1, 7, m)
    mem = np.concatenate([rng.choice(n - 1, int(k), replace=False) for k in sizes]).astype(np.int32)
    ptr = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(sizes, out=ptr[1:])
    w = rng.random(m) + 0.05
    X = rng.standard_normal((n, c))
    H = _H(n, m, ptr, mem)
    _, _, s, t = degrees(H, w)
    for small in (0, 3, 6):
        Z = np.zeros((n, c))
        for e in range(m):
            vs = [int(v) for v in mem[ptr[e]:ptr[e + 1]]]
            if len(vs) > small:   # through the intermediate
                T = t[e] * sum(s[v] * X[v] for v in vs)
                for u in vs:
                    Z[u] += s[u] * T
            else:                 # vertex-to-vertex terms and the diagonal
                for u in vs:
                    Z[u] += s[u] * s[u] * t[e] * X[u]
                    for v in vs:
                        if v != u:
                            Z[u] += s[u] * t[e] * s[v] * X[v]
        assert np.allclose(Z, theta_apply(H, w, X), rtol=1e-13, atol=1e-15)
        assert np.all(Z[n - 1] == 0.0)
