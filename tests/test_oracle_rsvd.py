"""Pins of the oracle's block randomized SVD (Algorithm 1), the block inverse (Eq. 15
completed by the identity part) and the Philox/Box-Muller test matrix."""
import numpy as np
import pytest

import synth
from oracle import philox
from oracle.core import cg_iteration_bound, cg_solve, solve_dense, theta_dense
from oracle.incidence import build_incidence, incidence_matrix
from oracle.rsvd import (block_eig, block_rsvd, block_theta, precond_apply, range_finder,
                         rsvd_alg1, rsvd_ritz)
from tests._util import read_golden


def test_philox_known_answers():
    for row in read_golden("philox4x32_10_kat.txt"):
        v = [int(x, 16) for x in row]
        out = philox.philox4x32_10(*[np.uint64(x) for x in v[:4]], v[4], v[5])
        assert [int(o) for o in out] == v[6:]


def test_omega_statistics_and_tessellation_independence():
    Om = philox.omega(np.arange(20000), 8, seed=12345)
    assert abs(Om.mean()) < 0.01 and abs(Om.var() - 1) < 0.01
    # fourth moment of N(0,1) is 3
    assert abs((Om ** 4).mean() - 3) < 0.1
    part = philox.omega(np.arange(700, 900), 8, seed=12345)
    assert np.array_equal(part, Om[700:900])
    # columns are not copies of one another
    assert abs(np.corrcoef(Om[:, 0], Om[:, 1])[0, 1]) < 0.03


def _psd_rank(rng, b, r):
    B = rng.standard_normal((b, r))
    return B @ B.T / b


@pytest.mark.parametrize("seed", range(3))
def test_exact_low_rank_recovered(seed):
    rng = np.random.default_rng(seed)
    b, r, k, p = 120, 10, 12, 6
    X = _psd_rank(rng, b, r)
    Om = rng.standard_normal((b, k + p))
    Vx, lx = block_eig(X, k)
    Q, lr = rsvd_ritz(X, Om, 2, k)
    U, sig, V = rsvd_alg1(X, Om, 2, k)
    assert np.allclose(lr[:r], lx[:r], rtol=1e-10, atol=1e-12)
    assert np.allclose(sig[:r], lx[:r], rtol=1e-10, atol=1e-12)
    Px = Vx[:, :r] @ Vx[:, :r].T
    assert np.allclose(Q[:, :r] @ Q[:, :r].T, Px, atol=1e-10)
    assert np.allclose(U[:, :r] @ U[:, :r].T, Px, atol=1e-10)
    # symmetric input: U = V up to sign on the captured part
    assert np.allclose(np.abs(np.sum(U[:, :r] * V[:, :r], axis=0)), 1.0, atol=1e-10)


def test_halko_bound_on_hypergraph_block():
    rng = np.random.default_rng(4)
    d = synth.make_hypergraph(synth.WORKLOADS["batched_rsvd"], 0, n=3000, m=5000, c=2)
    H = incidence_matrix(build_incidence(d["n"], d["m"], d["edge_ptr"], d["members"]))
    w = np.full(d["m"], 1.0 / d["m"])
    Tb = block_theta(H, w, [0, 400])[0]
    k, p, q = 16, 10, 2
    Q, lr = rsvd_ritz(Tb, rng.standard_normal((400, k + p)), q, k)
    _, lx = block_eig(Tb, k + 1)
    S = range_finder(Tb, rng.standard_normal((400, k + p)), q)
    assert np.allclose(S.T @ S, np.eye(k + p), atol=1e-12)
    err = np.linalg.norm(Tb - Q @ np.diag(lr) @ Q.T, 2)
    # Halko-Martinsson-Tropp (2011), power scheme: expected error within
    # (1 + sqrt(k/(p-1)) + e sqrt(k+p)/p sqrt(b-k))^(1/(2q+1)) sigma_{k+1}; allow 4x for a single draw
    fac = (1 + np.sqrt(k / (p - 1)) + np.e * np.sqrt(k + p) / p * np.sqrt(400 - k)) ** (1 / (2 * q + 1))
    assert err <= 4 * fac * lx[k] + 1e-12
    # Ritz values never exceed the true eigenvalues (Cauchy interlacing)
    assert np.all(lr <= lx[:k] + 1e-12)


def test_block_theta_is_restriction():
    rng = np.random.default_rng(2)
    d = synth.make_hypergraph(synth.WORKLOADS["batched_rsvd"], 1, n=500, m=800, c=2)
    H = incidence_matrix(build_incidence(d["n"], d["m"], d["edge_ptr"], d["members"]))
    w = rng.random(d["m"])
    bp = d["block_ptr"]
    full = theta_dense(H, w)
    for b, Tb in enumerate(block_theta(H, w, bp)):
        assert np.allclose(Tb, full[bp[b]:bp[b + 1], bp[b]:bp[b + 1]], atol=1e-15)


def test_full_rank_woodbury_is_exact_block_inverse():
    rng = np.random.default_rng(8)
    d = synth.make_hypergraph(synth.WORKLOADS["batched_rsvd"], 2, n=300, m=500, c=3)
    H = incidence_matrix(build_incidence(d["n"], d["m"], d["edge_ptr"], d["members"]))
    w = rng.random(d["m"])
    lam = 0.5
    bp = np.array([0, 100, 180, 300])
    blocks = block_theta(H, w, bp)
    factors = [block_eig(Tb, Tb.shape[0]) for Tb in blocks]
    R = rng.standard_normal((300, 3))
    Z = precond_apply([(V, ev) for V, ev in factors], bp, lam, R)
    for b, Tb in enumerate(blocks):
        Mb = (1 + lam) * np.eye(Tb.shape[0]) - Tb
        assert np.allclose(Z[bp[b]:bp[b + 1]], np.linalg.solve(Mb, R[bp[b]:bp[b + 1]]), atol=1e-12)


def test_preconditioned_cg_reaches_the_same_solution():
    d = synth.make_hypergraph(synth.WORKLOADS["batched_rsvd"], 3, n=1500, m=2500, c=4)
    H = incidence_matrix(build_incidence(d["n"], d["m"], d["edge_ptr"], d["members"]))
    w = np.full(d["m"], 1.0 / d["m"])
    lam = 0.5
    bp = d["block_ptr"]
    fac = block_rsvd(H, w, bp, k=8, p=4, q=2, seed=99)
    Y = d["Y"]
    Y[0] = 1.0
    out = cg_solve(H, w, lam, Y, tol=1e-12, precond=lambda R: precond_apply(fac, bp, lam, R))
    Fd = solve_dense(H, w, lam, Y)
    assert np.allclose(out["F"], Fd, atol=1e-10)
    # the preconditioner keeps kappa(P^-1 M) <= (1+lam)/lam, so the same bound holds
    assert out["iters"].max() <= cg_iteration_bound(lam, 1e-12) + 2
