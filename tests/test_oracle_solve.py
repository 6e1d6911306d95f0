"""Pins of the oracle's ranking solve (Eqs. 3 and 6) and its CG (Eqs. 16-20)."""
import numpy as np
import pytest

import synth
from oracle.core import (block_cg_solve, certified_solve, cg_iteration_bound, cg_solve, solve_dense,
                         system_dense, theta_apply, theta_dense)
from oracle.incidence import build_incidence, incidence_matrix


@pytest.fixture(scope="module")
def small():
    wl = synth.WORKLOADS["small_fp64"]
    d = synth.make_hypergraph(wl, 11)
    H = incidence_matrix(build_incidence(d["n"], d["m"], d["edge_ptr"], d["members"]))
    rng = np.random.default_rng(5)
    w = rng.random(d["m"]) + 0.2
    w /= w.sum()
    return H, w, d["Y"], d["lam"]


def test_dense_solve_satisfies_the_paper_form(small):
    H, w, Y, lam = small
    F = solve_dense(H, w, lam, Y)
    # f* = theta/(1+theta) X^-1 y with X = I - Theta/(1+theta)  (Eq. 3), via X f = rhs
    X = np.eye(H.shape[0]) - theta_dense(H, w) / (1 + lam)
    resid = X @ F - lam / (1 + lam) * Y
    assert np.abs(resid).max() < 1e-13


def test_cg_matches_dense(small):
    H, w, Y, lam = small
    Fd = solve_dense(H, w, lam, Y)
    out = cg_solve(H, w, lam, Y, tol=1e-12)
    err = np.linalg.norm(out["F"] - Fd, axis=0) / np.linalg.norm(Fd, axis=0)
    assert err.max() < 1e-11
    assert out["true_relres"].max() < 1e-11
    # iteration count within the Chebyshev bound for kappa <= (1+lam)/lam (+2 for rounding)
    assert out["iters"].max() <= cg_iteration_bound(lam, 1e-12) + 2


def test_certificate(small):
    H, w, Y, lam = small
    Fd = solve_dense(H, w, lam, Y[:, :3])
    F, bound = certified_solve(H, w, lam, Y[:, :3], tol=1e-6)
    err = np.linalg.norm(F - Fd, axis=0)
    assert np.all(err <= bound * (1 + 1e-6) + 1e-15)


def test_cg_identities():
    rng = np.random.default_rng(9)
    d = synth.make_hypergraph(synth.WORKLOADS["small_fp64"], 2, n=300, m=450, c=2)
    H = incidence_matrix(build_incidence(d["n"], d["m"], d["edge_ptr"], d["members"]))
    w = rng.random(d["m"]) + 0.1
    lam = 0.5
    Y = d["Y"].copy()
    Y[0, :] = 1.0
    out = cg_solve(H, w, lam, Y, tol=1e-10, record=True)
    M = system_dense(H, w, lam)
    Fs = solve_dense(H, w, lam, Y)
    R = out["history"]["R"]
    P = out["history"]["P"]
    Fh = out["history"]["F"]
    for j in range(Y.shape[1]):
        k = int(out["iters"][j])
        rs = [R[i][:, j] for i in range(min(k, 6))]
        ps = [P[i][:, j] for i in range(min(k, 6))]
        for a in range(len(rs)):
            for b in range(a):
                assert abs(rs[a] @ rs[b]) <= 1e-10 * np.linalg.norm(rs[a]) * np.linalg.norm(rs[b])
                assert abs(ps[a] @ M @ ps[b]) <= 1e-10 * np.sqrt((ps[a] @ M @ ps[a]) * (ps[b] @ M @ ps[b]))
        # M-norm of the error never increases
        errs = [np.sqrt((Fh[i][:, j] - Fs[:, j]) @ M @ (Fh[i][:, j] - Fs[:, j])) for i in range(k + 1)]
        assert all(errs[i + 1] <= errs[i] * (1 + 1e-12) for i in range(k))
    # the recursive residual agrees with the recomputed one
    assert np.allclose(out["relres"], out["true_relres"], rtol=0, atol=1e-12)


def test_zero_column_and_warm_start():
    d = synth.make_hypergraph(synth.WORKLOADS["small_fp64"], 4, n=200, m=300, c=3)
    H = incidence_matrix(build_incidence(d["n"], d["m"], d["edge_ptr"], d["members"]))
    w = np.full(d["m"], 1.0 / d["m"])
    Y = d["Y"].copy()
    Y[:, 1] = 0.0
    out = cg_solve(H, w, 1.0, Y, tol=1e-10)
    assert out["iters"][1] == 0 and np.all(out["F"][:, 1] == 0)
    again = cg_solve(H, w, 1.0, Y, F0=solve_dense(H, w, 1.0, Y), tol=1e-10)
    assert again["iters"].max() == 0


def test_isolated_vertex_solution():
    # a vertex with dv = 0 decouples: (1+lam) f_v = lam y_v
    ptr = np.array([0, 3, 5])
    mem = np.array([0, 1, 2, 3, 2])
    H = incidence_matrix(build_incidence(4, 2, ptr, mem))
    w = np.array([1.0, 0.0])
    Y = np.array([[1.0], [0.0], [0.0], [1.0]])
    F = solve_dense(H, w, 2.0, Y)
    assert abs(F[3, 0] - 2.0 / 3.0) < 1e-15
    assert np.allclose(theta_apply(H, w, F, 3.0, -1.0), 2.0 * Y, atol=1e-14)


def test_iteration_bound_values():
    # kappa = 2 at lam = 1 and 3 at lam = 0.5
    assert cg_iteration_bound(1.0, 1e-10) == 14
    assert cg_iteration_bound(0.5, 1e-8) == 15


# ---------------------------------------------------------------- block CG ---

def _spd_case(n=24, m=40, c=6, seed=3):
    """A small hypergraph whose M has well-spread eigenvalues (random sizes 2..6)."""
    rng = np.random.default_rng(seed)
    ptr, mem = [0], []
    for _ in range(m):
        k = int(rng.integers(2, 7))
        mem.extend(sorted(rng.choice(n, k, replace=False)))
        ptr.append(len(mem))
    H = incidence_matrix(build_incidence(n, m, np.asarray(ptr, np.int64), np.asarray(mem, np.int32)))
    w = rng.random(m) + 0.1
    w /= w.sum()
    Y = rng.standard_normal((n, c))
    return H, w, Y


def test_block_cg_matches_dense(small):
    """Block CG in groups of 4 (a ragged last group of 2) reaches the dense solution."""
    H, w, Y, lam = small
    Fd = solve_dense(H, w, lam, Y)
    out = block_cg_solve(H, w, lam, Y, s=4, tol=1e-12)
    err = np.linalg.norm(out["F"] - Fd, axis=0) / np.linalg.norm(Fd, axis=0)
    assert err.max() < 1e-10
    assert out["true_relres"].max() < 1e-11
    assert list(out["group_of"]) == [0, 0, 0, 0, 1, 1, 1, 1, 2, 2]


def test_block_cg_finite_termination():
    """In exact arithmetic the shared Krylov space grows by s dimensions per iteration,
    so s columns finish within ceil(n/s) iterations (here n = 24, s = 6: at most 4, plus
    one for rounding), where per-column CG needs up to n."""
    H, w, Y = _spd_case()
    lam = 0.05  # kappa(M) up to 21: per-column CG needs many iterations
    out = block_cg_solve(H, w, lam, Y, s=6, tol=1e-11)
    assert out["true_relres"].max() < 1e-10
    assert out["iters"].max() <= 24 // 6 + 1, out["iters"]
    per_col = cg_solve(H, w, lam, Y, tol=1e-11)
    assert per_col["iters"].max() > out["iters"].max()


def test_block_cg_s1_is_per_column_cg(small):
    """With s = 1 the block recurrences are CG's, up to the normalisation of p: the same
    iteration count and solution."""
    H, w, Y, lam = small
    a = block_cg_solve(H, w, lam, Y, s=1, tol=1e-10)
    b = cg_solve(H, w, lam, Y, tol=1e-10)
    assert np.array_equal(a["iters"], b["iters"])
    assert np.abs(a["F"] - b["F"]).max() < 1e-10 * np.abs(b["F"]).max()


def test_block_cg_dependent_and_zero_columns():
    """A repeated column and a zero column in one group: the rank-revealing search block
    drops the dependent directions instead of breaking down; the repeated columns get
    equal solutions and the zero column stays zero."""
    H, w, Y = _spd_case(seed=4)
    Y[:, 2] = Y[:, 0]
    Y[:, 3] = 0.0
    lam = 0.3
    out = block_cg_solve(H, w, lam, Y, s=6, tol=1e-12)
    Fd = solve_dense(H, w, lam, Y)
    assert np.abs(out["F"] - Fd).max() < 1e-10 * np.abs(Fd).max()
    assert np.abs(out["F"][:, 2] - out["F"][:, 0]).max() < 1e-10 * np.abs(Fd).max()
    assert np.abs(out["F"][:, 3]).max() == 0.0


def test_block_cg_preconditioned_and_warm_start(small):
    """With a Jacobi-like SPD preconditioner and a warm start from a nearby F, block CG
    still reaches the dense solution, in fewer iterations than from zero."""
    H, w, Y, lam = small
    Fd = solve_dense(H, w, lam, Y)
    d = np.diag(system_dense(H, w, lam))
    pre = lambda R: R / d[:, None]
    cold = block_cg_solve(H, w, lam, Y, s=5, tol=1e-12, precond=pre)
    warm = block_cg_solve(H, w, lam, Y, s=5, tol=1e-12, precond=pre, F0=Fd * (1 + 1e-6))
    for out in (cold, warm):
        assert np.abs(out["F"] - Fd).max() < 1e-10 * np.abs(Fd).max()
    assert warm["iters"].max() < cold["iters"].max()
