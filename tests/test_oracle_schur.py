"""Pins of the oracle's nested 2 x 2 Schur-complement inverse (Section 3, Eqs. 12-14)."""
import numpy as np
import pytest

from oracle.core import theta_dense
from oracle.incidence import build_incidence, incidence_matrix
from oracle.schur import lowrank_inverse, schur_inverse, schur_inverse_exact


def _theta(n, m, seed):
    rng = np.random.default_rng(seed)
    ptr, mem = [0], []
    for _ in range(m):
        k = int(rng.integers(2, 8))
        mem.extend(sorted(rng.choice(n, k, replace=False)))
        ptr.append(len(mem))
    H = incidence_matrix(build_incidence(n, m, np.asarray(ptr, np.int64), np.asarray(mem, np.int32)))
    w = rng.random(m) + 0.1
    return theta_dense(H, w / w.sum())


def test_two_by_two_formula_is_the_inverse():
    """One level with exact inverses of M11, M22, Z1, Z2 (the formula of Section 3)
    equals the inverse of a generic SPD matrix, odd size included."""
    rng = np.random.default_rng(1)
    for n in (40, 41):
        A = rng.standard_normal((n, n))
        M = A @ A.T + n * np.eye(n)
        assert np.abs(schur_inverse_exact(M) @ M - np.eye(n)).max() < 1e-12


@pytest.mark.parametrize("n,r_min", [(64, 8), (61, 5), (30, 20)])
def test_nested_full_rank_is_exact(n, r_min):
    """With the rank at least every block's size the randomized SVD captures each matrix
    exactly, so the nested scheme (several levels for (64, 8), odd halves for (61, 5),
    a single leaf for (30, 20)) returns M^-1 to rounding, and it is symmetric."""
    lam = 0.5
    T = _theta(n, 2 * n, seed=n)
    M = (1 + lam) * np.eye(n) - T
    Minv = schur_inverse(T, lam, r_min=r_min, k=n, p=0, q=1, seed=7)
    assert np.abs(Minv @ M - np.eye(n)).max() < 1e-10
    assert np.abs(Minv - Minv.T).max() < 1e-10


def test_lowrank_inverse_is_exact_on_the_captured_subspace():
    """((1+lam) I - L)^-1 from a rank-k Rayleigh-Ritz factorisation: exact when L has
    rank <= k (the captured subspace holds all of it)."""
    rng = np.random.default_rng(2)
    n, r, lam = 50, 6, 1.0
    U = np.linalg.qr(rng.standard_normal((n, r)))[0]
    L = U @ np.diag(rng.random(r) * 1.5) @ U.T
    Minv = lowrank_inverse(L, lam, np.arange(n), k=r, p=4, q=2, seed=3)
    assert np.abs(Minv @ ((1 + lam) * np.eye(n) - L) - np.eye(n)).max() < 1e-12


def test_error_falls_with_the_rank():
    """Truncated ranks: the distance to M^-1 falls as k grows, down to rounding at full
    rank (a dropped eigen-direction or a wrong gain would break the ordering)."""
    n, lam = 64, 0.5
    T = _theta(n, 160, seed=5)
    Mi = np.linalg.inv((1 + lam) * np.eye(n) - T)
    errs = [np.linalg.norm(schur_inverse(T, lam, r_min=8, k=k, p=4, q=2, seed=11) - Mi) / np.linalg.norm(Mi)
            for k in (1, 3, 8, 64)]
    assert errs[0] > errs[1] > errs[2] > 1e3 * errs[3], errs
    assert errs[3] < 1e-10
