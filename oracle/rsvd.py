"""Oracle: tessellation blocks, randomized SVD by subspace iteration (Algorithm 1),
and the low-rank block inverse used as a preconditioner (Section 3, Eqs. 7-15).

Readings (also listed in the design notes):
  * The diagonal blocks X_bb of X = I - Theta/(1+theta) contain a scaled identity and
    are not low rank (Section 3 calls them low rank).  Algorithm 1 is applied to the
    low-rank part Theta_bb (symmetric positive semidefinite), and M_bb = (1+lam) I -
    Theta_bb is inverted exactly on the captured subspace:
        M_bb^-1 ~= I/(1+lam) + Q diag(g) Q^T,   g_i = l_i / ((1+lam)(1+lam-l_i)),
    the eigen form of X^-1 = V Sigma^-1 U^T (Eq. 15) completed by the identity part.
  * Tessellation blocks are contiguous vertex ranges in natural order; only the
    diagonal blocks are used (block Jacobi).  The Schur-complement 2x2 inverse of
    Eqs. 12-14 is not part of this path.
  * The oversampling and the iteration count are both called pi in Section 3 and
    Algorithm 1; here p is the oversampling (l = k + p) and q the iteration count.
  * Theta_bb is symmetric, so the X^T products of Algorithm 1 equal X products.
    ``rsvd_alg1`` follows Algorithm 1 as printed (SVD of B = S^T X);
    ``rsvd_ritz`` keeps the same range finder and replaces steps 4-6 by the
    Rayleigh-Ritz eigendecomposition of S^T Theta S (l x l), which gives a symmetric
    factorisation Q diag(l) Q^T.  QR factors are normalised to a non-negative
    diagonal of R, which makes them unique.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .core import degrees
from .philox import omega


def block_theta(H: sp.spmatrix, w: np.ndarray, block_ptr) -> list:
    """Dense diagonal blocks Theta[b0:b1, b0:b1] of Eq. 1 for each block [b0, b1)."""
    _, _, s, t = degrees(H, w)
    Hc = sp.csr_matrix(H)
    out = []
    for b in range(len(block_ptr) - 1):
        b0, b1 = int(block_ptr[b]), int(block_ptr[b + 1])
        Hb = Hc[b0:b1, :]
        inner = (Hb @ sp.diags(t) @ Hb.T).toarray()
        sb = s[b0:b1]
        out.append(sb[:, None] * inner * sb[None, :])
    return out


def qr_pos(Y: np.ndarray):
    """Thin QR with diag(R) >= 0 (Householder QR from LAPACK, signs normalised)."""
    Q, R = np.linalg.qr(Y, mode="reduced")
    sgn = np.sign(np.diag(R))
    sgn[sgn == 0] = 1.0
    return Q * sgn[None, :], R * sgn[:, None]


def range_finder(X: np.ndarray, Omega: np.ndarray, q: int) -> np.ndarray:
    """Steps 1-3 of Algorithm 1: S0 from QR(X Omega), then q times
    S~ = QR(X^T S), S = QR(X S~)."""
    S, _ = qr_pos(X @ Omega)
    for _ in range(q):
        St, _ = qr_pos(X.T @ S)
        S, _ = qr_pos(X @ St)
    return S


def rsvd_alg1(X: np.ndarray, Omega: np.ndarray, q: int, k: int):
    """Algorithm 1 as printed: B = S^T X, SVD B = U~ Sigma V^T, U = S U~ (top k)."""
    S = range_finder(X, Omega, q)
    B = S.T @ X
    Ut, sig, Vt = np.linalg.svd(B, full_matrices=False)
    U = S @ Ut
    return U[:, :k], sig[:k], Vt[:k, :].T


def rsvd_ritz(X: np.ndarray, Omega: np.ndarray, q: int, k: int):
    """Same range finder; steps 4-6 as Rayleigh-Ritz on the symmetric X:
    T = S^T X S, eig T = V diag(l) V^T (descending), Q = S V (top k)."""
    S = range_finder(X, Omega, q)
    T = S.T @ X @ S
    T = 0.5 * (T + T.T)
    lam, V = np.linalg.eigh(T)
    order = np.argsort(lam)[::-1]
    lam, V = lam[order], V[:, order]
    return S @ V[:, :k], lam[:k]


def block_eig(Xb: np.ndarray, k: int):
    """Exact top-k eigenpairs of a symmetric block (numpy eigh), descending."""
    lam, V = np.linalg.eigh(0.5 * (Xb + Xb.T))
    order = np.argsort(lam)[::-1][:k]
    return V[:, order], lam[order]


def block_rsvd(H, w, block_ptr, k: int, p: int, q: int, seed: int):
    """Rayleigh-Ritz rSVD of every diagonal block with the shared Philox Omega.

    Returns a list of (Q_b [b x k], l_b [k]).
    """
    l = k + p
    blocks = block_theta(H, w, block_ptr)
    out = []
    for b, Tb in enumerate(blocks):
        b0, b1 = int(block_ptr[b]), int(block_ptr[b + 1])
        kb = min(k, b1 - b0)
        lb = min(l, b1 - b0)
        Om = omega(np.arange(b0, b1), l, seed)[:, :lb]
        out.append(rsvd_ritz(Tb, Om, q, kb))
    return out


def precond_apply(factors, block_ptr, lam: float, R: np.ndarray) -> np.ndarray:
    """z_b = r_b/(1+lam) + Q_b diag(g_b) Q_b^T r_b with g = l/((1+lam)(1+lam-l))."""
    R = np.asarray(R, dtype=np.float64)
    Z = R / (1.0 + lam)
    for b, (Q, ev) in enumerate(factors):
        b0, b1 = int(block_ptr[b]), int(block_ptr[b + 1])
        g = ev / ((1.0 + lam) * (1.0 + lam - ev))
        Z[b0:b1] += Q @ (g[:, None] * (Q.T @ R[b0:b1]))
    return Z
