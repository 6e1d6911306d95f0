"""Oracle: the nested 2 x 2 Schur-complement inverse of Section 3 (Hackbusch's block
inverse, Eqs. 12-14), with the diagonal blocks and the Schur complements inverted by
randomized SVD (Algorithm 1) and nested tessellation of the diagonal blocks -- TEST
INFRASTRUCTURE (see the package docstring for who may import it).

For a symmetric positive definite M split as [[M11, M12], [M21, M22]]:

    M^-1 = [[ Z1^-1,                 -M11^-1 M12 Z2^-1 ],
            [ -Z2^-1 M21 M11^-1,      Z2^-1            ]]
    Z1 = M11 - M12 M22^-1 M21,   Z2 = M22 - M21 M11^-1 M12.

Readings (also listed in the design notes):
  * The matrix is M = (1+lam) I - Theta (the paper's X scaled by 1+lam).  Every matrix
    this scheme inverts has the form (1+lam) I - L with L symmetric positive
    semidefinite: a diagonal block (L = Theta_bb) or a Schur complement (L = Theta_11 +
    Theta_12 M22^-1 Theta_21, since M12 = -Theta_12).  As for the block preconditioner,
    "inverted by randomized SVD" is read as the exact inverse on the subspace that
    Algorithm 1 (Rayleigh-Ritz form) captures for L, and 1/(1+lam) on its complement:
        ((1+lam) I - L)^-1 ~= I/(1+lam) + Q diag(l/((1+lam)(1+lam-l))) Q^T.
  * Nested tessellation: a diagonal block larger than 2 * r_min is itself split in
    two halves (the first half rounded down) and inverted by the same scheme; blocks of
    at most 2 * r_min rows (the "minimum rank" of Section 3 read as the smallest block
    that is split no further) are inverted by the randomized SVD directly.  The Schur
    complements are inverted by the randomized SVD directly.
  * Omega for a submatrix uses the Philox stream of the block preconditioner on the
    submatrix's global rows; the rank is min(k, rows) and the sketch min(k + p, rows).
"""
from __future__ import annotations

import numpy as np

from .philox import omega
from .rsvd import rsvd_ritz


def lowrank_inverse(L: np.ndarray, lam: float, rows: np.ndarray, k: int, p: int, q: int, seed: int) -> np.ndarray:
    """((1+lam) I - L)^-1 from the Rayleigh-Ritz rSVD of the symmetric PSD part L (dense)."""
    nb = L.shape[0]
    kb, lb = min(k, nb), min(k + p, nb)
    Om = omega(rows, k + p, seed)[:, :lb]
    Q, ev = rsvd_ritz(0.5 * (L + L.T), Om, q, kb)
    ev = np.clip(ev, 0.0, None)
    g = ev / ((1.0 + lam) * (1.0 + lam - ev))
    return np.eye(nb) / (1.0 + lam) + (Q * g[None, :]) @ Q.T


def schur_inverse(Theta: np.ndarray, lam: float, r_min: int, k: int, p: int, q: int, seed: int,
                  row0: int = 0) -> np.ndarray:
    """Approximate M^-1 for M = (1+lam) I - Theta (dense symmetric Theta, rows row0...)
    by the nested 2 x 2 Schur-complement scheme above."""
    n = Theta.shape[0]
    rows = np.arange(row0, row0 + n)
    if n <= 2 * r_min:
        return lowrank_inverse(Theta, lam, rows, k, p, q, seed)
    h = n // 2
    T11, T12 = Theta[:h, :h], Theta[:h, h:]
    T21, T22 = Theta[h:, :h], Theta[h:, h:]
    inv11 = schur_inverse(T11, lam, r_min, k, p, q, seed, row0)
    inv22 = schur_inverse(T22, lam, r_min, k, p, q, seed, row0 + h)
    # M12 = -T12, M21 = -T21: Z1 = (1+lam) I - (T11 + T12 M22^-1 T21), likewise Z2
    Z1inv = lowrank_inverse(T11 + T12 @ inv22 @ T21, lam, rows[:h], k, p, q, seed)
    Z2inv = lowrank_inverse(T22 + T21 @ inv11 @ T12, lam, rows[h:], k, p, q, seed)
    out = np.empty((n, n))
    out[:h, :h] = Z1inv
    out[h:, h:] = Z2inv
    out[:h, h:] = inv11 @ T12 @ Z2inv       # -M11^-1 M12 Z2^-1
    out[h:, :h] = Z2inv @ T21 @ inv11       # -Z2^-1 M21 M11^-1
    return out


def schur_inverse_exact(M: np.ndarray) -> np.ndarray:
    """One level of the 2 x 2 formula with exact inverses of M11, M22, Z1 and Z2."""
    n = M.shape[0]
    h = n // 2
    M11, M12, M21, M22 = M[:h, :h], M[:h, h:], M[h:, :h], M[h:, h:]
    i11, i22 = np.linalg.inv(M11), np.linalg.inv(M22)
    Z1 = M11 - M12 @ i22 @ M21
    Z2 = M22 - M21 @ i11 @ M12
    z1, z2 = np.linalg.inv(Z1), np.linalg.inv(Z2)
    out = np.empty((n, n))
    out[:h, :h] = z1
    out[h:, h:] = z2
    out[:h, h:] = -i11 @ M12 @ z2
    out[h:, :h] = -z2 @ M21 @ i11
    return out
