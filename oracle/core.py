"""Oracle: degrees, the operator Theta, the ranking solve, the weight gradient and the
simplex-constrained weight step (Sections 2 and 3, Eqs. 1-6 and 16-20).

All arithmetic is float64.  H is an n x m scipy sparse 0/1 matrix (see
``incidence.incidence_matrix``).

Readings of points the paper leaves open (each also listed in the design notes):
  * Zero-degree vertices.  A vertex whose hyperedges all have weight 0 has
    dv = 0; Dv^-1/2 is taken as the pseudo-inverse, s_v = 0, so its row and column
    of Theta vanish.
  * Gradient.  Section 2 defines dv through w, so the gradient of P(w) differentiates
    dv as well (``dv_frozen=True`` keeps only the explicit W term).
  * Weight step.  The active-set steepest descent of Eq. 5 is read as the Euclidean
    projection of w - eta * grad P onto {w >= 0, 1^T w = 1} (sort and threshold).
  * "Block" CG is one independent CG per right-hand-side column (Eqs. 16-20 applied
    column by column); the stopping test is ||r_j|| <= tol * ||lam y_j|| on the
    recursively updated residual.  O'Leary's shared-Krylov block CG is provided
    beside it (``block_cg_solve``) for groups of columns.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp

# ----------------------------------------------------------------------------
# degrees and scalings (Section 2)
# ----------------------------------------------------------------------------


def degrees(H: sp.spmatrix, w: np.ndarray):
    """dv = H w (weighted vertex degree), de = H^T 1 (hyperedge size), Section 2.

    Returns (dv, de, s, t) with s = dv^-1/2 (0 where dv = 0) and t = w / de, the two
    diagonal scalings of Eq. 1.
    """
    w = np.asarray(w, dtype=np.float64)
    dv = np.asarray(H @ w, dtype=np.float64).ravel()
    de = np.asarray(H.sum(axis=0), dtype=np.float64).ravel()
    s = np.zeros_like(dv)
    pos = dv > 0
    s[pos] = 1.0 / np.sqrt(dv[pos])
    t = w / de
    return dv, de, s, t


# ----------------------------------------------------------------------------
# the operator (Eq. 1) and the system matrix (Eq. 3 / Eq. 6)
# ----------------------------------------------------------------------------


def theta_dense(H: sp.spmatrix, w: np.ndarray) -> np.ndarray:
    """Theta = Dv^-1/2 H W De^-1 H^T Dv^-1/2 as a dense n x n array (Eq. 1)."""
    _, _, s, t = degrees(H, w)
    Hd = H.toarray()
    S = np.diag(s)
    return S @ Hd @ np.diag(t) @ Hd.T @ S


def theta_apply(H: sp.spmatrix, w: np.ndarray, X: np.ndarray, a: float = 0.0,
                b: float = 1.0) -> np.ndarray:
    """Z = a X + b Theta X, with Theta applied factor by factor from Eq. 1.

    (a, b) = (1 + lam, -1) gives M X with M = (1 + lam) I - Theta.
    """
    _, _, s, t = degrees(H, w)
    X = np.asarray(X, dtype=np.float64)
    G = s[:, None] * X                 # Dv^-1/2 X
    T = t[:, None] * (H.T @ G)         # W De^-1 H^T Dv^-1/2 X
    Z = s[:, None] * (H @ T)           # Dv^-1/2 H (...)
    return a * X + b * Z


def incidence_lists(n: int, m: int, edge_ptr, members):
    """Hyperedge -> members and vertex -> hyperedges lists (CSR-like arrays) built on the
    host from the input member lists: (edge_ptr, members, vert_ptr, vert_edges)."""
    edge_ptr = np.asarray(edge_ptr, dtype=np.int64)
    members = np.asarray(members, dtype=np.int64)
    edge_of = np.repeat(np.arange(m, dtype=np.int64), np.diff(edge_ptr))
    order = np.argsort(members, kind="stable")
    vert_edges = edge_of[order]
    vert_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(np.bincount(members, minlength=n), out=vert_ptr[1:])
    return edge_ptr, members, vert_ptr, vert_edges


def _dv_all(lists, w) -> np.ndarray:
    """dv = H w for every vertex (Section 2), summed over each vertex's hyperedge list."""
    edge_ptr, members, vert_ptr, vert_edges = lists
    n = vert_ptr.size - 1
    return np.bincount(np.repeat(np.arange(n), np.diff(vert_ptr)), weights=np.asarray(w)[vert_edges], minlength=n)


def theta_rows(lists, w, X_rows, rows, a: float = 0.0, b: float = 1.0) -> np.ndarray:
    """Rows `rows` of Z = a X + b Theta X evaluated one by one from Eq. 1:
        Z_v = a X_v + b s_v sum_{e ni v} (w_e / de_e) sum_{u in e} s_u X_u,
        s_u = (sum_{e' ni u} w_e')^-1/2 (0 where that sum is 0).
    `lists` is ``incidence_lists``; X_rows(u) returns the rows u of X (float64 array).
    For large graphs where only a few outputs can be checked."""
    edge_ptr, members, vert_ptr, vert_edges = lists
    w = np.asarray(w, dtype=np.float64)
    dv_all = _dv_all(lists, w)

    def s_of(u):
        dv = dv_all[np.asarray(u)]
        out = np.zeros_like(dv)
        out[dv > 0] = 1.0 / np.sqrt(dv[dv > 0])
        return out

    out = []
    for v in rows:
        sv = s_of([v])[0]
        acc = None
        for e in vert_edges[vert_ptr[v]:vert_ptr[v + 1]]:
            mem = members[edge_ptr[e]:edge_ptr[e + 1]]
            part = (s_of(mem)[:, None] * X_rows(mem)).sum(axis=0) * (w[e] / mem.size)
            acc = part if acc is None else acc + part
        xv = X_rows(np.array([v]))[0]
        z = a * xv
        if acc is not None:
            z = z + b * sv * acc
        out.append(z)
    return np.array(out)


def system_dense(H: sp.spmatrix, w: np.ndarray, lam: float) -> np.ndarray:
    """M = (1 + lam) I - Theta; M F = lam Y is Eq. 6 multiplied by (1 + lam)."""
    Th = theta_dense(H, w)
    return (1.0 + lam) * np.eye(Th.shape[0]) - Th


def solve_dense(H: sp.spmatrix, w: np.ndarray, lam: float, Y: np.ndarray) -> np.ndarray:
    """F* = lam/(1+lam) X^-1 Y (Eq. 3) through a dense Cholesky factorisation of M."""
    M = system_dense(H, w, lam)
    L = np.linalg.cholesky(M)
    Z = np.linalg.solve(L, lam * np.asarray(Y, dtype=np.float64))
    return np.linalg.solve(L.T, Z)


def cg_solve(H: sp.spmatrix, w: np.ndarray, lam: float, Y: np.ndarray, F0=None,
             tol: float = 1e-10, max_iter: int = 1000, record: bool = False,
             precond=None):
    """Conjugate gradient on M F = lam Y, one independent recurrence per column.

    Follows Eqs. 16-20: f_i = f_{i-1} + alpha_i p_{i-1}; r_i = r_{i-1} - alpha_i M p_{i-1};
    p_i = r_i + beta_i p_{i-1}; alpha_i = r^T r / p^T M p; beta_i = r_i^T r_i / r_{i-1}^T r_{i-1},
    starting from r_0 = lam y - M f_0, p_0 = r_0.  Column j stops once
    ||r_j|| <= tol ||lam y_j|| (a zero column stops at once with f = f_0 = 0).

    With ``precond`` (a function R -> P^-1 R, symmetric positive definite) this is
    the preconditioned form of the same recurrences (Barrett et al., Templates,
    the PCG algorithm): alpha = r^T z / p^T M p, beta = r_i^T z_i / r_{i-1}^T z_{i-1},
    p_i = z_i + beta p_{i-1} with z = P^-1 r; the stopping test stays on ||r||.

    Returns dict(F, iters[c], relres[c] (recursive), true_relres[c], history).
    """
    Y = np.asarray(Y, dtype=np.float64)
    n, c = Y.shape
    B = lam * Y
    F = np.zeros((n, c)) if F0 is None else np.array(F0, dtype=np.float64)
    R = B - theta_apply(H, w, F, 1.0 + lam, -1.0)
    Zp = R if precond is None else precond(R)
    P = Zp.copy()
    bnorm = np.sqrt((B * B).sum(axis=0))
    rr = (R * R).sum(axis=0)
    rz = (R * Zp).sum(axis=0)
    active = np.sqrt(rr) > tol * bnorm
    iters = np.zeros(c, dtype=np.int64)
    hist = {"R": [R.copy()], "P": [P.copy()], "F": [F.copy()]} if record else None
    for _ in range(max_iter):
        if not active.any():
            break
        Q = theta_apply(H, w, P, 1.0 + lam, -1.0)
        pq = (P * Q).sum(axis=0)
        alpha = np.where(active, rz / np.where(active, pq, 1.0), 0.0)
        F = F + alpha * P
        R = R - alpha * Q
        Zp = R if precond is None else precond(R)
        rz_new = (R * Zp).sum(axis=0)
        beta = np.where(active, rz_new / np.where(active, rz, 1.0), 0.0)
        P = np.where(active, Zp + beta * P, P)
        rz = np.where(active, rz_new, rz)
        rr = np.where(active, (R * R).sum(axis=0), rr)
        iters += active
        active = active & (np.sqrt(rr) > tol * bnorm)
        if record:
            hist["R"].append(R.copy())
            hist["P"].append(P.copy())
            hist["F"].append(F.copy())
    true_r = B - theta_apply(H, w, F, 1.0 + lam, -1.0)
    safe = np.where(bnorm > 0, bnorm, 1.0)
    return {
        "F": F, "iters": iters,
        "relres": np.sqrt(rr) / safe,
        "true_relres": np.sqrt((true_r * true_r).sum(axis=0)) / safe,
        "history": hist,
    }


def block_cg_solve(H: sp.spmatrix, w: np.ndarray, lam: float, Y: np.ndarray, s: int, F0=None,
                   tol: float = 1e-10, max_iter: int = 1000, precond=None, rank_tol: float = 1e-12):
    """Block CG with a shared Krylov space (O'Leary, "The block conjugate gradient
    algorithm and related methods", Linear Algebra Appl. 29, 1980) on M F = lam Y, the
    columns taken in groups of s.  Each group runs the block recurrences with the search
    block kept orthonormal and rank revealed, the breakdown-free form of Ji and Li
    (2017), so that columns that converge or become dependent leave the search space
    instead of making P^T M P singular:

        R_0 = B - M F_0,  Z_0 = P^-1 R_0,  P_0 = orth(Z_0)
        repeat:  Q = M P;  a = (P^T Q)^-1 P^T R;  F += P a;  R -= Q a
                 stop when ||r_j|| <= tol ||b_j|| for every column of the group
                 Z = P^-1 R;  b = -(P^T Q)^-1 Q^T Z;  P = orth(Z + P b)

    orth(.) is an orthonormal basis of the range from the SVD, dropping singular values
    below rank_tol times the largest (so P can have fewer than s columns).  With s = 1
    this is per-column CG up to the normalisation of p.  Returns dict(F, iters[groups],
    group_of[c], relres[c] (recursive), true_relres[c]).
    """
    Y = np.asarray(Y, dtype=np.float64)
    n, c = Y.shape
    B = lam * Y
    F = np.zeros((n, c)) if F0 is None else np.array(F0, dtype=np.float64)
    bnorm = np.sqrt((B * B).sum(axis=0))
    safe = np.where(bnorm > 0, bnorm, 1.0)
    relres = np.zeros(c)
    groups = [list(range(g0, min(g0 + s, c))) for g0 in range(0, c, s)]
    iters = np.zeros(len(groups), dtype=np.int64)
    group_of = np.zeros(c, dtype=np.int64)

    def orth(A):
        if A.shape[1] == 0:
            return A
        U, sv, _ = np.linalg.svd(A, full_matrices=False)
        if sv.size == 0 or sv[0] == 0.0:
            return A[:, :0]
        return U[:, sv > rank_tol * sv[0]]

    for gi, cols in enumerate(groups):
        group_of[cols] = gi
        R = B[:, cols] - theta_apply(H, w, F[:, cols], 1.0 + lam, -1.0)
        Fg = F[:, cols].copy()
        conv = lambda R_: bool((np.sqrt((R_ * R_).sum(axis=0)) <= tol * bnorm[cols]).all())
        if not conv(R):
            P = orth(R if precond is None else precond(R))
            for _ in range(max_iter):
                if P.shape[1] == 0:
                    break
                Q = theta_apply(H, w, P, 1.0 + lam, -1.0)
                PQ = P.T @ Q
                a = np.linalg.solve(PQ, P.T @ R)
                Fg = Fg + P @ a
                R = R - Q @ a
                iters[gi] += 1
                if conv(R):
                    break
                Z = R if precond is None else precond(R)
                b = -np.linalg.solve(PQ, Q.T @ Z)
                P = orth(Z + P @ b)
        F[:, cols] = Fg
        relres[cols] = np.sqrt((R * R).sum(axis=0)) / safe[cols]
    true_r = B - theta_apply(H, w, F, 1.0 + lam, -1.0)
    return {"F": F, "iters": iters, "group_of": group_of, "relres": relres,
            "true_relres": np.sqrt((true_r * true_r).sum(axis=0)) / safe}


def cg_iteration_bound(lam: float, tol: float) -> int:
    """Chebyshev bound on CG iterations for ||e||_M reduction tol with
    kappa(M) <= (1 + lam) / lam (spectrum of Theta in [0, 1])."""
    kappa = (1.0 + lam) / lam
    rate = (math.sqrt(kappa) + 1.0) / (math.sqrt(kappa) - 1.0)
    return int(math.ceil(math.log(2.0 / tol) / math.log(rate)))


def certified_solve(H, w, lam, Y, tol=1e-13, max_iter=2000):
    """CG to a tight residual with the a-posteriori bound ||F_j - F*_j|| <= ||r_j|| / lam.

    The bound holds because lambda_min(M) >= lam (spectrum of Theta in [0, 1]).
    Returns (F, err_bound[c]) with err_bound from the recomputed residual.
    """
    out = cg_solve(H, w, lam, Y, tol=tol, max_iter=max_iter)
    F = out["F"]
    R = lam * np.asarray(Y, dtype=np.float64) - theta_apply(H, w, F, 1.0 + lam, -1.0)
    return F, np.sqrt((R * R).sum(axis=0)) / lam


# ----------------------------------------------------------------------------
# objective and weight gradient (Section 2, Eqs. 2 and 4)
# ----------------------------------------------------------------------------


def objective(H, w, F, mu: float) -> float:
    """P(w) = tr(F^T Delta F) + mu ||w||^2 (Eq. 4 summed over the columns of F)."""
    F = np.asarray(F, dtype=np.float64)
    TF = theta_apply(H, w, F, 0.0, 1.0)
    return float((F * F).sum() - (F * TF).sum() + mu * np.dot(w, w))


def full_loss(H, w, F, Y, lam: float, mu: float) -> float:
    """tr(F^T Delta F) + lam ||F - Y||^2 + mu ||w||^2."""
    D = np.asarray(F) - np.asarray(Y)
    return objective(H, w, F, mu) + lam * float((D * D).sum())


def bilinear_theta_grad(H, w, F, Z, dv_frozen: bool = False) -> np.ndarray:
    """d/dw_e of tr(Z^T Theta(w) F), including the dependence of dv on w.

    With G = Dv^-1/2 F, R = Dv^-1/2 Z, sF = H^T G, sZ = H^T R (m x c) and
    UF = H diag(w/de) sF, UZ = H diag(w/de) sZ (n x c):
        d/dw_e = <sF_e, sZ_e> / de_e
                 - 1/2 sum_{v in e} (1/dv_v) (<G_v, UZ_v> + <R_v, UF_v>).
    The first term is the explicit W De^-1 factor; the second comes from
    dDv^-1/2 / dw_e = -1/2 Dv^-3/2 H(:, e).  Vertices with dv = 0 contribute 0.
    """
    dv, de, s, t = degrees(H, w)
    F = np.asarray(F, dtype=np.float64)
    Z = np.asarray(Z, dtype=np.float64)
    G = s[:, None] * F
    R = s[:, None] * Z
    sF = H.T @ G
    sZ = H.T @ R
    explicit = (sF * sZ).sum(axis=1) / de
    if dv_frozen:
        return explicit
    UF = H @ (t[:, None] * sF)
    UZ = H @ (t[:, None] * sZ)
    inv_dv = np.zeros_like(dv)
    inv_dv[dv > 0] = 1.0 / dv[dv > 0]
    per_vertex = inv_dv * ((G * UZ).sum(axis=1) + (R * UF).sum(axis=1))
    return explicit - 0.5 * (H.T @ per_vertex)


def weight_grad_entries(lists, w, F_rows, edges, mu: float) -> np.ndarray:
    """Entries `edges` of grad_w P(w) = -d tr(F^T Theta F)/dw + 2 mu w (Eq. 4 at fixed F,
    dv(w) included), evaluated hyperedge by hyperedge for large graphs:
        d/dw_e tr(F^T Theta F) = ||sF_e||^2 / de_e - sum_{v in e} <G_v, UF_v> / dv_v,
    G = Dv^-1/2 F, sF_e = sum_{u in e} G_u, UF_v = sum_{e' ni v} (w_e'/de_e') sF_e'.
    `lists` is ``incidence_lists``; F_rows(u) returns the rows u of F (float64)."""
    edge_ptr, members, vert_ptr, vert_edges = lists
    w = np.asarray(w, dtype=np.float64)
    dv_all = _dv_all(lists, w)

    def dv_of(u):
        return dv_all[np.asarray(u)]

    def g_rows(u):
        dv = dv_of(u)
        s = np.zeros_like(dv)
        s[dv > 0] = 1.0 / np.sqrt(dv[dv > 0])
        return s[:, None] * F_rows(u), dv

    def sF(e):
        return g_rows(members[edge_ptr[e]:edge_ptr[e + 1]])[0].sum(axis=0)

    out = []
    for e in edges:
        mem = members[edge_ptr[e]:edge_ptr[e + 1]]
        se = sF(e)
        val = float(se @ se) / mem.size
        G, dv = g_rows(mem)
        for i, v in enumerate(mem):
            if dv[i] <= 0:
                continue
            UF = sum((w[f] / (edge_ptr[f + 1] - edge_ptr[f])) * sF(f) for f in vert_edges[vert_ptr[v]:vert_ptr[v + 1]])
            val -= float(G[i] @ UF) / dv[i]
        out.append(-val + 2.0 * mu * w[e])
    return np.array(out)


def weight_grad(H, w, F, mu: float, dv_frozen: bool = False) -> np.ndarray:
    """grad_w P(w) at fixed F: -d tr(F^T Theta F)/dw + 2 mu w (Eq. 4, F fixed).

    tr(F^T Delta F) = ||F||^2 - tr(F^T Theta F), and ||F||^2 does not depend on w.
    """
    return -bilinear_theta_grad(H, w, F, F, dv_frozen) + 2.0 * mu * np.asarray(w, np.float64)


# ----------------------------------------------------------------------------
# differentiation through the solve (adjoint method)
# ----------------------------------------------------------------------------


def adjoint_solve(H, w, lam: float, G, dense: bool = True, tol: float = 1e-13) -> np.ndarray:
    """Z = M^-1 G.  M = (1+lam) I - Theta is symmetric, so the adjoint of the ranking
    system (Eq. 6) has the same operator; the transposed right-hand side is G."""
    G = np.asarray(G, dtype=np.float64)
    if dense:
        return np.linalg.solve(system_dense(H, w, lam), G)
    return cg_solve(H, w, lam, G / lam, tol=tol)["F"]


def solve_grad_w(H, w, lam: float, F, G, dv_frozen: bool = False, dense: bool = True):
    """d/dw of <G, F(w)> where M(w) F = lam Y, at fixed G (the gradient of a loss with
    respect to F).  Differentiating M F = lam Y gives dF = -M^-1 (dM) F, and
    dM/dw_e = -dTheta/dw_e, so with Z = M^-1 G

        <G, dF/dw_e> = d/dw_e tr(Z^T Theta(w) F)   (Z and F held fixed),

    the bilinear gradient of Eq. 1.  Returns (gradient[m], Z)."""
    Z = adjoint_solve(H, w, lam, G, dense=dense)
    return bilinear_theta_grad(H, w, F, Z, dv_frozen), Z


def zhou_loss(H, w, Y, lam: float, mu: float, F=None):
    """L(w) = tr(F^T Delta F) + lam ||F - Y||^2 + mu ||w||^2 at F = F(w) (Eq. 4 with the
    ranking term of Eq. 3).  Returns (L, F, dL/dF at fixed w, explicit dL/dw at fixed F)."""
    if F is None:
        F = solve_dense(H, w, lam, Y)
    L = full_loss(H, w, F, Y, lam, mu)
    dF = 2.0 * theta_apply(H, w, F, 1.0, -1.0) + 2.0 * lam * (F - np.asarray(Y, np.float64))
    dw = weight_grad(H, w, F, mu)
    return L, F, dF, dw


def heldout_loss(H, w, Y, lam: float, rows, Y_test, F=None):
    """L(w) = ||F(w)[rows] - Y_test||^2: a loss on held-out vertices with no explicit
    dependence on w, whose adjoint right-hand side does not vanish at the solution.
    Returns (L, F, dL/dF, explicit dL/dw = 0)."""
    if F is None:
        F = solve_dense(H, w, lam, Y)
    D = F[rows] - np.asarray(Y_test, np.float64)
    dF = np.zeros_like(F)
    dF[rows] = 2.0 * D
    return float((D * D).sum()), F, dF, np.zeros(np.asarray(w).shape[0])


def total_grad(H, w, Y, lam: float, loss, dense: bool = True, **kw):
    """dL/dw = explicit dL/dw + <dL/dF, dF/dw> (adjoint term), for ``loss`` one of
    ``zhou_loss`` / ``heldout_loss`` (extra keyword arguments go to the loss)."""
    L, F, dF, dw = loss(H, w, Y, lam, **kw)
    adj, Z = solve_grad_w(H, w, lam, F, dF, dense=dense)
    return L, dw + adj, adj, Z


# ----------------------------------------------------------------------------
# simplex projection (Eq. 5 read as a Euclidean projection)
# ----------------------------------------------------------------------------


def project_simplex(v: np.ndarray) -> np.ndarray:
    """Euclidean projection of v onto {w >= 0, sum w = 1} by sort and threshold.

    Sort v in decreasing order u; the support size is the largest j with
    u_j - (sum_{i<=j} u_i - 1) / j > 0; the threshold is tau = (sum_{i<=rho} u_i - 1)/rho
    and w = max(v - tau, 0) (Held, Wolfe and Crowder 1974; Duchi et al. 2008).
    """
    v = np.asarray(v, dtype=np.float64)
    u = np.sort(v)[::-1]
    css = np.cumsum(u)
    j = np.arange(1, v.size + 1)
    cond = u - (css - 1.0) / j > 0
    rho = int(j[cond][-1])
    tau = (css[rho - 1] - 1.0) / rho
    return np.maximum(v - tau, 0.0)


def active_set_step(w, g, eta: float) -> np.ndarray:
    """The steepest-descent step of Eq. 5 read literally.  Active constraints: G_1
    (1^T w = 1, always active) and G_j (w_e = 0) for every weight already at 0.  Their
    multipliers make the direction nabla S = nabla P + c_1 1 + sum_j c_j e_j vanish on the
    pinned weights and sum to zero over the free ones:
        d_e = g_e - mean_{free}(g)  (w_e > 0),   d_e = 0  (w_e = 0).
    w - eta d is clamped at 0 (weights that cross 0 join the pinned set) and rescaled to
    sum 1.  With no free weight, or nothing left after clamping, w is returned unchanged."""
    w = np.asarray(w, dtype=np.float64)
    g = np.asarray(g, dtype=np.float64)
    free = w > 0
    if not free.any():
        return w.copy()
    d = np.where(free, g - g[free].mean(), 0.0)
    v = np.where(free, np.maximum(w - eta * d, 0.0), 0.0)
    total = v.sum()
    return v / total if total > 0 else w.copy()


def simplex_threshold(v: np.ndarray) -> float:
    """The tau of ``project_simplex``."""
    v = np.asarray(v, dtype=np.float64)
    u = np.sort(v)[::-1]
    css = np.cumsum(u)
    j = np.arange(1, v.size + 1)
    rho = int(j[u - (css - 1.0) / j > 0][-1])
    return (css[rho - 1] - 1.0) / rho


# ----------------------------------------------------------------------------
# the alternation (Section 2: f at fixed w, then w at fixed f)
# ----------------------------------------------------------------------------


def adaptive_step(H, w, lam, mu, eta, Y, F0=None, tol=1e-10, solver="cg", max_iter=1000,
                  dv_frozen=False):
    """One outer iteration: solve M F = lam Y at the current w (warm start F0), then
    w <- Proj_simplex(w - eta grad P(w)) at that F.

    Returns dict(F, w_new, grad, iters, relres).
    """
    if solver == "dense":
        F = solve_dense(H, w, lam, Y)
        iters = None
        relres = None
    else:
        out = cg_solve(H, w, lam, Y, F0=F0, tol=tol, max_iter=max_iter)
        F, iters, relres = out["F"], out["iters"], out["relres"]
    g = weight_grad(H, w, F, mu, dv_frozen)
    w_new = project_simplex(np.asarray(w, np.float64) - eta * g)
    return {"F": F, "w_new": w_new, "grad": g, "iters": iters, "relres": relres}


def adaptive_loop(H, w0, lam, mu, eta, Y, steps, tol=1e-10, solver="cg"):
    """``steps`` outer iterations from w0 with F warm-started from the previous step.

    Returns (F_final_solve_at_last_w_before_update, w_after_last_update, trace).
    """
    w = np.array(w0, dtype=np.float64)
    F = None
    trace = []
    for _ in range(steps):
        out = adaptive_step(H, w, lam, mu, eta, Y, F0=F, tol=tol, solver=solver)
        F = out["F"]
        w = out["w_new"]
        trace.append(out)
    return F, w, trace
