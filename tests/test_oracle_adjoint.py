"""Pins of the oracle's differentiation through the ranking solve (adjoint method).

The adjoint gradient dL/dw = explicit dL/dw + d/dw tr(Z^T Theta F), Z = M^-1 dL/dF, is
checked against differentiations that share nothing with it: central differences of
the loss through a dense solve, and torch.autograd through a dense Theta(w) and
torch.linalg.solve.  Two losses: the regularised objective of Eqs. 3-4 (whose adjoint
right-hand side vanishes at the solution, since F minimises its first two terms) and
a held-out loss whose adjoint term is the whole gradient.
"""
import numpy as np
import pytest
import torch

from oracle.core import (adjoint_solve, heldout_loss, solve_dense, solve_grad_w, total_grad, zhou_loss)
from oracle.incidence import build_incidence, incidence_matrix
from tests._util import dense_incidence, tiny_hypergraph


def _case(seed, n=14, m=11, c=3):
    rng = np.random.default_rng(seed)
    ptr, mem = tiny_hypergraph(rng, n, m, 2)
    H = incidence_matrix(build_incidence(n, m, ptr, mem))
    w = rng.random(m) + 0.3
    Y = (rng.random((n, c)) < 0.3).astype(np.float64)
    rows = rng.choice(n, size=n // 3, replace=False)
    Yt = rng.random((rows.size, c))
    return H, w, Y, rows, Yt, dense_incidence(n, m, ptr, mem)


def _loss_value(H, w, Y, lam, kind, mu, rows, Yt):
    if kind == "zhou":
        return zhou_loss(H, w, Y, lam, mu)[0]
    return heldout_loss(H, w, Y, lam, rows, Yt)[0]


def _grad(H, w, Y, lam, kind, mu, rows, Yt):
    if kind == "zhou":
        return total_grad(H, w, Y, lam, zhou_loss, mu=mu)
    return total_grad(H, w, Y, lam, heldout_loss, rows=rows, Y_test=Yt)


@pytest.mark.parametrize("kind", ["zhou", "heldout"])
@pytest.mark.parametrize("seed", range(4))
def test_adjoint_gradient_central_differences(kind, seed):
    H, w, Y, rows, Yt, _ = _case(seed)
    lam, mu, h = 0.7, 1e-3, 1e-6
    _, g, _, _ = _grad(H, w, Y, lam, kind, mu, rows, Yt)
    fd = np.zeros_like(w)
    for e in range(w.size):
        wp, wm = w.copy(), w.copy()
        wp[e] += h
        wm[e] -= h
        fd[e] = (_loss_value(H, wp, Y, lam, kind, mu, rows, Yt) - _loss_value(H, wm, Y, lam, kind, mu, rows, Yt)) / (2 * h)
    assert np.allclose(g, fd, rtol=1e-6, atol=1e-8 * max(1.0, np.abs(fd).max()))


def _torch_loss(Hd, w, Y, lam, kind, mu, rows, Yt):
    """The same losses written with dense torch ops (Theta from Eq. 1, solve of Eq. 6)."""
    Ht = torch.tensor(Hd, dtype=torch.float64)
    wt = torch.tensor(w, dtype=torch.float64, requires_grad=True)
    Yt_ = torch.tensor(Y, dtype=torch.float64)
    de = Ht.sum(dim=0)
    dv = Ht @ wt
    S = torch.diag(dv.rsqrt())
    Th = S @ Ht @ torch.diag(wt / de) @ Ht.T @ S
    n = Hd.shape[0]
    M = (1 + lam) * torch.eye(n, dtype=torch.float64) - Th
    F = torch.linalg.solve(M, lam * Yt_)
    if kind == "zhou":
        L = (F * (F - Th @ F)).sum() + lam * ((F - Yt_) ** 2).sum() + mu * (wt ** 2).sum()
    else:
        L = ((F[torch.tensor(rows)] - torch.tensor(Yt)) ** 2).sum()
    L.backward()
    return float(L.detach()), wt.grad.numpy()


@pytest.mark.parametrize("kind", ["zhou", "heldout"])
@pytest.mark.parametrize("seed", range(3))
def test_adjoint_gradient_matches_torch_autograd(kind, seed):
    H, w, Y, rows, Yt, Hd = _case(10 + seed)
    lam, mu = 1.0, 1e-3
    L, g, _, _ = _grad(H, w, Y, lam, kind, mu, rows, Yt)
    Lt, gt = _torch_loss(Hd, w, Y, lam, kind, mu, rows, Yt)
    assert np.isclose(L, Lt, rtol=1e-12)
    assert np.allclose(g, gt, rtol=1e-9, atol=1e-12 * np.abs(gt).max())


@pytest.mark.parametrize("seed", range(3))
def test_envelope_adjoint_term_vanishes_for_the_regularised_objective(seed):
    """F(w) minimises tr(F^T Delta F) + lam ||F - Y||^2, so dL/dF = 2 (M F - lam Y) = 0:
    the adjoint term is zero up to the solve's rounding and the gradient is the
    fixed-F gradient of Eq. 4."""
    H, w, Y, rows, Yt, _ = _case(20 + seed)
    L, g, adj, Z = total_grad(H, w, Y, 0.5, zhou_loss, mu=1e-3)
    _, _, dF, dw = zhou_loss(H, w, Y, 0.5, 1e-3)
    assert np.abs(dF).max() <= 1e-12 * max(1.0, np.abs(Y).max())
    assert np.abs(adj).max() <= 1e-10 * np.abs(dw).max()


@pytest.mark.parametrize("seed", range(3))
def test_heldout_gradient_is_orthogonal_to_w(seed):
    """Theta(alpha w) = Theta(w) for alpha > 0 (dv and W scale alike), so a loss that
    depends on w only through F is constant along w: w^T dL/dw = 0."""
    H, w, Y, rows, Yt, _ = _case(30 + seed)
    _, g, adj, _ = total_grad(H, w, Y, 0.8, heldout_loss, rows=rows, Y_test=Yt)
    assert np.array_equal(g, adj)
    assert abs(float(w @ g)) <= 1e-10 * float(np.abs(w).sum() * np.abs(g).max())


def test_adjoint_solve_dense_and_cg_agree():
    H, w, Y, rows, Yt, _ = _case(40, n=40, m=30, c=4)
    G = np.random.default_rng(1).standard_normal((40, 4))
    Zd = adjoint_solve(H, w, 0.5, G, dense=True)
    Zc = adjoint_solve(H, w, 0.5, G, dense=False)
    assert np.allclose(Zd, Zc, rtol=1e-10, atol=1e-12)
    F = solve_dense(H, w, 0.5, Y)
    gd, _ = solve_grad_w(H, w, 0.5, F, G, dense=True)
    gc, _ = solve_grad_w(H, w, 0.5, F, G, dense=False)
    assert np.allclose(gd, gc, rtol=1e-9, atol=1e-12)
