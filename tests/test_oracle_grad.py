"""Pins of the oracle's weight gradient (Eq. 4 at fixed F) and simplex step (Eq. 5)."""
import itertools

import numpy as np
import pytest
import torch

from oracle.core import (adaptive_loop, bilinear_theta_grad, degrees, objective,
                         project_simplex, simplex_threshold, theta_apply, weight_grad)
from oracle.incidence import build_incidence, incidence_matrix
from tests._util import dense_incidence, tiny_hypergraph


def _case(seed, n=9, m=7, c=3):
    rng = np.random.default_rng(seed)
    ptr, mem = tiny_hypergraph(rng, n, m, 2)
    H = incidence_matrix(build_incidence(n, m, ptr, mem))
    w = rng.random(m) + 0.2
    F = rng.standard_normal((n, c))
    Z = rng.standard_normal((n, c))
    return H, w, F, Z, dense_incidence(n, m, ptr, mem)


@pytest.mark.parametrize("seed", range(5))
def test_central_differences(seed):
    H, w, F, _, _ = _case(seed)
    mu = 1e-3
    g = weight_grad(H, w, F, mu)
    h = 1e-6
    fd = np.zeros_like(w)
    for e in range(w.size):
        wp, wm = w.copy(), w.copy()
        wp[e] += h
        wm[e] -= h
        fd[e] = (objective(H, wp, F, mu) - objective(H, wm, F, mu)) / (2 * h)
    assert np.allclose(g, fd, rtol=1e-6, atol=1e-8)


def test_dv_frozen_reading_by_differences():
    H, w, F, _, _ = _case(11)
    dv, de, _, _ = degrees(H, w)
    s = 1.0 / np.sqrt(dv)

    def frozen_obj(wx):
        t = wx / de
        G = s[:, None] * F
        return float((F * F).sum() - ((t[:, None] * (H.T @ G) ** 2)).sum())

    g = weight_grad(H, w, F, 0.0, dv_frozen=True)
    h = 1e-6
    fd = np.array([(frozen_obj(w + h * np.eye(w.size)[e]) - frozen_obj(w - h * np.eye(w.size)[e])) / (2 * h)
                   for e in range(w.size)])
    assert np.allclose(g, fd, rtol=1e-6, atol=1e-8)


@pytest.mark.parametrize("seed", range(3))
def test_torch_autograd_dense(seed):
    H, w, F, Z, Hd = _case(20 + seed)
    mu = 0.01
    Ht = torch.tensor(Hd, dtype=torch.float64)
    wt = torch.tensor(w, dtype=torch.float64, requires_grad=True)
    Ft = torch.tensor(F, dtype=torch.float64)
    Zt = torch.tensor(Z, dtype=torch.float64)
    dv = Ht @ wt
    de = Ht.sum(0)
    Sv = torch.diag(dv.rsqrt())
    Th = Sv @ Ht @ torch.diag(wt / de) @ Ht.T @ Sv
    P = (Ft * Ft).sum() - (Ft * (Th @ Ft)).sum() + mu * (wt * wt).sum()
    P.backward()
    assert np.allclose(weight_grad(H, w, F, mu), wt.grad.numpy(), rtol=1e-11, atol=1e-13)
    # bilinear form tr(Z^T Theta F)
    wt2 = torch.tensor(w, dtype=torch.float64, requires_grad=True)
    dv2 = Ht @ wt2
    Sv2 = torch.diag(dv2.rsqrt())
    B = (Zt * ((Sv2 @ Ht @ torch.diag(wt2 / de) @ Ht.T @ Sv2) @ Ft)).sum()
    B.backward()
    assert np.allclose(bilinear_theta_grad(H, w, F, Z), wt2.grad.numpy(), rtol=1e-11, atol=1e-13)


def brute_projection(v):
    best, best_d = None, np.inf
    idx = range(v.size)
    for r in range(1, v.size + 1):
        for S in itertools.combinations(idx, r):
            S = list(S)
            tau = (v[S].sum() - 1.0) / len(S)
            w = np.zeros_like(v)
            w[S] = v[S] - tau
            if np.all(w >= -1e-15):
                d = np.sum((w - v) ** 2)
                if d < best_d:
                    best, best_d = w, d
    return best


@pytest.mark.parametrize("seed", range(8))
def test_projection_brute_force_and_kkt(seed):
    rng = np.random.default_rng(seed)
    v = rng.standard_normal(int(rng.integers(1, 9))) * rng.choice([0.1, 1.0, 5.0])
    w = project_simplex(v)
    assert np.allclose(w, brute_projection(v), atol=1e-14)
    tau = simplex_threshold(v)
    assert abs(w.sum() - 1.0) < 1e-14 and w.min() >= 0
    assert np.allclose(w, np.maximum(v - tau, 0), atol=0)


def test_projection_special_cases():
    w0 = np.array([0.2, 0.3, 0.5])
    assert np.allclose(project_simplex(w0), w0, atol=1e-16)
    assert np.allclose(project_simplex(np.full(4, 3.0)), np.full(4, 0.25))
    assert np.allclose(project_simplex(np.array([10.0, 0.0, -1.0])), [1.0, 0.0, 0.0])


def test_adaptive_loop_descends_objective():
    # at fixed F, a small projected step lowers P(w) (first-order descent)
    rng = np.random.default_rng(1)
    ptr, mem = tiny_hypergraph(rng, 30, 40, 2, 6)
    H = incidence_matrix(build_incidence(30, 40, ptr, mem))
    Y = (rng.random((30, 2)) < 0.2).astype(float)
    w0 = np.full(40, 1.0 / 40)
    F, w, trace = adaptive_loop(H, w0, 1.0, 0.0, 1e-3, Y, 3)
    for tr, wprev in zip(trace, [w0] + [t["w_new"] for t in trace[:-1]]):
        assert objective(H, tr["w_new"], tr["F"], 0.0) <= objective(H, wprev, tr["F"], 0.0) + 1e-15
        assert abs(tr["w_new"].sum() - 1) < 1e-13
    # F is the solve at the w in force before the last update: M F = lam Y, lam = 1
    w_prev = trace[-2]["w_new"]
    assert np.allclose(theta_apply(H, w_prev, F, 2.0, -1.0), Y, atol=1e-8)
    assert np.array_equal(w, trace[-1]["w_new"])


def test_weight_grad_entries_match_the_full_gradient():
    """Entry-by-entry evaluation of the Eq. 4 gradient (for sampled checks at full
    size) against the sparse-product gradient, with a zero-degree vertex."""
    from oracle.core import incidence_lists, weight_grad_entries
    rng = np.random.default_rng(8)
    n, m = 30, 25
    ptr, mem = tiny_hypergraph(rng, n, m, 2, 6)
    H = incidence_matrix(build_incidence(n, m, ptr, mem))
    w = rng.random(m) + 0.1
    w[np.asarray(H[4].nonzero()[1])] = 0.0
    F = rng.standard_normal((n, 4))
    lists = incidence_lists(n, m, ptr, mem)
    edges = np.arange(m)
    g = weight_grad_entries(lists, w, lambda u: F[np.asarray(u)], edges, 1e-3)
    assert np.allclose(g, weight_grad(H, w, F, 1e-3), rtol=1e-12, atol=1e-14)


def test_active_set_step_hand_example():
    """w = (0.5, 0.3, 0.2, 0), g = (1, 0, -1, 5): the pinned fourth weight stays 0, the
    free mean of g is 0.  eta = 0.1: (0.4, 0.3, 0.3, 0), already on the simplex.
    eta = 0.6: (-0.1, 0.3, 0.8, 0) clamps to (0, 0.3, 0.8, 0), sum 1.1, rescaled to
    (0, 3/11, 8/11, 0)."""
    from oracle.core import active_set_step
    w = np.array([0.5, 0.3, 0.2, 0.0])
    g = np.array([1.0, 0.0, -1.0, 5.0])
    assert np.allclose(active_set_step(w, g, 0.1), [0.4, 0.3, 0.3, 0.0], rtol=0, atol=1e-15)
    assert np.allclose(active_set_step(w, g, 0.6), [0.0, 3 / 11, 8 / 11, 0.0], rtol=0, atol=1e-15)
    # nothing free: unchanged
    assert np.array_equal(active_set_step(np.zeros(3), np.ones(3), 1.0), np.zeros(3))


@pytest.mark.parametrize("seed", range(4))
def test_active_set_step_equals_projection_without_clamping(seed):
    """Inside the simplex with a step too small to reach 0, both readings of Eq. 5 give
    w - eta (g - mean g): the active-set step and the Euclidean projection agree."""
    from oracle.core import active_set_step
    rng = np.random.default_rng(seed)
    w = rng.random(50) + 0.5
    w /= w.sum()
    g = rng.standard_normal(50)
    eta = 0.1 * w.min() / np.abs(g).max()
    assert np.allclose(active_set_step(w, g, eta), project_simplex(w - eta * g), rtol=0, atol=1e-15)


@pytest.mark.parametrize("seed", range(4))
def test_active_set_step_feasible_pinned_and_descending(seed):
    from oracle.core import active_set_step
    rng = np.random.default_rng(10 + seed)
    w = rng.random(200)
    w[rng.random(200) < 0.3] = 0.0
    w /= w.sum()
    g = rng.standard_normal(200)
    for eta in (1e-4, 1e-2, 1.0):
        wn = active_set_step(w, g, eta)
        assert wn.min() >= 0.0 and abs(wn.sum() - 1.0) <= 1e-12
        assert (wn[w == 0] == 0).all()
    # first order: the direction is a descent direction of <g, .> on the simplex
    wn = active_set_step(w, g, 1e-6)
    assert g @ (wn - w) < 0
