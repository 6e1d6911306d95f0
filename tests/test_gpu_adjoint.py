"""The adjoint gradient through the ranking solve on the GPU (hgl_adjoint_grad and the
torch.autograd wrappers) against the oracle and against central differences."""
import numpy as np
import pytest
import torch

import synth
from oracle import core, incidence
from paper_1908_08281_gb300 import autograd as hga
from paper_1908_08281_gb300 import build as _build
from paper_1908_08281_gb300 import hgl

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    _build.build()
    hgl.lib()


def _case(seed, n=3000, m=6000, c=6):
    """The differentiation workload's size laws at a reduced size; w of order 1 (the
    loss is invariant under scaling w, so no normalisation is needed)."""
    wl = synth.WORKLOADS["adjoint"]
    d = synth.make_hypergraph(wl, seed, n=n, m=m, c=c)
    H = incidence.incidence_matrix(incidence.build_incidence(d["n"], d["m"], d["edge_ptr"], d["members"]))
    rng = np.random.default_rng(seed + 100)
    w = rng.random(d["m"]) + 0.5
    g = hgl.build_incidence(d["n"], d["m"], d["edge_ptr"], d["members"])
    rows = rng.choice(d["n"], size=d["n"] // 5, replace=False)
    Yt = rng.random((rows.size, c))
    return wl, d, H, w, g, rows, Yt


def _panel(a, dtype=torch.float64):
    P = hgl.padded_panel(a.shape[0], a.shape[1], dtype, DEV)
    P.copy_(torch.from_numpy(np.ascontiguousarray(a)).to(dtype))
    return P


@pytest.mark.parametrize("mode,tol,rtol", [(hgl.HGL_FP64, 1e-12, 1e-9), (hgl.HGL_FP32, 1e-8, 1e-5)])
def test_adjoint_grad_matches_oracle(mode, tol, rtol):
    wl, d, H, w, g, _, _ = _case(1)
    lam = wl.lam
    wt = torch.tensor(w, device=DEV)
    F, _, _, _ = hgl.cg_solve(g, wt, lam, _panel(d["Y"]), tol=1e-13)
    G = np.random.default_rng(7).standard_normal((d["n"], d["c"]))
    grad, Z, st = hgl.adjoint_grad(g, wt, lam, F, _panel(G), tol=tol, dtype=mode)
    assert st.relres_max <= tol
    Fc = F.cpu().numpy()
    ref, Zref = core.solve_grad_w(H, w, lam, Fc, G, dense=False)
    zerr = np.linalg.norm(Z.cpu().numpy() - Zref, axis=0) / np.linalg.norm(Zref, axis=0)
    assert zerr.max() <= (1 + lam) / lam * tol * 1.01 + 1e-13
    gg = grad.cpu().numpy()
    assert np.abs(gg - ref).max() <= rtol * np.abs(ref).max()


def _fd(loss_of_w, w, edges, h=1e-6):
    out = []
    for e in edges:
        wp, wm = w.clone(), w.clone()
        wp[e] += h
        wm[e] -= h
        out.append((loss_of_w(wp) - loss_of_w(wm)) / (2 * h))
    return np.array(out)


def _gpu_loss(g, Y, lam, kind, mu, rows_t, Yt_t, w, tol=1e-14):
    """The loss through the library's FP64 solve (no autograd)."""
    F, _, _, st = hgl.cg_solve(g, w, lam, Y, tol=tol, max_iter=400, raise_on_fail=False)
    assert st.relres_max <= 1e-13
    if kind == "zhou":
        DF = hgl.apply_theta(g, w, F, 1.0, -1.0)
        return float((F * DF).sum() + lam * ((F - Y) ** 2).sum() + mu * (w * w).sum())
    return float(((F[rows_t] - Yt_t) ** 2).sum())


@pytest.mark.parametrize("kind", ["zhou", "heldout"])
def test_autograd_gradient_vs_oracle_and_central_differences(kind):
    wl, d, H, w, g, rows, Yt = _case(2, n=2000, m=4000, c=4)
    lam, mu = wl.lam, wl.mu
    Y = _panel(d["Y"])
    rows_t = torch.tensor(rows, device=DEV)
    Yt_t = torch.tensor(Yt, device=DEV)
    wt = torch.tensor(w, device=DEV, requires_grad=True)
    F = hga.solve(g, wt, Y, lam, tol=1e-13)
    if kind == "zhou":
        L = hga.laplacian_quadratic(g, wt, F) + lam * ((F - Y) ** 2).sum() + mu * (wt * wt).sum()
    else:
        L = ((F[rows_t] - Yt_t) ** 2).sum()
    L.backward()
    gpu = wt.grad.cpu().numpy()
    # the oracle's adjoint gradient (certified CG solves)
    if kind == "zhou":
        Lo, ref, _, _ = core.total_grad(H, w, d["Y"], lam, core.zhou_loss, dense=False,
                                        mu=mu, F=core.certified_solve(H, w, lam, d["Y"])[0])
    else:
        Lo, ref, _, _ = core.total_grad(H, w, d["Y"], lam, core.heldout_loss, dense=False, rows=rows,
                                        Y_test=Yt, F=core.certified_solve(H, w, lam, d["Y"])[0])
    assert np.isclose(float(L.detach()), Lo, rtol=1e-10)
    assert np.abs(gpu - ref).max() <= 1e-8 * np.abs(ref).max()
    # central differences of the loss on 50 random hyperedges (h = 1e-6, FP64 solves)
    edges = np.random.default_rng(3).choice(d["m"], size=50, replace=False)
    w0 = torch.tensor(w, device=DEV)
    fd = _fd(lambda ww: _gpu_loss(g, Y, lam, kind, mu, rows_t, Yt_t, ww), w0, edges)
    # FD error: roundoff |L| eps / h plus solve noise at relres ~1e-14, about 1e-5 of max|g| here
    assert np.abs(gpu[edges] - fd).max() <= 1e-4 * np.abs(ref).max()


def test_heldout_gradient_is_orthogonal_to_w():
    """Theta(alpha w) = Theta(w): a loss that sees w only through F has w^T dL/dw = 0."""
    wl, d, H, w, g, rows, Yt = _case(3, n=2000, m=4000, c=3)
    Y = _panel(d["Y"])
    wt = torch.tensor(w, device=DEV, requires_grad=True)
    F = hga.solve(g, wt, Y, wl.lam, tol=1e-13)
    L = ((F[torch.tensor(rows, device=DEV)] - torch.tensor(Yt, device=DEV)) ** 2).sum()
    L.backward()
    gr = wt.grad
    assert abs(float((gr * wt.detach()).sum())) <= 1e-9 * float(gr.abs().max() * wt.detach().abs().sum())


def test_adjoint_grad_argument_errors():
    wl, d, H, w, g, _, _ = _case(4, n=500, m=800, c=2)
    wt = torch.tensor(w, device=DEV)
    F = _panel(np.ones((d["n"], 2)))
    with pytest.raises(hgl.HglError):
        hgl.adjoint_grad(g, wt, -1.0, F, _panel(np.ones((d["n"], 2))))
    with pytest.raises(hgl.HglError):
        hgl.adjoint_grad(g, wt, wl.lam, F, F, Z=F)


def test_laplacian_quadratic_matches_oracle():
    """hgl_laplacian_quadratic: tr(F^T Delta F) against the oracle's objective at mu = 0
    (Eq. 4), and Delta F element-wise against the oracle's operator apply (Eq. 1), on a
    ragged column count; the trace of a panel of sqrt(dv) columns vanishes (Delta
    annihilates Dv^1/2 1)."""
    wl, d, H, w, g, _, _ = _case(3, c=7)
    wt = torch.tensor(w, device=DEV)
    F = np.random.default_rng(11).standard_normal((d["n"], d["c"]))
    val, DF = hgl.laplacian_quadratic(g, wt, _panel(F))
    ref = core.objective(H, w, F, 0.0)
    assert abs(val - ref) <= 1e-12 * abs(ref)
    DFr = core.theta_apply(H, w, F, 1.0, -1.0)
    assert np.abs(DF.cpu().numpy() - DFr).max() <= 1e-13 * np.abs(DFr).max()
    dv = np.asarray(H @ w).ravel()
    S = np.repeat(np.sqrt(dv)[:, None], 2, axis=1)
    v0, _ = hgl.laplacian_quadratic(g, wt, _panel(S))
    assert abs(v0) <= 1e-12 * float((S * S).sum())
