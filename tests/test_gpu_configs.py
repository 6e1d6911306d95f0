"""Parity at the stated sizes of the mixed-CG, batched-rSVD and differentiation
workloads (n = 50k / 120k / 200k), against the oracle at full size where it finishes in
about a minute, else on sampled outputs.

* mixed CG (n = 50,000, m = 80,000, c = 100): BF16 and FP32 panels with FP64-accurate
  refinement to relres 1e-8 (Eq. 6), per-column error against the certified oracle solve.
* batched rSVD (n = 120,000, m = 200,000, 64 blocks of 512..4,096, k = 64, p = 10,
  q = 2, c = 256): the FP64 route against Algorithm 1 on sampled blocks (same Philox
  Omega), the tcgen05 product Theta_bb S element by element against the FP64 product
  at the BF16 rounding bound, the BF16 route's Ritz residuals, and PCG to the certified
  solve (Section 3, Algorithm 1, Eq. 15).
* differentiation (n = 200,000, m = 400,000, c = 256): the adjoint gradient through the
  solve against the oracle's total gradient (sampled entries) and against central
  differences on 50 hyperedges (h = 1e-6, FP64 solves; Eq. 4, Eq. 6).
"""
import numpy as np
import pytest
import torch

import synth
from oracle import core, incidence, philox, rsvd
from paper_1908_08281_gb300 import autograd as hga
from paper_1908_08281_gb300 import build as _build
from paper_1908_08281_gb300 import hgl

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda")
SEED = 5150


@pytest.fixture(scope="module", autouse=True)
def _lib():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    _build.build()
    hgl.lib()


def _panel(a, dtype=torch.float64):
    P = hgl.padded_panel(a.shape[0], a.shape[1], dtype, DEV)
    P.copy_(torch.from_numpy(np.ascontiguousarray(a)).to(dtype))
    return P


def _workload(name, seed):
    wl = synth.WORKLOADS[name]
    d = synth.make_hypergraph(wl, seed)
    H = incidence.incidence_matrix(incidence.build_incidence(d["n"], d["m"], d["edge_ptr"], d["members"]))
    g = hgl.build_incidence(d["n"], d["m"], d["edge_ptr"], d["members"])
    return wl, d, H, g


# ---------------------------------------------------------------------------
# mixed-precision CG at n = 50,000
# ---------------------------------------------------------------------------

@pytest.fixture(scope="module")
def mixed():
    wl, d, H, g = _workload("mixed_cg", 7)
    assert (d["n"], d["m"], d["c"]) == (50000, 80000, 100)
    ref, bound = core.certified_solve(H, d["w0"], wl.lam, d["Y"])
    return wl, d, H, g, ref, bound


@pytest.mark.parametrize("mode", [hgl.HGL_FP32, hgl.HGL_BF16])
def test_mixed_cg_fullsize_error_per_column(mixed, mode):
    """Every tag column within (1+lam)/lam * 1e-8 of the oracle (the tolerance's error
    bound, plus the oracle's own certificate), for BF16 and FP32 panels."""
    wl, d, H, g, ref, bound = mixed
    tol = wl.tol
    F, relres, iters, st = hgl.cg_solve(g, torch.tensor(d["w0"], device=DEV), wl.lam, _panel(d["Y"]), tol=tol,
                                        dtype=mode)
    assert st.relres_max <= tol
    nr = np.linalg.norm(ref, axis=0)
    err = np.linalg.norm(F.cpu().numpy() - ref, axis=0) / nr
    assert err.max() <= (1 + wl.lam) / wl.lam * tol * 1.01 + (bound / nr).max(), err.max()
    # the recomputed residual on the host agrees with the reported one
    R = wl.lam * d["Y"] - core.theta_apply(H, d["w0"], F.cpu().numpy(), 1.0 + wl.lam, -1.0)
    rel = np.linalg.norm(R, axis=0) / np.linalg.norm(wl.lam * d["Y"], axis=0)
    assert rel.max() <= tol * 1.001


# ---------------------------------------------------------------------------
# batched block rSVD at n = 120,000 (64 blocks of 512..4,096, k = 64, p = 10, q = 2)
# ---------------------------------------------------------------------------

@pytest.fixture(scope="module")
def batched():
    wl, d, H, g = _workload("batched_rsvd", 8)
    assert (d["n"], d["m"], d["c"]) == (120000, 200000, 256)
    bp = np.asarray(d["block_ptr"], dtype=np.int64)
    sizes = np.diff(bp)
    assert len(sizes) == 64 and sizes.min() >= 512 and sizes.max() <= 4096
    rng = np.random.default_rng(12)
    w = rng.random(d["m"]) + 0.05
    w /= w.sum()
    # sampled blocks: the largest, the smallest and the first
    pick = sorted({int(np.argmax(sizes)), int(np.argmin(sizes)), 0})
    return wl, d, H, g, bp, w, pick


_BLOCKS = {}


def _oracle_block(H, w, bp, b, k, p, q, seed):
    """The oracle's dense Theta_bb and its Rayleigh-Ritz Algorithm 1 (cached per block)."""
    key = (b, k, p, q, seed)
    if key not in _BLOCKS:
        _BLOCKS[key] = _oracle_block_uncached(H, w, bp, b, k, p, q, seed)
    return _BLOCKS[key]


def _oracle_block_uncached(H, w, bp, b, k, p, q, seed):
    b0, b1 = int(bp[b]), int(bp[b + 1])
    Tb = rsvd.block_theta(H, w, [b0, b1])[0]
    Om = philox.omega(np.arange(b0, b1), k + p, seed)[:, :min(k + p, b1 - b0)]
    Q, ev = rsvd.rsvd_ritz(Tb, Om, q, min(k, b1 - b0))
    return Tb, Q, ev


def test_batched_rsvd_fp64_route_matches_algorithm1_on_sampled_blocks(batched):
    """FP64 route (CUDA cores, FP64 CholeskyQR2 and Jacobi) against the oracle's
    Rayleigh-Ritz Algorithm 1 with the same Philox Omega: Ritz values to 1e-10, and the
    block's low-rank part Q diag(g) Q^T applied to random vectors to 1e-9 (invariant
    under rotations inside clusters of equal Ritz values)."""
    wl, d, H, g, bp, w, pick = batched
    k, p, q = wl.k, wl.p, wl.q
    Pc = hgl.block_rsvd(g, torch.tensor(w, device=DEV), wl.lam, bp, k, p, q, SEED, gemm_dtype=hgl.HGL_FP64)
    rng = np.random.default_rng(1)
    for b in pick:
        Tb, Qo, evo = _oracle_block(H, w, bp, b, k, p, q, SEED)
        Qg, evg = hgl.precond_export(Pc, b)
        Qg, evg = Qg.cpu().numpy(), evg.cpu().numpy()
        assert Qg.shape == Qo.shape
        assert np.allclose(evg, np.clip(evo, 0, None), rtol=1e-10, atol=1e-12 * evo.max()), b
        gain = lambda ev: ev / ((1 + wl.lam) * (1 + wl.lam - ev))
        R = rng.standard_normal((Tb.shape[0], 3))
        Zg = Qg @ (gain(evg)[:, None] * (Qg.T @ R))
        Zo = Qo @ (gain(np.clip(evo, 0, None))[:, None] * (Qo.T @ R))
        assert np.abs(Zg - Zo).max() <= 1e-9 * np.abs(Zo).max(), b


@pytest.mark.parametrize("route", [hgl.HGL_BLOCKS_DENSE, hgl.HGL_BLOCKS_SPARSE])
def test_batched_block_product_elementwise(batched, route):
    """One product of Algorithm 1, D_b = Theta_bb S_b for all 64 blocks in one launch,
    element by element on the sampled blocks against the oracle's FP64 product.
    Dense route (tcgen05, BF16 operands, FP32 accumulation in TMEM): each entry of
    Theta_bb and S is rounded to BF16 (relative error < 2^-8 each), Theta_bb's entries are
    first summed in FP32 from FP32 copies of s and t (< 64 * 2^-24), and the K-term sums
    accumulate in FP32 (< K * 2^-23), so
        |D - D_exact| <= (2^-7 + 2^-16 + 64 * 2^-24 + K * 2^-23) (|Theta_bb| |S|).
    Sparse route (FP32 products from the incidence lists): (64 + K) * 2^-23 (|Theta||S|)."""
    wl, d, H, g, bp, w, pick = batched
    l = wl.k + wl.p
    rng = np.random.default_rng(3)
    S = rng.standard_normal((d["n"], l)).astype(np.float32)
    hgl.set_block_product(g, route)
    try:
        D = hgl.block_product(g, torch.tensor(w, device=DEV), bp, torch.from_numpy(S).to(DEV)).cpu().numpy()
    finally:
        hgl.set_block_product(g, hgl.HGL_BLOCKS_AUTO)
    for b in pick:
        b0, b1 = int(bp[b]), int(bp[b + 1])
        K = b1 - b0
        Tb = rsvd.block_theta(H, w, [b0, b1])[0]
        Sb = S[b0:b1].astype(np.float64)
        exact = Tb @ Sb
        mag = np.abs(Tb) @ np.abs(Sb)
        if route == hgl.HGL_BLOCKS_DENSE:
            rel = 2.0 ** -7 + 2.0 ** -16 + 64 * 2.0 ** -24 + K * 2.0 ** -23
        else:
            rel = (64 + K) * 2.0 ** -23
        err = np.abs(D[b0:b1] - exact)
        assert (err <= rel * mag + 1e-30).all(), (b, (err / np.maximum(mag, 1e-300)).max(), rel)
        # and the bound is not vacuous: the typical error sits well inside it
        assert np.median(err / np.maximum(mag, 1e-300)) < 0.25 * rel


def test_batched_rsvd_bf16_route_on_sampled_blocks(batched):
    """The BF16 tensor-core route (the bench's build): orthonormal Ritz vectors, Ritz
    values within a few units of 2^-8 of the oracle's, and Ritz residuals against the
    exact FP64 block no worse than the oracle's own plus the BF16 operand rounding."""
    wl, d, H, g, bp, w, pick = batched
    k, p, q = wl.k, wl.p, wl.q
    Pc = hgl.block_rsvd(g, torch.tensor(w, device=DEV), wl.lam, bp, k, p, q, SEED, gemm_dtype=hgl.HGL_BF16)
    for b in pick:
        Tb, Qo, evo = _oracle_block(H, w, bp, b, k, p, q, SEED)
        q16, e16 = hgl.precond_export(Pc, b)
        q16, e16 = q16.cpu().numpy(), e16.cpu().numpy()
        assert np.abs(q16.T @ q16 - np.eye(q16.shape[1])).max() <= 3e-5
        assert np.abs(e16 - np.clip(evo, 0, None)).max() <= 3e-2 * evo.max(), b
        r16 = np.linalg.norm(Tb @ q16 - q16 * e16, axis=0)
        ro = np.linalg.norm(Tb @ Qo - Qo * evo, axis=0)
        assert (r16 <= ro + 2e-2 * evo.max()).all(), (b, r16.max(), ro.max())


def test_batched_pcg_reaches_certified_solve(batched):
    """PCG with the BF16-built block preconditioner, FP32 panels and FP64-accurate
    refinement, all 256 columns, to relres 1e-8: every column within the tolerance's
    error bound of the oracle's certified FP64 solve."""
    wl, d, H, g, bp, w, pick = batched
    wt = torch.tensor(w, device=DEV)
    Pc = hgl.block_rsvd(g, wt, wl.lam, bp, wl.k, wl.p, wl.q, SEED, gemm_dtype=hgl.HGL_BF16)
    F, relres, iters, st = hgl.cg_solve(g, wt, wl.lam, _panel(d["Y"]), tol=1e-8, dtype=hgl.HGL_FP32, precond=Pc)
    assert st.relres_max <= 1e-8
    ref, bound = core.certified_solve(H, w, wl.lam, d["Y"])
    nr = np.linalg.norm(ref, axis=0)
    err = np.linalg.norm(F.cpu().numpy() - ref, axis=0) / nr
    assert err.max() <= (1 + wl.lam) / wl.lam * 1e-8 * 1.01 + (bound / nr).max(), err.max()


# ---------------------------------------------------------------------------
# differentiation at n = 200,000 (m = 400,000, c = 256, lam = 1, mu = 1e-3)
# ---------------------------------------------------------------------------

@pytest.fixture(scope="module")
def adjoint():
    wl, d, H, g = _workload("adjoint", 9)
    assert (d["n"], d["m"], d["c"]) == (200000, 400000, 256)
    rng = np.random.default_rng(21)
    # weights of order one: Theta is invariant under scaling w, and unit-size weights
    # keep the central differences' step h = 1e-6 a small relative perturbation
    w = rng.random(d["m"]) + 0.5
    rows = rng.choice(d["n"], size=d["n"] // 5, replace=False)
    Yt = rng.random((rows.size, d["c"]))
    F, _ = core.certified_solve(H, w, wl.lam, d["Y"])
    edges = rng.choice(d["m"], size=50, replace=False)
    return wl, d, H, g, w, rows, Yt, F, edges


def _fixed_solve(g, w, lam, Y, iters=40):
    """FP64 CG with a fixed iteration count: at lam = 1, kappa(M) <= 2, so 40 iterations
    take the error ~0.172^40 below rounding, and the solution is the same polynomial in
    M(w) for every w (central differences then see no change of iteration count)."""
    F, _, _, st = hgl.cg_solve(g, w, lam, Y, tol=1e-300, max_iter=iters, raise_on_fail=False)
    assert st.relres_max <= 1e-13
    return F


def _fd(loss_of_w, w, edges, h=1e-6):
    out, mags = [], []
    for e in edges:
        wp, wm = w.clone(), w.clone()
        wp[e] += h
        wm[e] -= h
        lp, lm = loss_of_w(wp), loss_of_w(wm)
        out.append((lp - lm) / (2 * h))
        mags.append(max(abs(lp), abs(lm)))
    return np.array(out), max(mags)


def test_adjoint_heldout_gradient_fullsize(adjoint):
    """L = ||F(w)[rows] - Y_test||^2 (its adjoint right-hand side does not vanish): the
    torch.autograd gradient through hgl_adjoint_grad against the oracle's total gradient
    (sampled entries, 1e-8 of max|g|) and against central differences on 50 hyperedges
    (h = 1e-6; their error is the FP64 rounding of L over 2h, |L| 2^-52 / h, plus
    1e-5 of max|g|)."""
    wl, d, H, g, w, rows, Yt, Fo, edges = adjoint
    lam = wl.lam
    Y = _panel(d["Y"])
    rows_t = torch.tensor(rows, device=DEV)
    Yt_t = torch.tensor(Yt, device=DEV)
    wt = torch.tensor(w, device=DEV, requires_grad=True)
    F = hga.solve(g, wt, Y, lam, tol=1e-13)
    L = ((F[rows_t] - Yt_t) ** 2).sum()
    L.backward()
    gpu = wt.grad.cpu().numpy()
    Lo, Fo2, dF, dw = core.heldout_loss(H, w, d["Y"], lam, rows, Yt, F=Fo)
    adj, _ = core.solve_grad_w(H, w, lam, Fo, dF, dense=False)
    ref = dw + adj
    sample = np.random.default_rng(5).choice(d["m"], size=2000, replace=False)
    assert np.isclose(float(L.detach()), Lo, rtol=1e-10)
    assert np.abs(gpu[sample] - ref[sample]).max() <= 1e-8 * np.abs(ref).max()
    w0 = torch.tensor(w, device=DEV)
    fd, lmag = _fd(lambda ww: float(((_fixed_solve(g, ww, lam, Y)[rows_t] - Yt_t) ** 2).sum()), w0, edges)
    assert np.abs(gpu[edges] - fd).max() <= 1e-5 * np.abs(ref).max() + 4 * lmag * 2.0 ** -52 / 1e-6


def test_adjoint_regularised_loss_gradient_fullsize(adjoint):
    """L = tr(F^T Delta F) + lam ||F - Y||^2 + mu ||w||^2 with mu = 1e-3: stationary in F
    at the solution, so its gradient is the explicit one (Eq. 4 at fixed F plus 2 mu w);
    the autograd gradient against the oracle's (sampled entries) and against central
    differences on 50 hyperedges (the F error enters L only quadratically here)."""
    wl, d, H, g, w, rows, Yt, Fo, edges = adjoint
    lam, mu = wl.lam, wl.mu
    Y = _panel(d["Y"])
    wt = torch.tensor(w, device=DEV, requires_grad=True)
    F = hga.solve(g, wt, Y, lam, tol=1e-13)
    L = hga.laplacian_quadratic(g, wt, F) + lam * ((F - Y) ** 2).sum() + mu * (wt * wt).sum()
    L.backward()
    gpu = wt.grad.cpu().numpy()
    ref = core.weight_grad(H, w, Fo, mu)
    sample = np.random.default_rng(6).choice(d["m"], size=2000, replace=False)
    assert np.isclose(float(L.detach()), core.full_loss(H, w, Fo, d["Y"], lam, mu), rtol=1e-10)
    assert np.abs(gpu[sample] - ref[sample]).max() <= 1e-8 * np.abs(ref).max()

    # central differences from the per-entry differences of L's terms at w + h e and
    # w - h e (summing the small differences, not subtracting two sums of ~5e7 terms
    # whose tree-summation rounding, ~26 eps |L|, would swamp the quotient): the
    # rounding left is at most eps (sum |t+| + sum |t-|) / 2h
    def terms(ww):
        Fw = _fixed_solve(g, ww, lam, Y)
        _, DF = hgl.laplacian_quadratic(g, ww, Fw)
        return Fw * DF + lam * (Fw - Y) ** 2

    h = 1e-6
    w0 = torch.tensor(w, device=DEV)
    fd, err_bound = [], []
    for e in edges:
        wp, wm = w0.clone(), w0.clone()
        wp[e] += h
        wm[e] -= h
        tp, tm = terms(wp), terms(wm)
        diff = float((tp - tm).sum()) + mu * float((wp[e] ** 2 - wm[e] ** 2))
        fd.append(diff / (2 * h))
        err_bound.append(2.0 ** -52 * float(tp.abs().sum() + tm.abs().sum()) / (2 * h))
    fd = np.array(fd)
    assert (np.abs(gpu[edges] - fd) <= 1e-5 * np.abs(ref).max() + np.array(err_bound)).all(), \
        (np.abs(gpu[edges] - fd).max(), max(err_bound))
