"""Parity at the full adaptive workload (n = 1,000,000, m = 2,000,000, c = 512) in the
launch configuration the bench times: FP32 panels with 128-column chunks, the block
rSVD route with k = 64, p = 10, q = 2, one captured CUDA graph per outer iteration.
Outputs the oracle can compute one by one are sampled (incidence lists, operator rows,
gradient entries, block factors); the rest is checked through properties that hold at
any size (residual recomputed in FP64 on the host for sampled columns, the projection's
optimality conditions)."""
import numpy as np
import pytest
import torch

import synth
from oracle import core, incidence, rsvd
from paper_1908_08281_gb300 import build as _build
from paper_1908_08281_gb300 import hgl

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda")
SEED = 20190822           # the bench's seed
TOL = 3e-6                # the bench's relative residual
K, P_, Q_ = 64, 10, 2


@pytest.fixture(scope="module")
def full():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    _build.build()
    hgl.lib()
    wl = synth.WORKLOADS["full_adaptive"]
    d = synth.make_hypergraph(wl, SEED, tags_dtype=np.float64)
    g = hgl.build_incidence(d["n"], d["m"], d["edge_ptr"], d["members"])
    lists = core.incidence_lists(d["n"], d["m"], d["edge_ptr"], d["members"])
    bp = d["block_ptr"]
    return wl, d, g, lists, bp


def test_fullsize_incidence_sampled_bit_exact(full):
    wl, d, g, lists, bp = full
    n, m = d["n"], d["m"]
    ex = hgl.graph_export(g)
    edge_ptr, members, vert_ptr, vert_edges = lists
    assert np.array_equal(ex["de"].cpu().numpy(), np.diff(edge_ptr))
    assert np.array_equal(ex["csc_ptr"].cpu().numpy(), edge_ptr)
    assert np.array_equal(ex["csr_ptr"].cpu().numpy(), vert_ptr)
    rng = np.random.default_rng(1)
    ci, ri = ex["csc_idx"].cpu().numpy(), ex["csr_idx"].cpu().numpy()
    for e in rng.choice(m, 2000, replace=False):
        assert np.array_equal(ci[edge_ptr[e]:edge_ptr[e + 1]], np.sort(members[edge_ptr[e]:edge_ptr[e + 1]]))
    for v in rng.choice(n, 2000, replace=False):
        assert np.array_equal(ri[vert_ptr[v]:vert_ptr[v + 1]], vert_edges[vert_ptr[v]:vert_ptr[v + 1]])


def test_fullsize_operator_sampled_rows(full):
    """Z = (1+lam) X - Theta X on FP32 panels (the CG's operator), 128-column chunks:
    64 sampled rows against the row-by-row oracle on the same FP32 inputs."""
    wl, d, g, lists, bp = full
    n, m, c = d["n"], d["m"], d["c"]
    gen = torch.Generator(device=DEV).manual_seed(7)
    X = hgl.padded_panel(n, c, torch.float32, DEV)
    X.copy_(torch.randn(n, c, device=DEV, generator=gen))
    w = d["w0"] * (0.5 + np.random.default_rng(2).random(m))
    wt = torch.tensor(w, device=DEV)
    Z = hgl.apply_theta(g, wt, X, 1.0 + wl.lam, -1.0)
    rows = np.random.default_rng(3).choice(n, 64, replace=False)
    Xrows = lambda u: X[torch.as_tensor(np.asarray(u), device=DEV)].double().cpu().numpy()
    ref = core.theta_rows(lists, w, Xrows, rows, 1.0 + wl.lam, -1.0)
    absX = core.theta_rows(lists, w, lambda u: np.abs(Xrows(u)), rows, 0.0, 1.0)
    got = Z[torch.as_tensor(rows, device=DEV)].double().cpu().numpy()
    scale = np.abs(ref) + (1.0 + wl.lam) * np.abs(Xrows(rows)) + absX
    assert (np.abs(got - ref) <= 2e-6 * scale + 1e-30).all()


def test_fullsize_captured_steps(full):
    """Two outer iterations as the bench runs them (the first eager, the second captured
    and replayed), then a replay: reported and host-recomputed residuals, gradient
    entries, the projection's optimality conditions, the block factors."""
    wl, d, g, lists, bp = full
    n, m, c = d["n"], d["m"], d["c"]
    eta = wl.eta
    Y = hgl.padded_panel(n, c, torch.float64, DEV)
    Y.copy_(torch.from_numpy(d["Y"]))
    w = torch.tensor(d["w0"], device=DEV)
    F = hgl.padded_panel(n, c, torch.float64, DEV)
    for i in range(3):
        w_before = w.clone()
        st = hgl.adaptive_step(g, w, Y, F, lam=wl.lam, mu=wl.mu, eta=eta, tol=TOL, dtype=hgl.HGL_FP32,
                               route=hgl.HGL_ROUTE_BR, block_ptr=bp, k=K, p=P_, q=Q_, seed=SEED + i,
                               flags=hgl.HGL_STEP_GRAPH)
        assert st.solve.relres_max <= TOL, (i, st.solve.relres_max)
    wb = w_before.cpu().numpy()
    # the residual of two sampled columns, recomputed on the host in FP64
    H = incidence.incidence_matrix(incidence.build_incidence(n, m, d["edge_ptr"], d["members"]))
    cols = [0, 311]
    Fc = F[:, cols].cpu().numpy()
    R = wl.lam * d["Y"][:, cols] - core.theta_apply(H, wb, Fc, 1.0 + wl.lam, -1.0)
    rel = np.linalg.norm(R, axis=0) / np.linalg.norm(wl.lam * d["Y"][:, cols], axis=0)
    assert (rel <= TOL * 1.01).all(), rel
    # gradient entries at the step's F (FP64 panel) against the entry-by-entry oracle
    grad = hgl.weight_grad(g, w_before, F, wl.mu).cpu().numpy()
    sizes = np.diff(lists[0])
    edges = np.random.default_rng(4).choice(np.flatnonzero(sizes <= 40), 24, replace=False)
    Frows = lambda u: F[torch.as_tensor(np.asarray(u), device=DEV)].cpu().numpy()
    ref = core.weight_grad_entries(lists, wb, Frows, edges, wl.mu)
    assert np.abs(grad[edges] - ref).max() <= 1e-9 * np.abs(grad).max()
    # the projected step: w = max(v - tau, 0), sum w = 1, with v = w_before - eta grad
    wn = w.cpu().numpy()
    assert wn.min() >= 0.0 and abs(wn.sum() - 1.0) <= 1e-12
    w_ref = core.project_simplex(wb - eta * grad)
    assert np.linalg.norm(wn - w_ref) <= 1e-6 * np.linalg.norm(w_ref)
    # block factors at w_before: the smallest block against Algorithm 1 in the oracle, on
    # the route the loop takes (dense tcgen05 GEMM: these blocks hold 0.8% of their dense
    # size, above the sparse route's 1/512) and on the sparse route
    b = int(np.argmin(np.diff(np.asarray(bp))))
    Qo, evo = rsvd.block_rsvd(H, wb, [bp[b], bp[b + 1]], K, P_, Q_, SEED)[0]
    for route, tol_ev in ((hgl.HGL_BLOCKS_AUTO, 3e-2), (hgl.HGL_BLOCKS_SPARSE, 1e-3)):
        hgl.set_block_product(g, route)
        Pc = hgl.block_rsvd(g, w_before, wl.lam, bp, K, P_, Q_, SEED, gemm_dtype=hgl.HGL_BF16)
        Qg, evg = hgl.precond_export(Pc, b)
        Qg, evg = Qg.cpu().numpy(), evg.cpu().numpy()
        assert np.abs(Qg.T @ Qg - np.eye(Qg.shape[1])).max() <= 3e-5
        assert np.abs(evg - np.clip(evo, 0, 1)).max() <= tol_ev * max(evo.max(), 1e-12), route
    # the preconditioner on the block's rows against its definition from the factors
    R32 = hgl.padded_panel(n, c, torch.float32, DEV)
    R32.copy_(torch.randn(n, c, device=DEV, generator=torch.Generator(device=DEV).manual_seed(5)))
    Z = hgl.precond_apply(Pc, R32)
    Rb = R32[bp[b]:bp[b + 1]].double().cpu().numpy()
    gain = evg / ((1.0 + wl.lam) * (1.0 + wl.lam - evg))
    zref = Rb / (1.0 + wl.lam) + Qg @ (gain[:, None] * (Qg.T @ Rb))
    zg = Z[bp[b]:bp[b + 1]].double().cpu().numpy()
    assert (np.linalg.norm(zg - zref, axis=0) <= 2e-6 * np.linalg.norm(zref, axis=0)).all()
