"""GPU parity of the block randomized SVD (Algorithm 1) and the block preconditioner:
FP64 path against the oracle's Rayleigh-Ritz rSVD with the same Philox Omega, BF16
tensor-core path against the FP64 path, and preconditioned CG against the oracle."""
import numpy as np
import pytest
import torch

import synth
from oracle import core, incidence, rsvd
from paper_1908_08281_gb300 import build as _build
from paper_1908_08281_gb300 import hgl

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    assert torch.cuda.is_available()
    _build.build()
    hgl.lib()


def _setup(n=1500, m=2500, c=4, seed=0, wseed=1):
    wl = synth.WORKLOADS["batched_rsvd"]
    d = synth.make_hypergraph(wl, seed, n=n, m=m, c=c)
    og = incidence.build_incidence(d["n"], d["m"], d["edge_ptr"], d["members"])
    H = incidence.incidence_matrix(og)
    rng = np.random.default_rng(wseed)
    w = rng.random(d["m"]) + 0.05
    w /= w.sum()
    g = hgl.build_incidence(d["n"], d["m"], d["edge_ptr"], d["members"])
    return wl, d, H, w, g


def _panel(a, dtype=torch.float64):
    P = hgl.padded_panel(a.shape[0], a.shape[1], dtype, DEV)
    P.copy_(torch.from_numpy(np.ascontiguousarray(a)).to(dtype))
    return P


K, P_, Q_, SEED = 8, 4, 2, 1234


def _route_used(g, w, bp, k=8):
    """Which products a BF16 build runs: (tcgen05 GEMM launches, sparse product launches)."""
    hgl.profile_enable(True)
    hgl.block_rsvd(g, w, 0.5, bp, k, 4, 1, SEED, gemm_dtype=hgl.HGL_BF16)
    torch.cuda.synchronize()
    used = (hgl.profile_read(hgl.PROF_GEMM)[1], hgl.profile_read(hgl.PROF_BLOCKSPMM)[1])
    hgl.profile_enable(False)
    return used


def test_block_product_route_by_fill():
    """HGL_BLOCKS_AUTO: small hyperedges with random members put few of Theta's entries
    inside large diagonal blocks (sparse route); hyperedges drawn inside one block fill
    them (dense route, the tcgen05 GEMM); the explicit settings override."""
    rng = np.random.default_rng(8)
    n, m = 40000, 60000
    mem = np.sort(np.stack([rng.choice(n, 3, replace=False) for _ in range(m)]), axis=1).ravel()
    g = hgl.build_incidence(n, m, np.arange(0, 3 * m + 1, 3, dtype=np.int64), mem.astype(np.int32))
    wt = torch.full((m,), 1.0 / m, dtype=torch.float64, device=DEV)
    bp = [0, 10000, 20000, 30000, 40000]
    # q = 1: 1 + 2q products in the range finder and one for the Rayleigh-Ritz matrix
    assert _route_used(g, wt, bp) == (0, 4)
    hgl.set_block_product(g, hgl.HGL_BLOCKS_DENSE)
    assert _route_used(g, wt, bp) == (4, 0)
    hgl.set_block_product(g, hgl.HGL_BLOCKS_AUTO)
    # community hypergraph: 4 blocks of 512 vertices, 300 hyperedges of 40 members each
    rng = np.random.default_rng(9)
    n, nbk, size = 2048, 4, 512
    ptr, mem = [0], []
    for e in range(1200):
        b = e % nbk
        mem.extend(sorted(rng.choice(size, 40, replace=False) + b * size))
        ptr.append(len(mem))
    gc = hgl.build_incidence(n, 1200, np.asarray(ptr, np.int64), np.asarray(mem, np.int32))
    wc = torch.full((1200,), 1.0 / 1200, dtype=torch.float64, device=DEV)
    assert _route_used(gc, wc, [0, 512, 1024, 1536, 2048]) == (4, 0)
    with pytest.raises(hgl.HglError):
        hgl.set_block_product(g, 7)


def test_tune_block_rsvd_keeps_the_faster_route():
    """hgl_tune_block_rsvd times both product routes for the blocks and sets the faster
    one: later builds take it, and the factors still match the FP64 route's."""
    rng = np.random.default_rng(17)
    n, m = 40000, 60000
    mem = np.sort(np.stack([rng.choice(n, 3, replace=False) for _ in range(m)]), axis=1).ravel()
    g = hgl.build_incidence(n, m, np.arange(0, 3 * m + 1, 3, dtype=np.int64), mem.astype(np.int32))
    wt = torch.full((m,), 1.0 / m, dtype=torch.float64, device=DEV)
    bp = [0, 10000, 20000, 30000, 40000]
    route, md, ms = hgl.tune_block_rsvd(g, wt, bp, 8, 4, 1)
    assert md > 0 and ms > 0
    assert route == (hgl.HGL_BLOCKS_SPARSE if ms < md else hgl.HGL_BLOCKS_DENSE)
    gemm, spmm = _route_used(g, wt, bp)
    assert (spmm > 0) == (route == hgl.HGL_BLOCKS_SPARSE) and (gemm > 0) == (route == hgl.HGL_BLOCKS_DENSE)
    P16 = hgl.block_rsvd(g, wt, 0.5, bp, 8, 4, 1, SEED, gemm_dtype=hgl.HGL_BF16)
    P64 = hgl.block_rsvd(g, wt, 0.5, bp, 8, 4, 1, SEED, gemm_dtype=hgl.HGL_FP64)
    for b in range(len(bp) - 1):
        e16 = hgl.precond_export(P16, b)[1].cpu().numpy()
        e64 = hgl.precond_export(P64, b)[1].cpu().numpy()
        assert np.abs(e16 - e64).max() <= 3e-2 * e64.max()


def test_rsvd_fp64_matches_oracle():
    wl, d, H, w, g = _setup()
    bp = d["block_ptr"]
    lam = wl.lam
    Pc = hgl.block_rsvd(g, torch.tensor(w, device=DEV), lam, bp, K, P_, Q_, SEED, gemm_dtype=hgl.HGL_FP64)
    fac = rsvd.block_rsvd(H, w, bp, K, P_, Q_, SEED)
    for b in range(len(bp) - 1):
        Qg, evg = hgl.precond_export(Pc, b)
        Qo, evo = fac[b]
        evg = evg.cpu().numpy()
        assert Qg.shape[1] == len(evo)
        assert np.allclose(evg, np.clip(evo, 0, 1), rtol=1e-10, atol=1e-12), (b, evg, evo)
    # the preconditioner itself (invariant under rotations inside eigenspaces)
    rng = np.random.default_rng(3)
    R = rng.standard_normal((d["n"], 5))
    Z = hgl.precond_apply(Pc, _panel(R)).cpu().numpy()
    Zo = rsvd.precond_apply(fac, bp, lam, R)
    assert np.allclose(Z, Zo, rtol=1e-9, atol=1e-10 * np.abs(Zo).max())
    # FP32 panels through the same factors
    Z32 = hgl.precond_apply(Pc, _panel(R, torch.float32)).to(torch.float64).cpu().numpy()
    assert np.abs(Z32 - Zo).max() <= 1e-5 * np.abs(Zo).max()


@pytest.mark.parametrize("route", [hgl.HGL_BLOCKS_DENSE, hgl.HGL_BLOCKS_SPARSE])
@pytest.mark.parametrize("k,p", [(8, 4), (16, 8), (40, 8), (64, 10)])
def test_rsvd_bf16_tensor_cores_vs_fp64(k, p, route):
    """The BF16 path's factors against the FP64 path's (same Omega): dense BF16 blocks on
    the tcgen05 GEMM, or the FP32 products from the incidence lists."""
    wl, d, H, w, g = _setup(n=12000, m=20000, seed=2)
    bp = d["block_ptr"]
    wt = torch.tensor(w, device=DEV)
    P64 = hgl.block_rsvd(g, wt, wl.lam, bp, k, p, Q_, SEED, gemm_dtype=hgl.HGL_FP64)
    hgl.set_block_product(g, route)
    P16 = hgl.block_rsvd(g, wt, wl.lam, bp, k, p, Q_, SEED, gemm_dtype=hgl.HGL_BF16)
    hgl.set_block_product(g, hgl.HGL_BLOCKS_AUTO)
    blocks = rsvd.block_theta(H, w, bp)
    worst = 0.0
    for b in range(len(bp) - 1):
        q64, e64 = hgl.precond_export(P64, b)
        q16, e16 = hgl.precond_export(P16, b)
        e64, e16 = e64.cpu().numpy(), e16.cpu().numpy()
        q64, q16 = q64.cpu().numpy(), q16.cpu().numpy()
        worst = max(worst, np.abs(e64 - e16).max() / max(e64.max(), 1e-12))
        # orthonormal Ritz vectors: FP32 CholeskyQR2 on FP32 products, then FP32 Jacobi
        # rotations (about a thousand per column, each orthogonal to FP32 rounding)
        assert np.abs(q16.T @ q16 - np.eye(q16.shape[1])).max() <= 3e-5
        if b < 8:
            # Ritz residual against the exact FP64 block: BF16 operands cost ~2^-8 relative
            Tb = blocks[b]
            r16 = np.linalg.norm(Tb @ q16 - q16 * e16, axis=0)
            r64 = np.linalg.norm(Tb @ q64 - q64 * e64, axis=0)
            assert (r16 <= r64 + 2e-2 * max(e64.max(), 1e-12)).all(), (b, r16.max(), r64.max())
    # BF16 storage of Theta_bb and of the basis: a few units of 2^-8 in the Ritz values;
    # the sparse route keeps FP32 products
    assert worst <= (3e-2 if route == hgl.HGL_BLOCKS_DENSE else 1e-3), worst
    rng = np.random.default_rng(4)
    Rn = rng.standard_normal((d["n"], 7))
    Z64 = hgl.precond_apply(P64, _panel(Rn)).cpu().numpy()
    for Pc, dt in ((P16, torch.float64), (P16, torch.float32), (P64, torch.float32)):
        Z = hgl.precond_apply(Pc, _panel(Rn, dt)).to(torch.float64).cpu().numpy()
        assert np.isfinite(Z).all()
        # symmetric positive definite: r^T P^-1 r > 0 for every column
        assert ((Rn * Z).sum(axis=0) > 0).all()
        # eigenvectors near the rank cut may trade places between the two factorisations;
        # the operators still agree in norm
        assert np.linalg.norm(Z - Z64) <= 3e-2 * np.linalg.norm(Z64)


def test_pcg_fp32_tensor_core_apply_matches_cuda_core_apply():
    """The FP32 PCG with the tensor-core apply (whose projection also gives r.z) against
    the same solve with the CUDA-core apply: both converge, with iteration counts within
    one of each other, to the same solution within the tolerance's error bound."""
    wl, d, H, w, g = _setup(n=9000, m=15000, c=40, seed=8)
    bp = d["block_ptr"]
    wt = torch.tensor(w, device=DEV)
    Pc = hgl.block_rsvd(g, wt, wl.lam, bp, 64, 10, 2, SEED, gemm_dtype=hgl.HGL_BF16)
    Y = _panel(d["Y"])
    out = {}
    for tc in (True, False):
        assert hgl.precond_tensor_cores(Pc, tc)
        F, relres, iters, st = hgl.cg_solve(g, wt, wl.lam, Y, tol=1e-8, dtype=hgl.HGL_FP32, precond=Pc)
        assert st.relres_max <= 1e-8
        out[tc] = (F.cpu().numpy(), iters.cpu().numpy())
    assert np.abs(out[True][1].astype(int) - out[False][1].astype(int)).max() <= 1
    ref, _ = core.certified_solve(H, w, wl.lam, d["Y"])
    for tc in (True, False):
        err = np.linalg.norm(out[tc][0] - ref, axis=0) / np.linalg.norm(ref, axis=0)
        assert err.max() <= (1 + wl.lam) / wl.lam * 1e-8 * 1.01, (tc, err.max())


def test_pcg_fp64_reaches_oracle_solution():
    wl, d, H, w, g = _setup(n=2000, m=3000, c=6, seed=5)
    bp = d["block_ptr"]
    wt = torch.tensor(w, device=DEV)
    Pc = hgl.block_rsvd(g, wt, wl.lam, bp, K, P_, Q_, SEED, gemm_dtype=hgl.HGL_FP64)
    Y = _panel(d["Y"])
    F, relres, iters, st = hgl.cg_solve(g, wt, wl.lam, Y, tol=1e-10, precond=Pc)
    ref = core.solve_dense(H, w, wl.lam, d["Y"])
    err = np.linalg.norm(F.cpu().numpy() - ref, axis=0) / np.linalg.norm(ref, axis=0)
    assert err.max() <= 1e-10
    fac = rsvd.block_rsvd(H, w, bp, K, P_, Q_, SEED)
    oc = core.cg_solve(H, w, wl.lam, d["Y"], tol=1e-10, precond=lambda R: rsvd.precond_apply(fac, bp, wl.lam, R))
    assert np.abs(iters.cpu().numpy() - oc["iters"]).max() <= 1


@pytest.mark.parametrize("mode", [hgl.HGL_FP32, hgl.HGL_BF16])
def test_pcg_mixed_with_tensor_core_preconditioner(mode):
    wl, d, H, w, g = _setup(n=6000, m=10000, c=16, seed=6)
    bp = d["block_ptr"]
    wt = torch.tensor(w, device=DEV)
    Pc = hgl.block_rsvd(g, wt, wl.lam, bp, 16, 8, 2, SEED, gemm_dtype=hgl.HGL_BF16)
    Y = _panel(d["Y"])
    F, relres, iters, st = hgl.cg_solve(g, wt, wl.lam, Y, tol=1e-8, dtype=mode, precond=Pc)
    ref, _ = core.certified_solve(H, w, wl.lam, d["Y"])
    err = np.linalg.norm(F.cpu().numpy() - ref, axis=0) / np.linalg.norm(ref, axis=0)
    assert err.max() <= 1e-5
    assert st.relres_max <= 1e-8


def test_adaptive_step_br_route_matches_oracle():
    wl, d, H, w, g = _setup(n=1500, m=2500, c=5, seed=7)
    bp = d["block_ptr"]
    wt = torch.tensor(d["w0"], device=DEV)
    Y = _panel(d["Y"])
    F = hgl.padded_panel(d["n"], d["c"])
    for _ in range(2):
        st = hgl.adaptive_step(g, wt, Y, F, wl.lam, 0.0, 1e-2, tol=1e-10, route=hgl.HGL_ROUTE_BR, block_ptr=bp,
                               k=K, p=P_, q=Q_, seed=SEED)
        assert st.solve.relres_max <= 1e-10
    Fr, wr, _ = core.adaptive_loop(H, d["w0"], wl.lam, 0.0, 1e-2, d["Y"], 2, tol=1e-12)
    err = np.linalg.norm(F.cpu().numpy() - Fr, axis=0) / np.linalg.norm(Fr, axis=0)
    assert err.max() <= 1e-9
    assert np.linalg.norm(wt.cpu().numpy() - wr) / np.linalg.norm(wr) <= 1e-9


def test_rsvd_argument_errors():
    wl, d, H, w, g = _setup(n=600, m=900)
    wt = torch.tensor(w, device=DEV)
    for bp, k, p in [([0, 300, 599], 4, 2), ([0, 300, 300, 600], 4, 2), ([0, 600], 90, 10)]:
        with pytest.raises(hgl.HglError) as ei:
            hgl.block_rsvd(g, wt, 0.5, bp, k, p, 1, 1)
        assert ei.value.name == "HGL_ERR_INVALID_ARG"


def test_br_loop_through_weight_collapse_mixed_precision():
    # with mu = 0 the projected step drives w onto a few hyperedges within a few outer
    # iterations; most diagonal blocks then lose rank (isolated vertices have s = 0).
    # Past that point the projection is discontinuous in its input (the support changes
    # at near-ties), so each step is checked against the oracle from the GPU's own w.
    wl, d, H, w, g = _setup(n=6000, m=10000, c=8, seed=9)
    bp = d["block_ptr"]
    wt = torch.tensor(d["w0"], device=DEV)
    Y = _panel(d["Y"])
    F = hgl.padded_panel(d["n"], d["c"])
    eta = 1e-2
    for i in range(6):
        w_before = wt.cpu().numpy().copy()
        st = hgl.adaptive_step(g, wt, Y, F, wl.lam, 0.0, eta, tol=1e-8, dtype=hgl.HGL_FP32,
                               route=hgl.HGL_ROUTE_BR, block_ptr=bp, k=16, p=8, q=2, seed=SEED + i)
        assert st.solve.relres_max <= 1e-8
        Fg = F.cpu().numpy()
        Fr, _ = core.certified_solve(H, w_before, wl.lam, d["Y"])
        err = np.linalg.norm(Fg - Fr, axis=0) / np.linalg.norm(Fr, axis=0)
        assert err.max() <= 1e-5, (i, err.max())
        w_ref = core.project_simplex(w_before - eta * core.weight_grad(H, w_before, Fr, 0.0))
        assert np.linalg.norm(wt.cpu().numpy() - w_ref) <= 1e-4 * np.linalg.norm(w_ref), i
    # the weight mass has concentrated on a handful of hyperedges
    assert torch.topk(wt, 10).values.sum().item() > 0.9


@pytest.mark.parametrize("tc", [True, False])
@pytest.mark.parametrize("k", [64, 20, 18])
@pytest.mark.parametrize("c", [5, 130, 300])
def test_precond_apply_fp32_matches_definition(k, c, tc):
    """Z = R/(1+lam) + sum_b Q_b diag(g_b) Q_b^T R_b (Eq. 15 with the Woodbury gains),
    evaluated in FP64 from the exported factors, against the FP32 apply: blocks that
    start off every 32-row boundary and span several tiles, ragged tiles, ragged column
    chunks.  tc: the TF32 tensor-core apply with split operands (rank padded to 32 or
    64); else k = 64 and k = 20 take the register-tiled CUDA-core kernels, k = 18 the
    generic ones."""
    wl, d, H, w, g = _setup(n=20000, m=33000, seed=5)
    bp = [0, 5000, 8000, 8130, 10179, 14275, 20000]
    lam = wl.lam
    Pc = hgl.block_rsvd(g, torch.tensor(w, device=DEV), lam, bp, k, 8, 1, SEED, gemm_dtype=hgl.HGL_BF16)
    assert hgl.precond_tensor_cores(Pc, tc)
    rng = np.random.default_rng(k + c)
    R32 = _panel(rng.standard_normal((d["n"], c)), torch.float32)
    R = R32.to(torch.float64).cpu().numpy()
    ref = R / (1.0 + lam)
    for b in range(len(bp) - 1):
        Qb, ev = hgl.precond_export(Pc, b)
        Qb, ev = Qb.cpu().numpy(), ev.cpu().numpy()
        gain = ev / ((1.0 + lam) * (1.0 + lam - ev))
        sl = slice(bp[b], bp[b + 1])
        ref[sl] += Qb @ (gain[:, None] * (Qb.T @ R[sl]))
    Z = hgl.precond_apply(Pc, R32).to(torch.float64).cpu().numpy()
    scale = np.linalg.norm(ref, axis=0)
    assert (np.linalg.norm(Z - ref, axis=0) <= 2e-6 * scale).all()
    # reproducible: fixed summation order
    Z2 = hgl.precond_apply(Pc, R32).to(torch.float64).cpu().numpy()
    assert np.array_equal(Z, Z2)


@pytest.mark.parametrize("route,dtype,tol", [(hgl.HGL_ROUTE_BR, hgl.HGL_FP32, 1e-8),
                                             (hgl.HGL_ROUTE_BR, hgl.HGL_FP32, 3e-6),
                                             (hgl.HGL_ROUTE_BR, hgl.HGL_BF16, 3e-6),
                                             (hgl.HGL_ROUTE_CG, hgl.HGL_BF16, 1e-6),
                                             (hgl.HGL_ROUTE_CG, hgl.HGL_FP64, 1e-10)])
def test_captured_step_matches_oracle_each_step(route, dtype, tol):
    """HGL_STEP_GRAPH: the first call runs eagerly, the second captures the step into a
    CUDA graph, later calls replay it.  Every step is checked against the oracle from
    the GPU's own w: the solve (error bound of the tolerance), the projected weights and
    the reported objective and step length."""
    wl, d, H, w, g = _setup(n=6000, m=10000, c=8, seed=12)
    bp = d["block_ptr"]
    mu, eta = 1e-3, 2e-3
    wt = torch.tensor(d["w0"], device=DEV)
    Y = _panel(d["Y"])
    F = hgl.padded_panel(d["n"], d["c"])
    launches = []
    for i in range(5):
        w_before = wt.cpu().numpy().copy()
        l0 = hgl.launch_count()
        st = hgl.adaptive_step(g, wt, Y, F, wl.lam, mu, eta, tol=tol, dtype=dtype, route=route, block_ptr=bp,
                               k=16, p=8, q=2, seed=SEED + i, flags=hgl.HGL_STEP_GRAPH)
        launches.append(hgl.launch_count() - l0)
        assert st.solve.relres_max <= tol, (i, st.solve.relres_max)
        Fg = F.cpu().numpy()
        Fr, _ = core.certified_solve(H, w_before, wl.lam, d["Y"])
        err = np.linalg.norm(Fg - Fr, axis=0) / np.linalg.norm(Fr, axis=0)
        assert err.max() <= (1 + wl.lam) / wl.lam * tol * 1.01 + 1e-13, (i, err.max())
        w_ref = core.project_simplex(w_before - eta * core.weight_grad(H, w_before, Fr, mu))
        w_new = wt.cpu().numpy()
        assert np.linalg.norm(w_new - w_ref) <= 1e-4 * np.linalg.norm(w_ref), i
        assert abs(w_new.sum() - 1.0) <= 1e-12 and w_new.min() >= 0.0
        assert np.isclose(st.objective, core.objective(H, w_before, Fg, mu), rtol=1e-6), i
        assert np.isclose(st.dw_norm, np.linalg.norm(w_new - w_before), rtol=1e-9, atol=1e-15), i
    # replays launch what the capture recorded: the same count every step
    assert launches[2] == launches[3] == launches[4] > 0
    # a different panel (new pointer) starts a new graph without error
    F2 = hgl.padded_panel(d["n"], d["c"])
    F2.copy_(F)
    st = hgl.adaptive_step(g, wt, Y, F2, wl.lam, mu, eta, tol=tol, dtype=dtype, route=route, block_ptr=bp,
                           k=16, p=8, q=2, seed=SEED + 9, flags=hgl.HGL_STEP_GRAPH)
    assert st.solve.relres_max <= tol


def test_captured_step_keeps_block_pattern_and_matches_fresh_build():
    """The captured step's block rSVD keeps the dense blocks' pattern from build to build
    (which members share a block does not depend on w) and clears only the entries it
    wrote: after steps that moved w and zeroed weights, its preconditioner equals a fresh
    build by hgl_block_rsvd (dense route, every row zeroed) at the same w and seed,
    factor for factor and bit for bit (Section 3, Algorithm 1)."""
    wl, d, H, w, g = _setup(n=6000, m=10000, c=8, seed=21)
    hgl.set_block_product(g, hgl.HGL_BLOCKS_DENSE)
    bp = d["block_ptr"]
    k, p, q = 16, 8, 2
    wt = torch.tensor(d["w0"], device=DEV)
    Y = _panel(d["Y"])
    F = hgl.padded_panel(d["n"], d["c"])
    compared = 0
    for i in range(5):
        w_before = wt.clone()
        hgl.adaptive_step(g, wt, Y, F, wl.lam, 1e-3, 5e-3, tol=3e-6, dtype=hgl.HGL_BF16, route=hgl.HGL_ROUTE_BR,
                          block_ptr=bp, k=k, p=p, q=q, seed=SEED + i, flags=hgl.HGL_STEP_GRAPH)
        if i < 2:
            continue  # eager call and capture; later calls replay the graph
        Ps = hgl.step_precond(g, bp, k)
        Pf = hgl.block_rsvd(g, w_before, wl.lam, bp, k, p, q, SEED + i, gemm_dtype=hgl.HGL_BF16)
        for b in range(len(bp) - 1):
            Qs, es = hgl.precond_export(Ps, b)
            Qf, ef = hgl.precond_export(Pf, b)
            assert torch.equal(es, ef), (i, b)
            assert torch.equal(Qs, Qf), (i, b)
        compared += 1
        Pf.close()
    assert compared == 3
    assert int((wt == 0).sum()) > 0  # the steps zeroed weights: entries of the pattern went to 0


@pytest.mark.parametrize("dtype", [hgl.HGL_FP32, hgl.HGL_BF16])
def test_captured_step_reports_fp64_accurate_relres_when_no_sweep_runs(dtype):
    """With eta = 0 the weights stay put, so from the second step on the warm-started F
    already meets tol and the captured solve skips its sweeps; at tol = 3e-6 it starts
    from an FP32 estimate of the residual, and the relres it reports must still be the
    FP64-accurate one (the host's FP64 residual of the returned F)."""
    wl, d, H, w, g = _setup(n=5000, m=8000, c=6, seed=14)
    tol = 3e-6
    wt = torch.tensor(w, device=DEV)
    Y = _panel(d["Y"])
    F = hgl.padded_panel(d["n"], d["c"])
    den = np.linalg.norm(wl.lam * d["Y"], axis=0)
    for i in range(4):
        w_before = wt.cpu().numpy().copy()
        st = hgl.adaptive_step(g, wt, Y, F, wl.lam, 0.0, 0.0, tol=tol, dtype=dtype,
                               route=hgl.HGL_ROUTE_BR, block_ptr=d["block_ptr"], k=16, p=8, q=2,
                               seed=SEED + i, flags=hgl.HGL_STEP_GRAPH)
        R = wl.lam * d["Y"] - core.theta_apply(H, w_before, F.cpu().numpy(), 1.0 + wl.lam, -1.0)
        rel = np.linalg.norm(R, axis=0) / den
        assert rel.max() <= tol and st.solve.relres_max <= tol, (i, rel.max(), st.solve.relres_max)
        assert np.isclose(st.solve.relres_max, rel.max(), rtol=1e-3, atol=1e-13), (i, rel.max(), st.solve.relres_max)
    assert np.allclose(wt.cpu().numpy(), w, rtol=1e-12, atol=0)
