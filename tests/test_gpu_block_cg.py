"""GPU parity of the block CG with a shared Krylov space (hgl_block_cg_solve, FP64)
against the oracle's block_cg_solve and the dense solve."""
import numpy as np
import pytest
import torch

import synth
from oracle.core import adaptive_loop, block_cg_solve, cg_solve, solve_dense
from oracle.incidence import build_incidence, incidence_matrix
from paper_1908_08281_gb300 import build as _build
from paper_1908_08281_gb300 import hgl

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    _build.build()
    hgl.lib()


def _panel(a):
    P = hgl.padded_panel(a.shape[0], a.shape[1], torch.float64, DEV)
    P.copy_(torch.from_numpy(np.ascontiguousarray(a)))
    return P


def _graph(n, m, ptr, mem):
    H = incidence_matrix(build_incidence(n, m, np.asarray(ptr, np.int64), np.asarray(mem, np.int32)))
    g = hgl.build_incidence(n, m, np.asarray(ptr, np.int64), np.asarray(mem, np.int32))
    return H, g


def _spd_case(n=24, m=40, c=6, seed=3):
    rng = np.random.default_rng(seed)
    ptr, mem = [0], []
    for _ in range(m):
        k = int(rng.integers(2, 7))
        mem.extend(sorted(rng.choice(n, k, replace=False)))
        ptr.append(len(mem))
    H, g = _graph(n, m, ptr, mem)
    w = rng.random(m) + 0.1
    w /= w.sum()
    return H, g, w, rng.standard_normal((n, c))


@pytest.mark.parametrize("s", [4, 3, 10, 1])
def test_block_cg_matches_oracle(s):
    """Groups of s columns (ragged last group for s = 3, 4; one group for s = 10; plain
    CG for s = 1): the same iteration counts as the oracle's block CG (up to one), and
    the solution within the tolerance's error bound of the dense solve."""
    wl = synth.WORKLOADS["small_fp64"]
    d = synth.make_hypergraph(wl, 11)
    H, g = _graph(d["n"], d["m"], d["edge_ptr"], d["members"])
    rng = np.random.default_rng(5)
    w = rng.random(d["m"]) + 0.2
    w /= w.sum()
    tol = 1e-10
    F, relres, iters, st = hgl.block_cg_solve(g, torch.tensor(w, device=DEV), wl.lam, _panel(d["Y"]), s, tol=tol)
    assert st == 0
    # the GPU drops Gram pivots below 1e-12, i.e. singular values below 1e-6 (the Gram
    # squares them): the oracle takes the same rank decision with rank_tol = 1e-6
    o = block_cg_solve(H, w, wl.lam, d["Y"], s=s, tol=tol, rank_tol=1e-6)
    assert np.abs(iters.cpu().numpy().astype(int) - o["iters"]).max() <= 1, (iters, o["iters"])
    Fd = solve_dense(H, w, wl.lam, d["Y"])
    err = np.linalg.norm(F.cpu().numpy() - Fd, axis=0) / np.linalg.norm(Fd, axis=0)
    assert err.max() <= (1 + wl.lam) / wl.lam * tol * 1.01, err.max()
    assert relres.cpu().numpy().max() <= tol
    if s == 1:
        assert np.abs(iters.cpu().numpy().astype(int) - cg_solve(H, w, wl.lam, d["Y"], tol=tol)["iters"]).max() <= 1


def test_block_cg_finite_termination():
    """Six columns in one group on a 24-vertex system: within ceil(24/6) + 1 iterations
    (the shared Krylov space grows by six dimensions per iteration), to rounding."""
    H, g, w, Y = _spd_case()
    F, relres, iters, st = hgl.block_cg_solve(g, torch.tensor(w, device=DEV), 0.05, _panel(Y), 6, tol=1e-11)
    assert st == 0 and int(iters.cpu()[0]) <= 5, iters
    Fd = solve_dense(H, w, 0.05, Y)
    assert np.abs(F.cpu().numpy() - Fd).max() <= 1e-9 * np.abs(Fd).max()


def test_block_cg_dependent_zero_columns_and_warm_start():
    """A repeated and a zero column in one group leave the search block instead of
    breaking it down; a warm start from a nearby F reaches the same solution in the
    oracle's iteration count (here also 6: the four independent columns need the whole
    24-dimensional space whatever the starting residual)."""
    H, g, w, Y = _spd_case(seed=4)
    Y[:, 2] = Y[:, 0]
    Y[:, 3] = 0.0
    lam = 0.3
    wt = torch.tensor(w, device=DEV)
    F, relres, iters, st = hgl.block_cg_solve(g, wt, lam, _panel(Y), 6, tol=1e-12)
    assert st == 0
    Fd = solve_dense(H, w, lam, Y)
    Fg = F.cpu().numpy()
    assert np.abs(Fg - Fd).max() <= 1e-10 * np.abs(Fd).max()
    assert np.abs(Fg[:, 2] - Fg[:, 0]).max() <= 1e-10 * np.abs(Fd).max()
    assert np.abs(Fg[:, 3]).max() == 0.0
    F0 = _panel(Fd * (1 + 1e-6))
    F2, _, iters2, st2 = hgl.block_cg_solve(g, wt, lam, _panel(Y), 6, F=F0, tol=1e-12, warm_start=True)
    o = block_cg_solve(H, w, lam, Y, s=6, tol=1e-12, F0=Fd * (1 + 1e-6), rank_tol=1e-6)
    assert st2 == 0 and abs(int(iters2.cpu()[0]) - int(o["iters"][0])) <= 1
    assert int(iters2.cpu()[0]) <= int(iters.cpu()[0])
    assert np.abs(F2.cpu().numpy() - Fd).max() <= 1e-10 * np.abs(Fd).max()


def test_block_cg_zero_column_with_nonzero_warm_start():
    """A zero right-hand-side column has the exact solution 0: a nonzero warm start there
    is discarded, the column comes back exactly 0 with relres 0, and the other columns
    match the oracle's block CG run from the same warm start with that column zeroed
    (what the solver starts from), in iterations and solution."""
    H, g, w, Y = _spd_case(seed=7)
    Y[:, 1] = 0.0
    lam = 0.4
    wt = torch.tensor(w, device=DEV)
    Fd = solve_dense(H, w, lam, Y)
    F0 = Fd * (1 + 1e-3)
    F0[:, 1] = 1.0
    F, relres, iters, st = hgl.block_cg_solve(g, wt, lam, _panel(Y), 6, F=_panel(F0), tol=1e-12, warm_start=True)
    assert st == 0
    Fg = F.cpu().numpy()
    assert np.abs(Fg[:, 1]).max() == 0.0
    assert float(relres.cpu()[1]) == 0.0
    F0z = F0.copy()
    F0z[:, 1] = 0.0
    o = block_cg_solve(H, w, lam, Y, s=6, tol=1e-12, F0=F0z, rank_tol=1e-6)
    assert abs(int(iters.cpu()[0]) - int(o["iters"][0])) <= 1, (iters, o["iters"])
    assert np.abs(Fg - o["F"]).max() <= 1e-10 * np.abs(Fd).max()
    assert np.abs(Fg - Fd).max() <= 1e-10 * np.abs(Fd).max()


def test_block_cg_argument_errors():
    H, g, w, Y = _spd_case(n=12, m=10, c=2, seed=6)
    wt = torch.tensor(w, device=DEV)
    for s in (0, 33):
        with pytest.raises(hgl.HglError):
            hgl.block_cg_solve(g, wt, 0.5, _panel(Y), s)


def test_adaptive_step_block_cg_route_matches_oracle_loop():
    """hgl_adaptive_step with HGL_ROUTE_BCG (block CG over groups of k = 4 columns,
    warm-started from the previous F) through two outer iterations of the small workload
    against the oracle's loop (FP64 CG to 1e-12): F and w to 1e-8."""
    wl = synth.WORKLOADS["small_fp64"]
    d = synth.make_hypergraph(wl, 13)
    H, g = _graph(d["n"], d["m"], d["edge_ptr"], d["members"])
    wt = torch.tensor(d["w0"], device=DEV)
    Y = _panel(d["Y"])
    F = hgl.padded_panel(d["n"], d["c"])
    F.zero_()
    for _ in range(2):
        st = hgl.adaptive_step(g, wt, Y, F, wl.lam, wl.mu, wl.eta, tol=1e-11, route=hgl.HGL_ROUTE_BCG, k=4)
        assert st.solve.relres_max <= 1e-11 and st.solve.iters > 0
    Fr, wr, _ = adaptive_loop(H, d["w0"], wl.lam, wl.mu, wl.eta, d["Y"], 2, tol=1e-12)
    err = np.linalg.norm(F.cpu().numpy() - Fr, axis=0) / np.linalg.norm(Fr, axis=0)
    assert err.max() <= 1e-8
    assert np.linalg.norm(wt.cpu().numpy() - wr) / np.linalg.norm(wr) <= 1e-8
    with pytest.raises(hgl.HglError):
        hgl.adaptive_step(g, wt, Y, F, wl.lam, wl.mu, wl.eta, tol=1e-11, route=hgl.HGL_ROUTE_BCG, k=4,
                          flags=hgl.HGL_STEP_GRAPH)
