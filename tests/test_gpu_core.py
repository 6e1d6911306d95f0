"""GPU parity: incidence, degrees, operator, CG, gradient, projection and the adaptive
step of libhgl against the CPU oracle, through the C ABI."""
import numpy as np
import pytest
import torch

import synth
from oracle import core, incidence
from paper_1908_08281_gb300 import build as _build
from paper_1908_08281_gb300 import hgl

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    _build.build()
    hgl.lib()


def _case(name="small_fp64", seed=0, n=None, m=None, c=None):
    wl = synth.WORKLOADS[name]
    d = synth.make_hypergraph(wl, seed, n=n, m=m, c=c)
    og = incidence.build_incidence(d["n"], d["m"], d["edge_ptr"], d["members"])
    H = incidence.incidence_matrix(og)
    return wl, d, og, H


def _panel(a: np.ndarray, dtype=torch.float64, pad_fill=None):
    n, c = a.shape
    P = hgl.padded_panel(n, c, dtype, DEV, fill=pad_fill)
    P.copy_(torch.from_numpy(np.ascontiguousarray(a)).to(dtype))
    return P


def _relcol(x, ref):
    den = np.linalg.norm(ref, axis=0)
    den[den == 0] = 1.0
    return np.linalg.norm(x - ref, axis=0) / den


# ---------------------------------------------------------------- incidence ---

@pytest.mark.parametrize("name,seed,n,m", [
    ("small_fp64", 0, None, None),
    ("mixed_cg", 1, 20_000, 30_000),
    ("adjoint", 2, 30_000, 50_000),
    ("full_adaptive", 3, 40_000, 80_000),
])
def test_incidence_bit_exact(name, seed, n, m):
    wl, d, og, _ = _case(name, seed, n, m, c=1)
    g = hgl.build_incidence(d["n"], d["m"], d["edge_ptr"], d["members"])
    ex = hgl.graph_export(g)
    for k in ("csc_ptr", "csc_idx", "csr_ptr", "csr_idx", "de"):
        assert np.array_equal(ex[k].cpu().numpy(), og[k]), k


def test_incidence_from_device_arrays_and_huge_edge():
    # one hyperedge larger than the shared-memory sort tile, members on the device
    rng = np.random.default_rng(5)
    n = 40_000
    sizes = np.array([20_000, 3, 40_000, 1, 17, 33, 12_289])
    ptr = np.zeros(len(sizes) + 1, np.int64)
    np.cumsum(sizes, out=ptr[1:])
    mem = np.concatenate([rng.permutation(n)[:s] for s in sizes]).astype(np.int32)
    og = incidence.build_incidence(n, len(sizes), ptr, mem)
    g = hgl.build_incidence(n, len(sizes), torch.from_numpy(ptr).to(DEV), torch.from_numpy(mem).to(DEV))
    ex = hgl.graph_export(g)
    for k in ("csc_ptr", "csc_idx", "csr_ptr", "csr_idx", "de"):
        assert np.array_equal(ex[k].cpu().numpy(), og[k]), k


@pytest.mark.parametrize("ptr,mem,code", [
    ([0, 2, 2], [0, 1], "HGL_ERR_EMPTY_EDGE"),
    ([0, 2], [0, 5], "HGL_ERR_INDEX_RANGE"),
    ([0, 2], [-1, 0], "HGL_ERR_INDEX_RANGE"),
    ([0, 3], [1, 2, 1], "HGL_ERR_DUPLICATE_MEMBER"),
    ([1, 2], [0, 1], "HGL_ERR_INVALID_ARG"),
    ([0, 3, 2], [0, 1, 2], "HGL_ERR_INVALID_ARG"),
])
def test_incidence_errors(ptr, mem, code):
    with pytest.raises(hgl.HglError) as ei:
        hgl.build_incidence(3, len(ptr) - 1, np.array(ptr, np.int64), np.array(mem, np.int32))
    assert ei.value.name == code


# ------------------------------------------------------------------ degrees ---

def test_degrees_and_zero_degree_vertex():
    _, d, og, H = _case("small_fp64", 4, n=500, m=700)
    rng = np.random.default_rng(0)
    w = rng.random(d["m"])
    # zero all hyperedges of vertex 7 -> dv_7 = 0 -> s_7 = 0
    w[og["csr_idx"][og["csr_ptr"][7]:og["csr_ptr"][8]]] = 0.0
    g = hgl.build_incidence(d["n"], d["m"], d["edge_ptr"], d["members"])
    dv, s, t = hgl.degrees(g, torch.tensor(w, device=DEV))
    rdv, _, rs, rt = core.degrees(H, w)
    assert np.allclose(dv.cpu().numpy(), rdv, rtol=1e-14, atol=0)
    assert np.allclose(s.cpu().numpy(), rs, rtol=1e-14, atol=0)
    assert np.array_equal(t.cpu().numpy(), rt)
    assert s.cpu().numpy()[7] == 0.0


# ----------------------------------------------------------------- operator ---

@pytest.mark.parametrize("c", [1, 3, 10, 64, 130, 300])
def test_apply_theta_fp64(c):
    _, d, og, H = _case("mixed_cg", 7, n=6000, m=9000, c=c)
    rng = np.random.default_rng(c)
    w = rng.random(d["m"]) + 0.01
    X = rng.standard_normal((d["n"], c))
    g = hgl.build_incidence(d["n"], d["m"], d["edge_ptr"], d["members"])
    wt = torch.tensor(w, device=DEV)
    Xt = _panel(X)
    Z = hgl.padded_panel(d["n"], c, torch.float64, DEV, fill=float("nan"))
    hgl.apply_theta(g, wt, Xt, 1.5, -1.0, Z=Z)
    ref = core.theta_apply(H, w, X, 1.5, -1.0)
    Zc = Z.cpu().numpy()
    assert np.allclose(Zc, ref, rtol=1e-12, atol=1e-13)
    # padding columns of Z untouched
    base = Z.as_strided((d["n"], Z.stride(0)), (Z.stride(0), 1))
    if Z.stride(0) > c:
        assert torch.isnan(base[:, c:]).all()


@pytest.mark.parametrize("dtype,rtol", [(torch.float32, 2e-6), (torch.bfloat16, 1.2e-2)])
@pytest.mark.parametrize("c", [5, 16, 30, 128, 200])
def test_apply_theta_low_precision(dtype, rtol, c):
    _, d, og, H = _case("mixed_cg", 8, n=5000, m=8000, c=c)
    rng = np.random.default_rng(3)
    w = rng.random(d["m"]) + 0.01
    Xt = _panel(rng.standard_normal((d["n"], c)), dtype)
    X = Xt.to(torch.float64).cpu().numpy()  # the values the kernel actually reads
    g = hgl.build_incidence(d["n"], d["m"], d["edge_ptr"], d["members"])
    Z = hgl.apply_theta(g, torch.tensor(w, device=DEV), Xt, 1.5, -1.0)
    ref = core.theta_apply(H, w, X, 1.5, -1.0)
    err = np.abs(Z.to(torch.float64).cpu().numpy() - ref)
    scale = np.abs(ref) + np.abs(1.5 * X) + core.theta_apply(H, w, np.abs(X), 0.0, 1.0)
    assert (err <= rtol * scale + 1e-30).all(), err.max()


@pytest.mark.parametrize("sizes", ["small", "large", "mixed"])
@pytest.mark.parametrize("dtype,rtol", [(torch.float64, 1e-12), (torch.float32, 2e-6), (torch.bfloat16, 1.2e-2)])
def test_apply_theta_small_and_large_hyperedges(sizes, dtype, rtol):
    """Hyperedges of at most three members (one-member ones included) enter the vertex
    pass straight from X, larger ones go through the intermediate: graphs with only
    small, only large, or both kinds (plus a heavy hyperedge and vertices in no
    hyperedge) match Eq. 1 in the oracle."""
    rng = np.random.default_rng({"small": 1, "large": 2, "mixed": 3}[sizes])
    n, m, c = 3000, 5000, 37
    if sizes == "small":
        sz = rng.integers(1, 4, m)
    elif sizes == "large":
        sz = rng.integers(4, 12, m)
    else:
        sz = rng.integers(1, 7, m)
        sz[7] = 400
    members = np.concatenate([rng.choice(n - 50, int(k), replace=False) for k in sz]).astype(np.int32)
    edge_ptr = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(sz, out=edge_ptr[1:])
    H = incidence.incidence_matrix(incidence.build_incidence(n, m, edge_ptr, members))
    w = rng.random(m) + 0.01
    g = hgl.build_incidence(n, m, edge_ptr, members)
    Xt = _panel(rng.standard_normal((n, c)), dtype)
    X = Xt.to(torch.float64).cpu().numpy()
    Z = hgl.apply_theta(g, torch.tensor(w, device=DEV), Xt, 1.5, -1.0)
    ref = core.theta_apply(H, w, X, 1.5, -1.0)
    err = np.abs(Z.to(torch.float64).cpu().numpy() - ref)
    scale = np.abs(ref) + np.abs(1.5 * X) + core.theta_apply(H, w, np.abs(X), 0.0, 1.0)
    assert (err <= rtol * scale + 1e-30).all(), err.max()
    # the last 50 vertices are in no hyperedge: Z = 1.5 X there (exact in FP64)
    if dtype == torch.float64:
        assert np.array_equal(Z.cpu().numpy()[-50:], 1.5 * X[-50:])


@pytest.mark.parametrize("dtype,ch", [(hgl.HGL_FP64, torch.float64), (hgl.HGL_FP32, torch.float32)])
def test_tuned_operator_and_residual_still_match(dtype, ch):
    """Tuning only changes the column chunk: results stay within each path's bound."""
    wl, d, og, H = _case("mixed_cg", 9, n=6000, m=9000, c=150)
    c = d["c"]
    rng = np.random.default_rng(11)
    w = rng.random(d["m"]) + 0.01
    w /= w.sum()
    g = hgl.build_incidence(d["n"], d["m"], d["edge_ptr"], d["members"])
    wt = torch.tensor(w, device=DEV)
    op_cc, pair_cc, grid = hgl.tune_operator(g, wt, c, dtype)
    assert grid in (0, 1)
    E = 16 // torch.tensor([], dtype=ch).element_size()
    assert 1 <= op_cc and (op_cc % E == 0 or op_cc >= c)
    if dtype == hgl.HGL_FP64:
        assert pair_cc == 0
    else:
        assert pair_cc >= 4 and pair_cc % 4 == 0
    Xt = _panel(rng.standard_normal((d["n"], c)), ch)
    X = Xt.to(torch.float64).cpu().numpy()
    Z = hgl.apply_theta(g, wt, Xt, 1.5, -1.0)
    ref = core.theta_apply(H, w, X, 1.5, -1.0)
    scale = np.abs(ref) + np.abs(1.5 * X) + core.theta_apply(H, w, np.abs(X), 0.0, 1.0)
    rtol = 1e-13 if dtype == hgl.HGL_FP64 else 2e-6
    assert (np.abs(Z.to(torch.float64).cpu().numpy() - ref) <= rtol * scale + 1e-30).all()
    # the mixed solver uses the tuned residual chunk and still certifies its tolerance
    Y = _panel(d["Y"])
    F, relres, iters, st = hgl.cg_solve(g, wt, wl.lam, Y, tol=1e-8, dtype=hgl.HGL_FP32)
    refF, _ = core.certified_solve(H, w, wl.lam, d["Y"])
    assert st.relres_max <= 1e-8
    assert _relcol(F.cpu().numpy(), refF).max() <= (1 + wl.lam) / wl.lam * 1e-8 * 1.01 + 1e-12


# ------------------------------------------------------------------------ CG ---

def test_cg_fp64_small_workload():
    wl, d, og, H = _case("small_fp64", 0)
    rng = np.random.default_rng(1)
    w = rng.random(d["m"]) + 0.1
    w /= w.sum()
    g = hgl.build_incidence(d["n"], d["m"], d["edge_ptr"], d["members"])
    Y = _panel(d["Y"])
    F, relres, iters, st = hgl.cg_solve(g, torch.tensor(w, device=DEV), wl.lam, Y, tol=1e-10)
    ref = core.solve_dense(H, w, wl.lam, d["Y"])
    err = _relcol(F.cpu().numpy(), ref)
    assert err.max() <= 1e-10
    assert st.relres_max <= 1e-10 and st.converged == d["c"]
    assert relres.cpu().numpy().max() <= 1e-10
    # same iteration counts as the oracle's CG (same recurrences)
    oc = core.cg_solve(H, w, wl.lam, d["Y"], tol=1e-10)
    it = iters.cpu().numpy()
    assert np.abs(it - oc["iters"]).max() <= 1


@pytest.mark.parametrize("mode", [hgl.HGL_FP32, hgl.HGL_BF16])
def test_cg_mixed_precision(mode):
    wl, d, og, H = _case("mixed_cg", 2, n=8000, m=12000, c=20)
    w = np.full(d["m"], 1.0 / d["m"])
    g = hgl.build_incidence(d["n"], d["m"], d["edge_ptr"], d["members"])
    Y = _panel(d["Y"])
    F, relres, iters, st = hgl.cg_solve(g, torch.tensor(w, device=DEV), wl.lam, Y, tol=1e-8, dtype=mode)
    ref, bound = core.certified_solve(H, w, wl.lam, d["Y"])
    err = _relcol(F.cpu().numpy(), ref)
    assert err.max() <= 1e-5, err.max()
    assert st.relres_max <= 1e-8
    # kappa(M) <= (1+lam)/lam bounds the error by the residual
    assert err.max() <= (1 + wl.lam) / wl.lam * 1e-8 * 1.01 + 1e-12


@pytest.mark.parametrize("mode", [hgl.HGL_FP32, hgl.HGL_BF16])
def test_cg_fp32_loose_tol_starts_from_fp32_residual(mode):
    """At tol >= 4 * 2^-24 * (1 + 2(1+lam)/lam) the mixed solve (FP32 or BF16 search
    directions) starts from an FP32 estimate of the first residual and checks with the
    compact pair residual (low parts in BF16); convergence is still decided on an
    FP64-accurate residual: the reported relres matches the host's FP64 residual of the
    returned F, and a warm start from a converged F ends without iterations (the
    estimate alone never ends a solve)."""
    wl, d, og, H = _case("mixed_cg", 4, n=9000, m=14000, c=21)
    tol = 3e-6
    assert tol >= 4 * 2.0 ** -24 * (1 + 2 * (1 + wl.lam) / wl.lam)
    w = np.random.default_rng(5).random(d["m"]) + 0.1
    w /= w.sum()
    g = hgl.build_incidence(d["n"], d["m"], d["edge_ptr"], d["members"])
    wt = torch.tensor(w, device=DEV)
    Y = _panel(d["Y"])
    F, relres, iters, st = hgl.cg_solve(g, wt, wl.lam, Y, tol=tol, dtype=mode)
    Fg = F.cpu().numpy()
    R = wl.lam * d["Y"] - core.theta_apply(H, w, Fg, 1.0 + wl.lam, -1.0)
    rel = np.linalg.norm(R, axis=0) / np.linalg.norm(wl.lam * d["Y"], axis=0)
    assert rel.max() <= tol, rel.max()
    assert np.allclose(relres.cpu().numpy(), rel, rtol=1e-3, atol=1e-12)
    ref, _ = core.certified_solve(H, w, wl.lam, d["Y"])
    assert _relcol(Fg, ref).max() <= (1 + wl.lam) / wl.lam * tol * 1.01
    F2, relres2, iters2, st2 = hgl.cg_solve(g, wt, wl.lam, Y, F=F, tol=tol, dtype=mode, warm_start=True)
    assert iters2.cpu().numpy().max() == 0 and st2.refinements == 0
    assert np.allclose(relres2.cpu().numpy(), rel, rtol=1e-3, atol=1e-12)
    assert np.array_equal(F2.cpu().numpy(), Fg)


def test_pair_split_conversions_match_fp64_definitions():
    """The mixed solver's FP64 <-> FP32-pair conversions (computed from the IEEE-754 bit
    fields, no FP64 arithmetic in range) equal their plain definitions bit for bit:
    hi = fl32(x), lo = fl32(x - hi), back = hi + lo in FP64 -- over random magnitudes,
    rounding ties, significands that carry into the next binade, signed zeros,
    subnormals, values outside the fast range, infinities and NaN."""
    rng = np.random.default_rng(17)
    x = rng.standard_normal(200000) * 10.0 ** rng.uniform(-25, 35, 200000)
    f = rng.standard_normal(5000).astype(np.float32).astype(np.float64)
    ulp = np.spacing(f.astype(np.float32)).astype(np.float64)
    special = np.concatenate([
        f + 0.5 * ulp, f - 0.5 * ulp,               # ties (rounded to even)
        f + 0.5 * ulp * (1 + 2.0 ** -20),           # just above a tie
        np.nextafter(2.0 ** np.arange(-60, 60), 0),  # all-ones significands: the rounding carries
        [0.0, -0.0, 5e-324, -2.2e-308, 1e-30, 3e-22, 1e38, 3.4e38, 1e40, -1e300, np.inf, -np.inf, np.nan],
    ])
    x = np.concatenate([x, special])
    hi, lo, back = hgl.selftest_pair_split(torch.tensor(x, device=DEV))
    with np.errstate(over="ignore", invalid="ignore"):
        rhi = x.astype(np.float32)
        rlo = (x - rhi.astype(np.float64)).astype(np.float32)
        rback = rhi.astype(np.float64) + rlo.astype(np.float64)
    for got, ref in ((hi.cpu().numpy(), rhi), (lo.cpu().numpy(), rlo), (back.cpu().numpy(), rback)):
        both_nan = np.isnan(got) & np.isnan(ref)
        bits = np.uint32 if got.dtype == np.float32 else np.uint64
        same = got.view(bits) == ref.view(bits)
        assert (same | both_nan).all(), (x[~(same | both_nan)][:5], got[~(same | both_nan)][:5], ref[~(same | both_nan)][:5])


def test_cg_zero_column_warm_start_and_ragged_c():
    wl, d, og, H = _case("small_fp64", 3, n=700, m=1000, c=7)
    w = np.full(d["m"], 1.0 / d["m"])
    Yn = d["Y"].copy()
    Yn[:, 2] = 0.0
    g = hgl.build_incidence(d["n"], d["m"], d["edge_ptr"], d["members"])
    wt = torch.tensor(w, device=DEV)
    Y = _panel(Yn)
    F, relres, iters, st = hgl.cg_solve(g, wt, 1.0, Y, tol=1e-10)
    assert iters.cpu().numpy()[2] == 0 and torch.all(F[:, 2] == 0)
    F0 = hgl.padded_panel(d["n"], d["c"])
    F0.copy_(F)
    F2, _, iters2, st2 = hgl.cg_solve(g, wt, 1.0, Y, F=F0, tol=1e-10, warm_start=True)
    assert iters2.cpu().numpy().max() <= 1
    ref = core.solve_dense(H, w, 1.0, Yn)
    assert _relcol(F2.cpu().numpy(), ref).max() <= 1e-10


def test_device_wait_timeout_reports_status_and_device_stays_usable():
    """A bounded device wait on a barrier that nothing arrives on gives up after its
    cycle limit and the call returns HGL_ERR_TIMEOUT; the next launches run normally."""
    for limit in (1000, 2_000_000):
        with pytest.raises(hgl.HglError) as ei:
            hgl.selftest_wait_timeout(limit)
        assert ei.value.status == -8
    wl, d, og, H = _case("small_fp64", 11, n=300, m=450, c=3)
    g = hgl.build_incidence(d["n"], d["m"], d["edge_ptr"], d["members"])
    w = np.full(d["m"], 1.0 / d["m"])
    Z = hgl.apply_theta(g, torch.tensor(w, device=DEV), _panel(d["Y"]), 1.5, -1.0).cpu().numpy()
    assert np.allclose(Z, core.theta_apply(H, w, d["Y"], 1.5, -1.0), rtol=1e-12, atol=1e-14)


def test_nonfinite_right_hand_side_reports_status():
    """A NaN in one column of Y: that column is reported non-finite (HGL_ERR_NONFINITE),
    the others still converge to the oracle's solution."""
    wl, d, og, H = _case("small_fp64", 12, n=500, m=800, c=4)
    w = np.full(d["m"], 1.0 / d["m"])
    Yn = d["Y"].copy()
    Yn[7, 1] = np.nan
    g = hgl.build_incidence(d["n"], d["m"], d["edge_ptr"], d["members"])
    for mode in (hgl.HGL_FP64, hgl.HGL_FP32):
        F, relres, iters, st = hgl.cg_solve(g, torch.tensor(w, device=DEV), 1.0, _panel(Yn), tol=1e-8, dtype=mode,
                                            raise_on_fail=False)
        assert st.status == -9, (mode, st.status)
        ref = core.solve_dense(H, w, 1.0, d["Y"])
        ok = [0, 2, 3]
        err = _relcol(F.cpu().numpy()[:, ok], ref[:, ok])
        assert err.max() <= 2 * 1e-8 * 1.01, (mode, err.max())


def test_cg_not_converged_status():
    wl, d, og, H = _case("small_fp64", 5, n=400, m=600, c=3)
    g = hgl.build_incidence(d["n"], d["m"], d["edge_ptr"], d["members"])
    Y = _panel(d["Y"])
    with pytest.raises(hgl.HglError) as ei:
        hgl.cg_solve(g, torch.full((d["m"],), 1.0 / d["m"], device=DEV, dtype=torch.float64), 1.0, Y, tol=1e-12,
                     max_iter=2)
    assert ei.value.name == "HGL_ERR_NOT_CONVERGED"


# ------------------------------------------------------------------ gradient ---

@pytest.mark.parametrize("c", [1, 10, 96])
def test_weight_grad_fp64(c):
    _, d, og, H = _case("adjoint", 4, n=3000, m=5000, c=c)
    rng = np.random.default_rng(c + 1)
    w = rng.random(d["m"]) + 0.05
    F = rng.standard_normal((d["n"], c))
    g = hgl.build_incidence(d["n"], d["m"], d["edge_ptr"], d["members"])
    wt = torch.tensor(w, device=DEV)
    Ft = _panel(F)
    gr = hgl.weight_grad(g, wt, Ft, mu=1e-3).cpu().numpy()
    ref = core.weight_grad(H, w, F, 1e-3)
    assert np.allclose(gr, ref, rtol=1e-11, atol=1e-12 * np.abs(ref).max())
    grf = hgl.weight_grad(g, wt, Ft, mu=1e-3, dv_frozen=True).cpu().numpy()
    reff = core.weight_grad(H, w, F, 1e-3, dv_frozen=True)
    assert np.allclose(grf, reff, rtol=1e-11, atol=1e-12 * np.abs(reff).max())
    Z = rng.standard_normal((d["n"], c))
    Zt = hgl.padded_panel(d["n"], c)
    Zt.copy_(torch.from_numpy(Z))
    gb = hgl.weight_grad(g, wt, Ft, mu=0.0, Z=Zt).cpu().numpy()
    refb = -core.bilinear_theta_grad(H, w, F, Z)
    assert np.allclose(gb, refb, rtol=1e-10, atol=1e-11 * np.abs(refb).max())


def test_weight_grad_fp32():
    _, d, og, H = _case("mixed_cg", 6, n=4000, m=6000, c=40)
    rng = np.random.default_rng(2)
    w = rng.random(d["m"]) + 0.05
    Ft = _panel(rng.standard_normal((d["n"], 40)), torch.float32)
    F = Ft.to(torch.float64).cpu().numpy()
    g = hgl.build_incidence(d["n"], d["m"], d["edge_ptr"], d["members"])
    gr = hgl.weight_grad(g, torch.tensor(w, device=DEV), Ft, mu=0.0).cpu().numpy()
    ref = core.weight_grad(H, w, F, 0.0)
    assert np.abs(gr - ref).max() <= 1e-5 * np.abs(ref).max()


# ---------------------------------------------------------------- projection ---

@pytest.mark.parametrize("m,scale", [(1, 1.0), (7, 0.3), (1000, 1e-2), (300_000, 1e-5), (300_000, 10.0)])
def test_project_simplex(m, scale):
    rng = np.random.default_rng(m)
    w = rng.random(m)
    w /= w.sum()
    gvec = rng.standard_normal(m) * scale
    wt = torch.tensor(w, device=DEV)
    hgl.project_simplex(wt, torch.tensor(gvec, device=DEV), 0.5)
    ref = core.project_simplex(w - 0.5 * gvec)
    out = wt.cpu().numpy()
    assert np.allclose(out, ref, rtol=0, atol=1e-13)
    assert abs(out.sum() - 1) < 1e-10 and out.min() >= 0


@pytest.mark.parametrize("m,frac0,eta", [(1, 0.0, 1.0), (9, 0.3, 0.05), (5000, 0.2, 1e-4), (5000, 0.2, 1e-1),
                                         (300_000, 0.5, 1e-6), (300_000, 0.0, 1e-3)])
def test_active_set_step(m, frac0, eta):
    """The literal active-set step of Eq. 5 against the oracle: pinned zeros, clamping
    at 0 and rescaling (large eta), and the unclamped regime (small eta)."""
    rng = np.random.default_rng(m + int(100 * frac0))
    w = rng.random(m)
    w[rng.random(m) < frac0] = 0.0
    if w.sum() == 0:
        w[0] = 1.0
    w /= w.sum()
    gvec = rng.standard_normal(m)
    wt = torch.tensor(w, device=DEV)
    hgl.active_set_step(wt, torch.tensor(gvec, device=DEV), eta)
    ref = core.active_set_step(w, gvec, eta)
    out = wt.cpu().numpy()
    assert np.allclose(out, ref, rtol=1e-12, atol=1e-15)
    assert abs(out.sum() - 1) < 1e-12 and out.min() >= 0 and (out[w == 0] == 0).all()


@pytest.mark.parametrize("flags", [hgl.HGL_STEP_ACTIVE_SET, hgl.HGL_STEP_ACTIVE_SET | hgl.HGL_STEP_GRAPH])
def test_adaptive_loop_active_set_step(flags):
    """Outer iterations with the active-set weight step (eager and captured), each step
    checked against the oracle from the GPU's own w."""
    wl, d, og, H = _case("small_fp64", 1)
    g = hgl.build_incidence(d["n"], d["m"], d["edge_ptr"], d["members"])
    wt = torch.tensor(d["w0"], device=DEV)
    Y = _panel(d["Y"])
    F = hgl.padded_panel(d["n"], d["c"])
    eta = 1e-3
    for i in range(5):
        w_before = wt.cpu().numpy().copy()
        st = hgl.adaptive_step(g, wt, Y, F, wl.lam, 1e-3, eta, tol=1e-10, flags=flags)
        assert st.solve.relres_max <= 1e-10
        Fr = core.solve_dense(H, w_before, wl.lam, d["Y"])
        assert _relcol(F.cpu().numpy(), Fr).max() <= 1e-9
        w_ref = core.active_set_step(w_before, core.weight_grad(H, w_before, Fr, 1e-3), eta)
        assert np.linalg.norm(wt.cpu().numpy() - w_ref) <= 1e-9 * np.linalg.norm(w_ref), i


# ------------------------------------------------------------- adaptive step ---

def test_adaptive_loop_small_workload():
    wl, d, og, H = _case("small_fp64", 0)
    g = hgl.build_incidence(d["n"], d["m"], d["edge_ptr"], d["members"])
    wt = torch.tensor(d["w0"], device=DEV)
    Y = _panel(d["Y"])
    F = hgl.padded_panel(d["n"], d["c"])
    objs = []
    for _ in range(wl.outer):
        st = hgl.adaptive_step(g, wt, Y, F, wl.lam, wl.mu, wl.eta, tol=wl.tol)
        objs.append(st.objective)
        assert st.solve.relres_max <= wl.tol
    Fr, wr, trace = core.adaptive_loop(H, d["w0"], wl.lam, wl.mu, wl.eta, d["Y"], wl.outer, tol=1e-12)
    assert _relcol(F.cpu().numpy(), Fr).max() <= 1e-10
    wg = wt.cpu().numpy()
    assert np.linalg.norm(wg - wr) / np.linalg.norm(wr) <= 1e-10
    # objective reported by the step equals P(w) at the solve's (w, F)
    wprev = trace[-2]["w_new"]
    assert abs(objs[-1] - core.objective(H, wprev, trace[-1]["F"], wl.mu)) <= 1e-9 * abs(objs[-1])
