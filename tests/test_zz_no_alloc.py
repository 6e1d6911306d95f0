"""hgl_apply_theta_noalloc through the C ABI: the variant of the operator apply that
allocates nothing in the call (for callers whose device memory all comes from their
own pool or budget, or that cannot take the synchronisation of cudaMalloc/cudaFree)
must give the same Z as hgl_apply_theta, on two calls in a row that share its fixed
scratch array, and for FP64 panels the oracle's Z = a X + b Theta X (Eq. 1).  This
file is named to be collected last."""
import ctypes

import numpy as np
import pytest
import torch

import synth
from oracle import core, incidence
from paper_1908_08281_gb300 import build as _build
from paper_1908_08281_gb300 import hgl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    _build.build()
    return hgl.lib()


def _raw_call(lib, fn, g, w, X, Z, a, b):
    px, ldx, dt = hgl._panel(X, "X")
    pz, ldz, _ = hgl._panel(Z, "Z")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return fn(g.handle, ctypes.c_void_p(w.data_ptr()), a, b, px, ldx, pz, ldz, X.shape[1], dt, stream)


@pytest.mark.parametrize("dtype,c,m", [(torch.float64, 64, 300_000), (torch.float32, 100, 20_000),
                                       (torch.bfloat16, 40, 50_000)])
def test_noalloc_matches_allocating_entry_point(lib, dtype, c, m):
    wl = synth.WORKLOADS["mixed_cg"]
    d = synth.make_hypergraph(wl, 11, n=m // 2, m=m, c=1)
    g = hgl.build_incidence(d["n"], d["m"], d["edge_ptr"], d["members"])
    dev = torch.device("cuda")
    rng = np.random.default_rng(c)
    w = torch.tensor(rng.random(d["m"]) + 0.01, device=dev)
    X = hgl.padded_panel(d["n"], c, dtype, dev)
    X.copy_(torch.from_numpy(rng.standard_normal((d["n"], c))).to(dtype))
    Zref = hgl.padded_panel(d["n"], c, dtype, dev)
    assert _raw_call(lib, lib.hgl_apply_theta, g, w, X, Zref, 1.5, -1.0) == 0
    ref = Zref.to(torch.float64).cpu().numpy()
    tol = {torch.float64: 1e-12, torch.float32: 1e-5, torch.bfloat16: 2e-2}[dtype]
    if dtype == torch.float64:
        H = incidence.incidence_matrix(incidence.build_incidence(d["n"], d["m"], d["edge_ptr"], d["members"]))
        ora = core.theta_apply(H, w.cpu().numpy(), X.cpu().numpy(), 1.5, -1.0)
        assert np.abs(ref - ora).max() <= tol * np.abs(ora).max()
    for call in range(2):
        Z = hgl.padded_panel(d["n"], c, dtype, dev, fill=float("nan"))
        st = _raw_call(lib, lib.hgl_apply_theta_noalloc, g, w, X, Z, 1.5, -1.0)
        assert st == 0, lib.hgl_last_error().decode()
        torch.cuda.synchronize()
        out = Z.to(torch.float64).cpu().numpy()
        scale = np.abs(ref).max()
        assert np.abs(out - ref).max() <= tol * scale, (call, np.abs(out - ref).max() / scale)
        if dtype == torch.float64:
            assert np.abs(out - ora).max() <= tol * np.abs(ora).max(), call
    g.close()


def test_noalloc_rejects_oversized_graph(lib):
    # 2,200,000 two-member hyperedges exceed the scratch for FP64 panels
    m, n = 2_200_000, 4096
    rng = np.random.default_rng(0)
    a = rng.integers(0, n, m)
    b = (a + 1 + rng.integers(0, n - 1, m)) % n
    mem = np.stack([a, b], 1).reshape(-1).astype(np.int32)
    ptr = np.arange(0, 2 * m + 1, 2, dtype=np.int64)
    g = hgl.build_incidence(n, m, ptr, mem)
    dev = torch.device("cuda")
    w = torch.full((m,), 1.0 / m, device=dev, dtype=torch.float64)
    X = hgl.padded_panel(n, 2, torch.float64, dev)
    Z = hgl.padded_panel(n, 2, torch.float64, dev)
    st = _raw_call(lib, lib.hgl_apply_theta_noalloc, g, w, X, Z, 0.0, 1.0)
    assert hgl.STATUS[st] == "HGL_ERR_INVALID_ARG"
    assert "scratch" in lib.hgl_last_error().decode()
    g.close()
