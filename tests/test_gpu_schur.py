"""The nested 2 x 2 Schur-complement inverse (Section 3, Eqs. 12-14) on the GPU
(hgl_schur_inverse) against the oracle's schur_inverse with the same Philox test
matrices, at the paper's scale (n = 5,867 vertices, minimum rank 50) on the tcgen05
tensor cores and at a smaller size on FP64 CUDA cores; and against M^-1 itself where
the scheme is exact (full rank)."""
import numpy as np
import pytest
import torch

import synth
from oracle import core, incidence, schur
from paper_1908_08281_gb300 import build as _build
from paper_1908_08281_gb300 import hgl

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda")
SEED = 777


@pytest.fixture(scope="module", autouse=True)
def _lib():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    _build.build()
    hgl.lib()


def _case(n, m, seed):
    """The small workload's hyperedge-size law (U{2..20}) at n vertices, weights drawn
    positive and normalised."""
    wl = synth.WORKLOADS["small_fp64"]
    d = synth.make_hypergraph(wl, seed, n=n, m=m, c=1)
    H = incidence.incidence_matrix(incidence.build_incidence(d["n"], d["m"], d["edge_ptr"], d["members"]))
    rng = np.random.default_rng(seed + 1)
    w = rng.random(m) + 0.1
    w /= w.sum()
    g = hgl.build_incidence(d["n"], d["m"], d["edge_ptr"], d["members"])
    return H, w, g


def test_schur_inverse_full_rank_is_exact_fp64():
    """With k at least every inverted matrix's size (n = 160: halves of 80, leaves of at
    most 40 rows) each randomized SVD captures its matrix exactly, so the nested scheme
    returns M^-1 to rounding (the formula of Section 3 is an identity)."""
    H, w, g = _case(160, 260, 1)
    lam = 0.5
    Mi = hgl.schur_inverse(g, torch.tensor(w, device=DEV), lam, 0, 160, 20, 80, 0, 0, SEED, hgl.HGL_FP64)
    M = (1 + lam) * np.eye(160) - core.theta_dense(H, w)
    assert np.abs(Mi.cpu().numpy() @ M - np.eye(160)).max() < 1e-10


def test_schur_inverse_fp64_matches_oracle():
    """FP64 CUDA cores, a sub-range of the vertices (global rows 300 .. 1,800: odd halves
    and the Philox rows offset), several nesting levels (r_min = 50 down to blocks of
    93 / 94 rows), truncated ranks: the oracle's schur_inverse with the same test
    matrices, element by element to 1e-9 of the largest entry."""
    H, w, g = _case(2000, 3000, 2)
    lam, row0, n = 0.5, 300, 1501
    Mi = hgl.schur_inverse(g, torch.tensor(w, device=DEV), lam, row0, n, 50, 32, 8, 2, SEED, hgl.HGL_FP64)
    T = core.theta_dense(H, w)[row0:row0 + n, row0:row0 + n]
    ref = schur.schur_inverse(T, lam, r_min=50, k=32, p=8, q=2, seed=SEED, row0=row0)
    got = Mi.cpu().numpy()
    assert np.abs(got - ref).max() <= 1e-9 * np.abs(ref).max(), np.abs(got - ref).max() / np.abs(ref).max()


def test_schur_inverse_tensor_cores_paper_scale():
    """The paper's scale: n = 5,867 vertices, minimum rank 50 (Section 3), the dense
    products on tcgen05 with TF32 pairs (about 2^-21 relative per product): against the
    FP64 oracle with the same test matrices in the Frobenius norm, and as good an
    approximation of M^-1 as the oracle's (the truncation error dominates rounding)."""
    n = 5867
    H, w, g = _case(n, 8800, 3)
    lam = 0.5
    wt = torch.tensor(w, device=DEV)
    hgl.profile_enable(True)
    Mi = hgl.schur_inverse(g, wt, lam, 0, n, 50, 50, 10, 2, SEED, hgl.HGL_FP32)
    torch.cuda.synchronize()
    tc_launches = hgl.profile_read(hgl.PROF_SCHUR_GEMM)[1]
    hgl.profile_enable(False)
    assert tc_launches > 0
    T = core.theta_dense(H, w)
    ref = schur.schur_inverse(T, lam, r_min=50, k=50, p=10, q=2, seed=SEED)
    got = Mi.cpu().numpy()
    rel = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert rel <= 1e-5, rel
    Me = np.linalg.inv((1 + lam) * np.eye(n) - T)
    e_gpu = np.linalg.norm(got - Me) / np.linalg.norm(Me)
    e_ref = np.linalg.norm(ref - Me) / np.linalg.norm(Me)
    assert abs(e_gpu - e_ref) <= 1e-5 + 1e-3 * e_ref, (e_gpu, e_ref)


def test_schur_inverse_argument_errors():
    H, w, g = _case(200, 300, 4)
    wt = torch.tensor(w, device=DEV)
    # (lam, row0, nrows, r_min, k, p, q): a range past n, lam <= 0, r_min = 0, k + p > 96
    for lam, row0, nrows, r_min, k, p, q in [(0.5, 150, 100, 10, 8, 2, 1), (-1.0, 0, 100, 10, 8, 2, 1),
                                             (0.5, 0, 100, 0, 8, 2, 1), (0.5, 0, 100, 10, 90, 10, 1)]:
        with pytest.raises(hgl.HglError):
            hgl.schur_inverse(g, wt, lam, row0, nrows, r_min, k, p, q, 1)
