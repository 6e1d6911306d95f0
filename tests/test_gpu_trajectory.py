"""The mixed-precision adaptive loop against the oracle's loop over several outer
iterations from w0 (Section 2: the solve at fixed w, then the projected step of Eq. 5):
F and w of the whole trajectory, each step compared with the oracle's same step -- not
re-seeded from the GPU's own w.

The step size follows the full workload's rule (a step moves w by about 5% of its
norm), under which the loop is well conditioned: two correct solvers that differ at
the tolerance stay within it over the whole loop."""
import numpy as np
import pytest
import torch

import synth
from oracle import core, incidence
from paper_1908_08281_gb300 import build as _build
from paper_1908_08281_gb300 import hgl

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda")
STEPS = 6
TOL = 2e-6     # relative residual of the mixed solve: per-column F error <= (1+lam)/lam * TOL = 6e-6
SEED = 4242


@pytest.fixture(scope="module")
def loop():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    _build.build()
    hgl.lib()
    wl = synth.WORKLOADS["full_adaptive"]
    d = synth.make_hypergraph(wl, 31, n=20000, m=40000, c=24)
    H = incidence.incidence_matrix(incidence.build_incidence(d["n"], d["m"], d["edge_ptr"], d["members"]))
    w0 = d["w0"]
    # step size: the first projected step moves w by 5% of its norm (for a step that
    # clamps nothing the projection subtracts the mean of the gradient)
    F0, _ = core.certified_solve(H, w0, wl.lam, d["Y"])
    g0 = core.weight_grad(H, w0, F0, wl.mu)
    eta = 0.05 * np.linalg.norm(w0) / np.linalg.norm(g0 - g0.mean())
    _, _, trace = core.adaptive_loop(H, w0, wl.lam, wl.mu, eta, d["Y"], STEPS, tol=1e-12)
    g = hgl.build_incidence(d["n"], d["m"], d["edge_ptr"], d["members"])
    return wl, d, H, g, eta, trace


@pytest.mark.parametrize("dtype", [hgl.HGL_FP32, hgl.HGL_BF16])
@pytest.mark.parametrize("route", [hgl.HGL_ROUTE_BR, hgl.HGL_ROUTE_CG])
@pytest.mark.parametrize("flags", [0, hgl.HGL_STEP_GRAPH])
def test_mixed_trajectory_matches_oracle_loop(loop, route, flags, dtype):
    """FP32 panels (or BF16 search directions) with FP64-accurate refinement, eager and
    captured (the first call eager, the second captured, later ones replayed),
    block-rSVD preconditioned or plain CG: after every outer iteration F (the solve at
    the step's w) and the new w agree with the oracle's loop (FP64 CG to 1e-12) to 1e-5
    relative."""
    wl, d, H, g, eta, trace = loop
    Y = hgl.padded_panel(d["n"], d["c"], torch.float64, DEV)
    Y.copy_(torch.from_numpy(d["Y"]))
    F = hgl.padded_panel(d["n"], d["c"], torch.float64, DEV)
    F.zero_()
    w = torch.tensor(d["w0"], device=DEV)
    moved = []
    for i in range(STEPS):
        w_before = w.clone()
        st = hgl.adaptive_step(g, w, Y, F, lam=wl.lam, mu=wl.mu, eta=eta, tol=TOL, dtype=dtype, route=route,
                               block_ptr=d["block_ptr"], k=16, p=8, q=2, seed=SEED + i, flags=flags)
        assert st.solve.relres_max <= TOL, (i, st.solve.relres_max)
        Fo, wo = trace[i]["F"], trace[i]["w_new"]
        Fg = F.cpu().numpy()
        dF = np.linalg.norm(Fg - Fo, axis=0) / np.linalg.norm(Fo, axis=0)
        dw = np.linalg.norm(w.cpu().numpy() - wo) / np.linalg.norm(wo)
        assert dF.max() <= 1e-5, (i, dF.max())
        assert dw <= 1e-5, (i, dw)
        moved.append(float(torch.linalg.norm(w - w_before) / torch.linalg.norm(w_before)))
    # the loop really moves w (about 5% per step) and shrinks its support
    assert min(moved) > 0.02, moved
    assert int((w == 0).sum()) > 0
