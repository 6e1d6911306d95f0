"""Python binding of libhgl (include/hgl.h): argument marshalling only.

Every function here checks shapes and dtypes of torch CUDA tensors, passes raw
device pointers, leading dimensions and the current CUDA stream to the C ABI, and
raises HglError on a non-zero status.  All computation happens in the library's
CUDA kernels; there is no fallback: if libhgl.so is missing or fails to load,
``lib()`` raises.
"""
from __future__ import annotations

import ctypes
import os
import re

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libhgl.so")
HEADER = os.path.join(os.path.dirname(_HERE), "include", "hgl.h")

HGL_FP64, HGL_FP32, HGL_BF16 = 0, 1, 2
HGL_SOLVE_WARM_START = 1
HGL_GRAD_DV_FROZEN = 1
HGL_ROUTE_CG, HGL_ROUTE_BR, HGL_ROUTE_BCG = 0, 1, 2
HGL_STEP_GRAPH = 1
HGL_STEP_ACTIVE_SET = 2

STATUS = {
    0: "HGL_OK", -1: "HGL_ERR_INVALID_ARG", -2: "HGL_ERR_INDEX_RANGE", -3: "HGL_ERR_DUPLICATE_MEMBER",
    -4: "HGL_ERR_EMPTY_EDGE", -5: "HGL_ERR_OOM", -6: "HGL_ERR_CUDA", -7: "HGL_ERR_NOT_CONVERGED",
    -8: "HGL_ERR_TIMEOUT", -9: "HGL_ERR_NONFINITE",
}

_DTYPES = {torch.float64: HGL_FP64, torch.float32: HGL_FP32, torch.bfloat16: HGL_BF16}


class HglError(RuntimeError):
    def __init__(self, status: int, message: str):
        self.status = status
        self.name = STATUS.get(status, str(status))
        super().__init__(f"{self.name}: {message}")


class SolveOpts(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("max_iter", ctypes.c_int32), ("dtype", ctypes.c_int32),
                ("inner_tol", ctypes.c_double), ("max_refine", ctypes.c_int32), ("flags", ctypes.c_int32)]


class SolveStats(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("iters", ctypes.c_int32), ("refinements", ctypes.c_int32),
                ("converged", ctypes.c_int32), ("relres_max", ctypes.c_double)]


class StepOpts(ctypes.Structure):
    _fields_ = [("lam", ctypes.c_double), ("mu", ctypes.c_double), ("eta", ctypes.c_double),
                ("route", ctypes.c_int32), ("flags", ctypes.c_int32), ("solve", SolveOpts),
                ("block_ptr", ctypes.POINTER(ctypes.c_int64)), ("nblocks", ctypes.c_int32),
                ("k", ctypes.c_int32), ("p", ctypes.c_int32), ("q", ctypes.c_int32), ("seed", ctypes.c_uint64)]


class StepStats(ctypes.Structure):
    _fields_ = [("solve", SolveStats), ("objective", ctypes.c_double), ("dw_norm", ctypes.c_double)]


_P = ctypes.c_void_p
_I32, _I64, _D, _U64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_uint64

_SIGNATURES = {
    "hgl_status_string": (ctypes.c_char_p, [_I32]),
    "hgl_last_error": (ctypes.c_char_p, []),
    "hgl_version": (_I32, []),
    "hgl_launch_count": (ctypes.c_uint64, []),
    "hgl_profile_enable": (_I32, [_I32]),
    "hgl_profile_read": (_I32, [_I32, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64)]),
    "hgl_build_incidence": (_I32, [_I64, _I64, _P, _P, _I64, _P, ctypes.POINTER(_P)]),
    "hgl_graph_destroy": (None, [_P]),
    "hgl_graph_info": (_I32, [_P, ctypes.POINTER(_I64), ctypes.POINTER(_I64), ctypes.POINTER(_I64)]),
    "hgl_graph_export": (_I32, [_P, _P, _P, _P, _P, _P, _P]),
    "hgl_degrees": (_I32, [_P, _P, _P, _P, _P, _P]),
    "hgl_apply_theta": (_I32, [_P, _P, _D, _D, _P, _I64, _P, _I64, _I32, _I32, _P]),
    "hgl_apply_theta_noalloc": (_I32, [_P, _P, _D, _D, _P, _I64, _P, _I64, _I32, _I32, _P]),
    "hgl_tune_operator": (_I32, [_P, _P, _I32, _I32, ctypes.POINTER(_I32), ctypes.POINTER(_I32),
                                 ctypes.POINTER(_I32), _P]),
    "hgl_cg_solve": (_I32, [_P, _P, _D, _P, _I64, _P, _I64, _I32, _P, ctypes.POINTER(SolveOpts), _P, _P,
                            ctypes.POINTER(SolveStats), _P]),
    "hgl_block_rsvd": (_I32, [_P, _P, _D, ctypes.POINTER(_I64), _I32, _I32, _I32, _I32, _U64, _I32, _P,
                              ctypes.POINTER(_P)]),
    "hgl_precond_destroy": (None, [_P]),
    "hgl_precond_export": (_I32, [_P, _I32, _P, _P, ctypes.POINTER(_I32), _P]),
    "hgl_precond_apply": (_I32, [_P, _P, _I64, _P, _I64, _I32, _I32, _P]),
    "hgl_precond_tensor_cores": (_I32, [_P, _I32, ctypes.POINTER(_I32)]),
    "hgl_set_block_product": (_I32, [_P, _I32]),
    "hgl_block_product": (_I32, [_P, _P, ctypes.POINTER(_I64), _I32, _I32, _P, _I64, _P, _I64, _P]),
    "hgl_schur_inverse": (_I32, [_P, _P, _D, _I64, _I64, _I32, _I32, _I32, _I32, _U64, _I32, _P, _I64, _P]),
    "hgl_tune_block_rsvd": (_I32, [_P, _P, ctypes.POINTER(_I64), _I32, _I32, _I32, _I32, ctypes.POINTER(_I32),
                                   ctypes.POINTER(_D), ctypes.POINTER(_D), _P]),
    "hgl_selftest_wait_timeout": (_I32, [_I64, _P]),
    "hgl_selftest_pair_split": (_I32, [_P, _I64, _P, _P, _P, _P]),
    "hgl_step_precond": (_I32, [_P, _P]),
    "hgl_block_cg_solve": (_I32, [_P, _P, _D, _P, _I64, _P, _I64, _I32, _I32, _D, _I32, _I32, _P, _P, _P]),
    "hgl_weight_grad": (_I32, [_P, _P, _P, _P, _I64, _I32, _I32, _D, _I32, _P, _P]),
    "hgl_project_simplex": (_I32, [_P, _P, _D, _I64, _P]),
    "hgl_active_set_step": (_I32, [_P, _P, _D, _I64, _P]),
    "hgl_adjoint_grad": (_I32, [_P, _P, _D, _P, _P, _P, _I64, _I32, _P, ctypes.POINTER(SolveOpts), _P,
                                ctypes.POINTER(SolveStats), _P]),
    "hgl_laplacian_quadratic": (_I32, [_P, _P, _P, _I64, _P, _I64, _I32, ctypes.POINTER(_D), _P]),
    "hgl_adaptive_step": (_I32, [_P, _P, ctypes.POINTER(StepOpts), _P, _I64, _P, _I64, _I32,
                                 ctypes.POINTER(StepStats), _P]),
}

_LIB = None


def lib() -> ctypes.CDLL:
    """Load libhgl.so (raises if it has not been built)."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_1908_08281_gb300.build.build()")
        handle = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGNATURES.items():
            fn = getattr(handle, name)
            fn.restype = res
            fn.argtypes = args
        _LIB = handle
    return _LIB


def launch_count() -> int:
    """Kernels launched by libhgl in this process so far."""
    return int(lib().hgl_launch_count())


PROF_OPERATOR, PROF_RESIDUAL, PROF_GEMM, PROF_GRADIENT = 0, 1, 2, 3
PROF_PRECOND, PROF_RSVD, PROF_VECTOR, PROF_PROJECT, PROF_OPRESID, PROF_BLOCKSPMM = 4, 5, 6, 7, 8, 9
PROF_SCHUR_GEMM = 10
HGL_BLOCKS_AUTO, HGL_BLOCKS_DENSE, HGL_BLOCKS_SPARSE = 0, 1, 2
PROF_NAMES = {0: "operator apply", 1: "pair-arithmetic residual", 2: "grouped block GEMM (tcgen05)",
              3: "weight gradient", 4: "preconditioner apply", 5: "block rSVD build (all)",
              6: "CG vector kernels", 7: "simplex projection", 8: "residual by one operator pass",
              9: "sparse block products (rSVD)", 10: "Schur-inverse dense products"}


def profile_enable(on: bool = True):
    """Start (clearing totals) or stop recording kernel-family timings."""
    _check(lib().hgl_profile_enable(1 if on else 0))


def profile_read(family: int):
    """(total ms, launches) recorded for a kernel family (synchronises the device)."""
    ms = ctypes.c_double()
    n = ctypes.c_int64()
    _check(lib().hgl_profile_read(family, ctypes.byref(ms), ctypes.byref(n)))
    return ms.value, n.value


def header_functions() -> list[str]:
    """Names of all functions declared in include/hgl.h."""
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(hgl_[a-z0-9_]+)\s*\(", text)))


def _check(status: int):
    if status != 0:
        msg = lib().hgl_last_error().decode(errors="replace")
        raise HglError(status, msg)


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _panel(t: torch.Tensor, name: str):
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dim() != 2 or t.stride(1) != 1:
        raise ValueError(f"{name} must be a row-major 2-D tensor (unit column stride)")
    if t.dtype not in _DTYPES:
        raise ValueError(f"{name} has unsupported dtype {t.dtype}")
    return ctypes.c_void_p(t.data_ptr()), t.stride(0), _DTYPES[t.dtype]


def _vec(t: torch.Tensor, name: str, dtype=torch.float64):
    if t is None:
        return None
    if not t.is_cuda or t.dtype != dtype or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous CUDA {dtype} vector")
    return ctypes.c_void_p(t.data_ptr())


def padded_panel(n: int, c: int, dtype=torch.float64, device="cuda", fill=None) -> torch.Tensor:
    """n x c view of an n x ld buffer with ld * element_size a multiple of 16 bytes."""
    elt = torch.empty((), dtype=dtype).element_size()
    per = 16 // elt
    ld = (c + per - 1) // per * per
    buf = torch.zeros((n, ld), dtype=dtype, device=device) if fill is None else torch.full((n, ld), fill, dtype=dtype, device=device)
    return buf[:, :c]


class Graph:
    """Owner of an hgl_graph handle (device incidence layouts and work buffers)."""

    def __init__(self, handle: int, n: int, m: int, nnz: int):
        self._h = ctypes.c_void_p(handle)
        self.n, self.m, self.nnz = n, m, nnz

    @property
    def handle(self):
        return self._h

    def close(self):
        if self._h and self._h.value:
            lib().hgl_graph_destroy(self._h)
            self._h = ctypes.c_void_p(0)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Precond:
    """Owner of an hgl_precond handle (block rSVD factors)."""

    def __init__(self, handle: int, block_ptr, k: int):
        self._h = ctypes.c_void_p(handle)
        self.block_ptr = list(block_ptr)
        self.k = k

    @property
    def handle(self):
        return self._h

    def close(self):
        if self._h and self._h.value and not getattr(self, "borrowed", False):
            lib().hgl_precond_destroy(self._h)
        self._h = ctypes.c_void_p(0)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def build_incidence(n: int, m: int, edge_ptr, members, stream=None) -> Graph:
    """hgl_build_incidence; edge_ptr (int64, m+1) and members (int32) as torch tensors
    (host or CUDA) or numpy arrays."""
    import numpy as np
    if isinstance(edge_ptr, np.ndarray):
        edge_ptr = torch.from_numpy(np.ascontiguousarray(edge_ptr, dtype=np.int64))
    if isinstance(members, np.ndarray):
        members = torch.from_numpy(np.ascontiguousarray(members, dtype=np.int32))
    edge_ptr = edge_ptr.contiguous()
    members = members.contiguous()
    if edge_ptr.dtype != torch.int64 or members.dtype != torch.int32:
        raise ValueError("edge_ptr must be int64 and members int32")
    out = ctypes.c_void_p()
    _check(lib().hgl_build_incidence(n, m, ctypes.c_void_p(edge_ptr.data_ptr()),
                                     ctypes.c_void_p(members.data_ptr()) if members.numel() else None,
                                     members.numel(), _stream(stream), ctypes.byref(out)))
    return Graph(out.value, n, m, members.numel())


def graph_export(g: Graph, stream=None):
    dev = torch.device("cuda")
    out = {
        "csc_ptr": torch.empty(g.m + 1, dtype=torch.int64, device=dev),
        "csc_idx": torch.empty(max(g.nnz, 1), dtype=torch.int32, device=dev),
        "csr_ptr": torch.empty(g.n + 1, dtype=torch.int64, device=dev),
        "csr_idx": torch.empty(max(g.nnz, 1), dtype=torch.int32, device=dev),
        "de": torch.empty(g.m, dtype=torch.int32, device=dev),
    }
    _check(lib().hgl_graph_export(g.handle, *[ctypes.c_void_p(out[k].data_ptr()) for k in
                                              ("csc_ptr", "csc_idx", "csr_ptr", "csr_idx", "de")], _stream(stream)))
    out["csc_idx"] = out["csc_idx"][:g.nnz]
    out["csr_idx"] = out["csr_idx"][:g.nnz]
    return out


def degrees(g: Graph, w: torch.Tensor, stream=None):
    dev = w.device
    dv = torch.empty(g.n, dtype=torch.float64, device=dev)
    s = torch.empty(g.n, dtype=torch.float64, device=dev)
    t = torch.empty(g.m, dtype=torch.float64, device=dev)
    _check(lib().hgl_degrees(g.handle, _vec(w, "w"), _vec(dv, "dv"), _vec(s, "s"), _vec(t, "t"), _stream(stream)))
    return dv, s, t


def apply_theta(g: Graph, w: torch.Tensor, X: torch.Tensor, a: float = 0.0, b: float = 1.0,
                Z: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """Z = a X + b Theta(w) X (Eq. 1)."""
    n, c = X.shape
    if Z is None:
        Z = padded_panel(n, c, X.dtype, X.device)
    px, ldx, dt = _panel(X, "X")
    pz, ldz, dtz = _panel(Z, "Z")
    if dt != dtz:
        raise ValueError("X and Z must have the same dtype")
    _check(lib().hgl_apply_theta(g.handle, _vec(w, "w"), a, b, px, ldx, pz, ldz, c, dt, _stream(stream)))
    return Z


def apply_theta_noalloc(g: Graph, w: torch.Tensor, X: torch.Tensor, Z: torch.Tensor, a: float = 0.0,
                        b: float = 1.0, stream=None) -> torch.Tensor:
    """Z = a X + b Theta(w) X without any device allocation in the call (Z is required)."""
    n, c = X.shape
    px, ldx, dt = _panel(X, "X")
    pz, ldz, dtz = _panel(Z, "Z")
    if dt != dtz:
        raise ValueError("X and Z must have the same dtype")
    _check(lib().hgl_apply_theta_noalloc(g.handle, _vec(w, "w"), a, b, px, ldx, pz, ldz, c, dt, _stream(stream)))
    return Z


def tune_operator(g: Graph, w: torch.Tensor, c: int, dtype: int = HGL_FP64,
                  stream=None) -> tuple[int, int, int]:
    """Time the supported column chunks of the operator (and, for FP32/BF16, of the
    pair residual) on this graph for c-column panels, then the grid of its gather
    passes; the graph keeps the fastest.  Returns (operator chunk, residual chunk) in
    columns and the grid policy (0 = one wave of resident blocks, 1 = eight per SM)."""
    op = ctypes.c_int32(0)
    pair = ctypes.c_int32(0)
    grid = ctypes.c_int32(0)
    _check(lib().hgl_tune_operator(g.handle, _vec(w, "w"), c, dtype, ctypes.byref(op), ctypes.byref(pair),
                                   ctypes.byref(grid), _stream(stream)))
    return op.value, pair.value, grid.value


def cg_solve(g: Graph, w: torch.Tensor, lam: float, Y: torch.Tensor, F: torch.Tensor | None = None,
             tol: float = 1e-10, max_iter: int = 1000, dtype: int = HGL_FP64, inner_tol: float = 0.0,
             max_refine: int = 0, warm_start: bool = False, precond: Precond | None = None,
             stream=None, raise_on_fail: bool = True):
    """Solve M F = lam Y (Eq. 6); returns (F, relres[c], iters[c], stats)."""
    n, c = Y.shape
    if F is None:
        F = padded_panel(n, c, torch.float64, Y.device)
    py, ldy, dty = _panel(Y, "Y")
    pf, ldf, dtf = _panel(F, "F")
    if dty != HGL_FP64 or dtf != HGL_FP64:
        raise ValueError("Y and F must be float64")
    relres = torch.empty(c, dtype=torch.float64, device=Y.device)
    iters = torch.empty(c, dtype=torch.int32, device=Y.device)
    opts = SolveOpts(tol, max_iter, dtype, inner_tol, max_refine, HGL_SOLVE_WARM_START if warm_start else 0)
    stats = SolveStats()
    st = lib().hgl_cg_solve(g.handle, _vec(w, "w"), lam, py, ldy, pf, ldf, c,
                            precond.handle if precond is not None else None, ctypes.byref(opts),
                            ctypes.c_void_p(relres.data_ptr()), ctypes.c_void_p(iters.data_ptr()),
                            ctypes.byref(stats), _stream(stream))
    if st != 0 and (raise_on_fail or st not in (-7, -9)):
        _check(st)
    return F, relres, iters, stats


def block_cg_solve(g: Graph, w: torch.Tensor, lam: float, Y: torch.Tensor, s: int, F: torch.Tensor | None = None,
                   tol: float = 1e-10, max_iter: int = 1000, warm_start: bool = False, stream=None,
                   raise_on_fail: bool = True):
    """Block CG with a shared Krylov space over groups of s columns (FP64); returns
    (F, relres[c], iters[ceil(c/s)], status)."""
    n, c = Y.shape
    if F is None:
        F = padded_panel(n, c, torch.float64, Y.device)
    py, ldy, dty = _panel(Y, "Y")
    pf, ldf, dtf = _panel(F, "F")
    if dty != HGL_FP64 or dtf != HGL_FP64:
        raise ValueError("Y and F must be float64")
    relres = torch.empty(c, dtype=torch.float64, device=Y.device)
    # one entry per group; an invalid s (rejected by the library) still gets a buffer
    iters = torch.empty(max(1, (c + s - 1) // s) if s >= 1 else 1, dtype=torch.int32, device=Y.device)
    st = lib().hgl_block_cg_solve(g.handle, _vec(w, "w"), lam, py, ldy, pf, ldf, c, s, tol, max_iter,
                                  HGL_SOLVE_WARM_START if warm_start else 0, ctypes.c_void_p(relres.data_ptr()),
                                  ctypes.c_void_p(iters.data_ptr()), _stream(stream))
    if st != 0 and (raise_on_fail or st not in (-7, -9)):
        _check(st)
    return F, relres, iters, st


def block_rsvd(g: Graph, w: torch.Tensor, lam: float, block_ptr, k: int, p: int, q: int, seed: int,
               gemm_dtype: int = HGL_BF16, stream=None) -> Precond:
    """Block randomized SVD preconditioner (Section 3, Algorithm 1)."""
    bp = (ctypes.c_int64 * len(block_ptr))(*[int(x) for x in block_ptr])
    out = ctypes.c_void_p()
    _check(lib().hgl_block_rsvd(g.handle, _vec(w, "w"), lam, bp, len(block_ptr) - 1, k, p, q, seed, gemm_dtype,
                                _stream(stream), ctypes.byref(out)))
    return Precond(out.value, block_ptr, k)


def step_precond(g: Graph, block_ptr, k: int) -> Precond:
    """The preconditioner the graph's captured block-rSVD step built in its last call
    (owned by the graph: valid until the next adaptive_step call; never destroyed here)."""
    h = ctypes.c_void_p()
    _check(lib().hgl_step_precond(g.handle, ctypes.byref(h)))
    P = Precond(h.value, block_ptr, k)
    P.borrowed = True
    return P


def precond_export(P: Precond, b: int, stream=None):
    size = P.block_ptr[b + 1] - P.block_ptr[b]
    Q = torch.zeros((size, P.k), dtype=torch.float64, device="cuda")
    ev = torch.zeros(P.k, dtype=torch.float64, device="cuda")
    kb = ctypes.c_int32()
    _check(lib().hgl_precond_export(P.handle, b, ctypes.c_void_p(Q.data_ptr()), ctypes.c_void_p(ev.data_ptr()),
                                    ctypes.byref(kb), _stream(stream)))
    return Q[:, :kb.value], ev[:kb.value]


def precond_apply(P: Precond, R: torch.Tensor, Z: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    n, c = R.shape
    if Z is None:
        Z = padded_panel(n, c, R.dtype, R.device)
    pr, ldr, dt = _panel(R, "R")
    pz, ldz, _ = _panel(Z, "Z")
    _check(lib().hgl_precond_apply(P.handle, pr, ldr, pz, ldz, c, dt, _stream(stream)))
    return Z


def block_product(g: Graph, w: torch.Tensor, block_ptr, S: torch.Tensor, stream=None) -> torch.Tensor:
    """D_b = Theta_bb S_b per diagonal block (Algorithm 1's products, BF16 route)."""
    if S.dtype != torch.float32 or S.stride(1) != 1:
        raise ValueError("S must be a row-major float32 panel")
    n, l = S.shape
    D = torch.empty((n, l), dtype=torch.float32, device=S.device)
    bp = (ctypes.c_int64 * len(block_ptr))(*[int(x) for x in block_ptr])
    _check(lib().hgl_block_product(g.handle, _vec(w, "w"), bp, len(block_ptr) - 1, l,
                                   ctypes.c_void_p(S.data_ptr()), S.stride(0), ctypes.c_void_p(D.data_ptr()),
                                   D.stride(0), _stream(stream)))
    return D


def schur_inverse(g: Graph, w: torch.Tensor, lam: float, row0: int, nrows: int, r_min: int, k: int, p: int,
                  q: int, seed: int, dtype: int = HGL_FP32, stream=None) -> torch.Tensor:
    """Dense approximate inverse of M on [row0, row0 + nrows) by the nested Schur scheme."""
    out = torch.empty((nrows, nrows), dtype=torch.float64, device=w.device)
    _check(lib().hgl_schur_inverse(g.handle, _vec(w, "w"), lam, row0, nrows, r_min, k, p, q, seed, dtype,
                                   ctypes.c_void_p(out.data_ptr()), nrows, _stream(stream)))
    return out


def tune_block_rsvd(g: Graph, w: torch.Tensor, block_ptr, k: int, p: int, q: int, stream=None):
    """Time the block rSVD's product routes on this graph and keep the faster;
    returns (route, ms_dense, ms_sparse)."""
    bp = (ctypes.c_int64 * len(block_ptr))(*[int(x) for x in block_ptr])
    route, md, ms = ctypes.c_int32(), ctypes.c_double(), ctypes.c_double()
    _check(lib().hgl_tune_block_rsvd(g.handle, _vec(w, "w"), bp, len(block_ptr) - 1, k, p, q, ctypes.byref(route),
                                     ctypes.byref(md), ctypes.byref(ms), _stream(stream)))
    return route.value, md.value, ms.value


def selftest_pair_split(x: torch.Tensor, stream=None):
    """(hi, lo, back) of the mixed solver's FP64 <-> FP32-pair conversions on x (FP64)."""
    x = x.contiguous()
    if x.dtype != torch.float64 or not x.is_cuda:
        raise ValueError("x must be a CUDA float64 tensor")
    hi = torch.empty(x.shape, dtype=torch.float32, device=x.device)
    lo = torch.empty_like(hi)
    back = torch.empty_like(x)
    _check(lib().hgl_selftest_pair_split(ctypes.c_void_p(x.data_ptr()), x.numel(), ctypes.c_void_p(hi.data_ptr()),
                                         ctypes.c_void_p(lo.data_ptr()), ctypes.c_void_p(back.data_ptr()),
                                         _stream(stream)))
    return hi, lo, back


def selftest_wait_timeout(limit_cycles: int, stream=None):
    """Run the kernels' bounded device wait against a barrier nothing arrives on; raises
    HglError with status HGL_ERR_TIMEOUT (the expected outcome)."""
    _check(lib().hgl_selftest_wait_timeout(int(limit_cycles), _stream(stream)))


def set_block_product(g: Graph, mode: int):
    """Route of the block rSVD's products Theta_bb S for later builds on g:
    HGL_BLOCKS_DENSE (tcgen05 GEMM on dense BF16 blocks), HGL_BLOCKS_SPARSE (from the
    incidence lists) or HGL_BLOCKS_AUTO (by the blocks' fill)."""
    _check(lib().hgl_set_block_product(g.handle, mode))


def precond_tensor_cores(P: Precond, on: bool) -> bool:
    """Select the TF32 tensor-core apply (split operands, FP32 accuracy) or the FP32
    CUDA-core apply for FP32 panels; returns whether P supports the tensor-core one."""
    active = ctypes.c_int32(0)
    _check(lib().hgl_precond_tensor_cores(P.handle, 1 if on else 0, ctypes.byref(active)))
    return bool(active.value)


def weight_grad(g: Graph, w: torch.Tensor, F: torch.Tensor, mu: float = 0.0, Z: torch.Tensor | None = None,
                dv_frozen: bool = False, stream=None) -> torch.Tensor:
    """grad = -d tr(Z^T Theta F)/dw + 2 mu w (Z = F: grad of P(w), Eq. 4)."""
    n, c = F.shape
    pf, ld, dt = _panel(F, "F")
    pz = None
    if Z is not None:
        pz, ldz, dtz = _panel(Z, "Z")
        if ldz != ld or dtz != dt:
            raise ValueError("Z must match F's dtype and leading dimension")
    grad = torch.empty(g.m, dtype=torch.float64, device=F.device)
    _check(lib().hgl_weight_grad(g.handle, _vec(w, "w"), pf, pz, ld, c, dt, mu,
                                 HGL_GRAD_DV_FROZEN if dv_frozen else 0, ctypes.c_void_p(grad.data_ptr()),
                                 _stream(stream)))
    return grad


def adjoint_grad(g: Graph, w: torch.Tensor, lam: float, F: torch.Tensor, G: torch.Tensor,
                 Z: torch.Tensor | None = None, tol: float = 1e-10, max_iter: int = 1000, dtype: int = HGL_FP64,
                 inner_tol: float = 0.0, max_refine: int = 0, precond: Precond | None = None, stream=None,
                 raise_on_fail: bool = True):
    """<G, dF/dw> for F = M(w)^-1 lam Y by the adjoint method: solves M Z = G and returns
    (grad[m], Z, stats) with grad_e = d/dw_e tr(Z^T Theta F)."""
    n, c = F.shape
    pf, ld, dtf = _panel(F, "F")
    pg, ldg, dtg = _panel(G, "G")
    if Z is None:
        Z = padded_panel(n, c, torch.float64, F.device)
    pz, ldz, dtz = _panel(Z, "Z")
    if dtf != HGL_FP64 or dtg != HGL_FP64 or dtz != HGL_FP64 or not (ld == ldg == ldz):
        raise ValueError("F, G and Z must be float64 panels with one leading dimension")
    grad = torch.empty(g.m, dtype=torch.float64, device=F.device)
    opts = SolveOpts(tol, max_iter, dtype, inner_tol, max_refine, 0)
    stats = SolveStats()
    st = lib().hgl_adjoint_grad(g.handle, _vec(w, "w"), lam, pf, pg, pz, ld, c,
                                precond.handle if precond is not None else None, ctypes.byref(opts),
                                ctypes.c_void_p(grad.data_ptr()), ctypes.byref(stats), _stream(stream))
    if st != 0 and (raise_on_fail or st not in (-7,)):
        _check(st)
    return grad, Z, stats


def active_set_step(w: torch.Tensor, grad: torch.Tensor, eta: float, stream=None) -> torch.Tensor:
    """In place: the active-set steepest-descent step of Eq. 5 (pinned zeros stay 0)."""
    _check(lib().hgl_active_set_step(_vec(w, "w"), _vec(grad, "grad"), eta, w.numel(), _stream(stream)))
    return w


def project_simplex(w: torch.Tensor, grad: torch.Tensor | None, eta: float, stream=None) -> torch.Tensor:
    """In place: w <- projection of w - eta grad onto the simplex (Eq. 5)."""
    _check(lib().hgl_project_simplex(_vec(w, "w"), _vec(grad, "grad") if grad is not None else None, eta,
                                     w.numel(), _stream(stream)))
    return w


def laplacian_quadratic(g: Graph, w: torch.Tensor, F: torch.Tensor, DF: torch.Tensor | None = None, stream=None):
    """tr(F^T Delta F) and Delta F (Eq. 1, Eq. 4); returns (value, DF)."""
    n, c = F.shape
    if DF is None:
        DF = padded_panel(n, c, torch.float64, F.device)
    pf, ldf, dtf = _panel(F, "F")
    pd, ldd, dtd = _panel(DF, "DF")
    if dtf != HGL_FP64 or dtd != HGL_FP64:
        raise ValueError("F and DF must be float64")
    val = ctypes.c_double()
    _check(lib().hgl_laplacian_quadratic(g.handle, _vec(w, "w"), pf, ldf, pd, ldd, c, ctypes.byref(val),
                                         _stream(stream)))
    return val.value, DF


def adaptive_step(g: Graph, w: torch.Tensor, Y: torch.Tensor, F: torch.Tensor, lam: float, mu: float = 0.0,
                  eta: float = 1e-2, tol: float = 1e-10, max_iter: int = 1000, dtype: int = HGL_FP64,
                  inner_tol: float = 0.0, route: int = HGL_ROUTE_CG, block_ptr=None, k: int = 0, p: int = 0,
                  q: int = 0, seed: int = 0, flags: int = 0, stream=None, raise_on_fail: bool = True):
    """One outer iteration (solve at w, then projected gradient step); F and w in place."""
    n, c = Y.shape
    py, ldy, _ = _panel(Y, "Y")
    pf, ldf, _ = _panel(F, "F")
    bp = None
    nb = 0
    if block_ptr is not None:
        bp = (ctypes.c_int64 * len(block_ptr))(*[int(x) for x in block_ptr])
        nb = len(block_ptr) - 1
    opts = StepOpts(lam, mu, eta, route, flags, SolveOpts(tol, max_iter, dtype, inner_tol, 0, 0),
                    ctypes.cast(bp, ctypes.POINTER(ctypes.c_int64)) if bp is not None else None, nb, k, p, q, seed)
    stats = StepStats()
    st = lib().hgl_adaptive_step(g.handle, _vec(w, "w"), ctypes.byref(opts), py, ldy, pf, ldf, c,
                                 ctypes.byref(stats), _stream(stream))
    if st != 0 and (raise_on_fail or st != -7):
        _check(st)
    return stats
