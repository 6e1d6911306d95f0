// cg.cu -- hgl_cg_solve: the ranking system M F = lam Y (Eqs. 3 and 6, multiplied by
// 1 + lam) solved by conjugate gradient (Eqs. 16-20), one independent recurrence per
// right-hand-side column.
//
// FP64 mode runs the recurrences on FP64 panels.  Mixed modes keep the solution F in
// FP64 and run iterative refinement: the residual lam Y - M F is recomputed from F in
// FP64, a CG on FP32 (or BF16 search-direction) panels with FP32 arithmetic solves
// M D = R to a loose relative tolerance, and F += D.  The per-column scalars
// (alpha, beta, r^T r, stopping tests) are always FP64.
#include <algorithm>
#include <cmath>
#include <vector>

#include "precond.cuh"
#include "solver.cuh"
#include "vec_kernels.cuh"

namespace hgl {

namespace {

inline int pow2_at_least(int v) {
  int p = 1;
  while (p < v) p <<= 1;
  return p;
}

inline size_t align256(size_t b) { return (b + 255) & ~static_cast<size_t>(255); }

}  // namespace

VecGrid vec_grid(const hgl_graph* g, int c, int elt) {
  VecGrid vg;
  const int E = 16 / elt;
  const int vecs = (c + E - 1) / E;
  vg.lg = std::min(32, pow2_at_least(vecs));
  const int G = 32 / vg.lg;
  const int64_t rows_per_block = (int64_t)(VEC_THREADS / 32) * G;
  int64_t need = (g->n + rows_per_block - 1) / rows_per_block;
  int64_t cap = (int64_t)g->num_sms * 4;
  vg.gx = (int)std::max<int64_t>(1, std::min(need, cap));
  vg.gy = (c + vg.lg * E - 1) / (vg.lg * E);
  return vg;
}

#define HGL_LG_SWITCH(lg, CALL) \
  switch (lg) {                 \
    case 1: { constexpr int LG = 1; CALL; } break;   \
    case 2: { constexpr int LG = 2; CALL; } break;   \
    case 4: { constexpr int LG = 4; CALL; } break;   \
    case 8: { constexpr int LG = 8; CALL; } break;   \
    case 16: { constexpr int LG = 16; CALL; } break; \
    default: { constexpr int LG = 32; CALL; } break; \
  }

template <class TA, class TB>
hgl_status panel_dot(const hgl_graph* g, int c, const TA* A, int64_t lda, const TB* B, int64_t ldb, double scale,
                     double* partials, cudaStream_t st, int* rows, const int32_t* run_flag = nullptr) {
  VecGrid vg = vec_grid(g, c, sizeof(TA));
  dim3 grid(vg.gx, vg.gy);
  HGL_PROFILED(HGL_PROF_VECTOR, hgl::count_launch(); HGL_LG_SWITCH(vg.lg, (k_panel_dot<TA, TB, LG><<<grid, VEC_THREADS, 0, st>>>(g->n, c, A, lda, B, ldb, scale, partials, run_flag))));
  HGL_CHECK_CUDA(cudaGetLastError());
  *rows = vg.gx;
  return HGL_OK;
}

template <class TX, class TZ, bool DOT>
hgl_status panel_scale(const hgl_graph* g, int c, const TX* X, int64_t ldx, double scale, TZ* Z, int64_t ldz,
                       double* partials, cudaStream_t st, int* rows, const int32_t* run_flag = nullptr) {
  VecGrid vg = vec_grid(g, c, sizeof(TZ));
  dim3 grid(vg.gx, vg.gy);
  HGL_PROFILED(HGL_PROF_VECTOR, hgl::count_launch(); HGL_LG_SWITCH(vg.lg, (k_panel_scale<TX, TZ, LG, DOT><<<grid, VEC_THREADS, 0, st>>>(g->n, c, X, ldx, scale, Z, ldz, partials, run_flag))));
  HGL_CHECK_CUDA(cudaGetLastError());
  if (rows) *rows = vg.gx;
  return HGL_OK;
}

template <int MODE>
hgl_status cg_reduce(const double* pa, const double* pb, int rows, const CgState& S, cudaStream_t st) {
  hgl::count_launch(); k_cg_reduce<MODE><<<(S.c + 7) / 8, 256, 0, st>>>(pa, pb, rows, S);
  HGL_CHECK_CUDA(cudaGetLastError());
  return HGL_OK;
}

__global__ void k_set_target(CgState S, double tol2) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < S.c; j += gridDim.x * blockDim.x) {
    S.target[j] = tol2 * S.b2[j];
    S.bad[j] = 0;
  }
}

// Inner-solve targets of a refinement sweep: columns already at tol are frozen
// (target +inf); the others aim at rr_inner <= rel^2 rr_true, rel = max(inner_tol,
// INNER_MARGIN tol / relres): three quarters of what the outer tolerance still needs.
// The last quarter covers what the recursive FP32 residual does not see -- the
// rounding of the correction and of F's FP32 pair (a few units of 2^-24 of ||lam Y||),
// and the error of an FP32 first-residual estimate -- so that another sweep (a
// pair-arithmetic residual and a CG restart) is rarely needed, without solving past
// the tolerance (measured at n = 1M, c = 512, tol 3e-6: final relres at most 2.25e-6,
// no second sweep in 20 outer iterations; a half margin took 0.25 more iterations per
// solve).  Also sets *S.need = 1 when some column needs the sweep (captured solves zero
// it before this kernel and guard the sweep's expensive launches with it).
constexpr double INNER_MARGIN = 0.75;

__global__ void k_inner_targets(CgState S, double tol, double inner_tol) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < S.c; j += gridDim.x * blockDim.x) {
    const double rel = S.relres[j];
    if (!(S.b2[j] > 0.0) || !(rel > tol) || !isfinite(rel)) {
      S.target[j] = INFINITY;
    } else {
      double want = fmax(inner_tol, INNER_MARGIN * tol / rel);
      S.target[j] = want * want * S.rr[j];
      *S.need = 1;
    }
  }
}

hgl_status solver_layout(hgl_graph* g, int c, int mode, bool precond, SolverMem* sm) {
  const int64_t n = g->n;
  sm->c = c;
  sm->ld64 = (c + 1) / 2 * 2;
  sm->ld32 = (c + 3) / 4 * 4;
  sm->ld16 = (c + 7) / 8 * 8;
  size_t bytes = 0;
  auto take = [&](size_t b) {
    size_t off = bytes;
    bytes += align256(b);
    return off;
  };
  size_t oR, oP, oQ, oZ, oX = 0;
  if (mode == HGL_FP64) {
    oR = take(sizeof(double) * n * sm->ld64);
    oP = take(sizeof(double) * n * sm->ld64);
    oQ = take(sizeof(double) * n * sm->ld64);
    oZ = precond ? take(sizeof(double) * n * sm->ld64) : 0;
  } else {
    oR = take(sizeof(float) * n * sm->ld32);
    oP = mode == HGL_BF16 ? take(sizeof(uint16_t) * n * sm->ld16) : take(sizeof(float) * n * sm->ld32);
    oQ = take(sizeof(float) * n * sm->ld32);
    oZ = precond ? take(sizeof(float) * n * sm->ld32) : 0;
    oX = take(sizeof(float) * n * sm->ld32);
  }
  size_t oFh = 0, oFl = 0, oFl16 = 0, oSc = 0;
  if (mode != HGL_FP64) {
    oFh = take(sizeof(float) * n * sm->ld32);
    oFl = take(sizeof(float) * n * sm->ld32);
    oFl16 = take(sizeof(uint16_t) * n * sm->ld16);
    oSc = take(sizeof(float) * 2 * (size_t)(g->n + g->m));
  }
  size_t oVec = take(sizeof(double) * 8 * (size_t)c);
  size_t oInt = take(sizeof(int32_t) * 4 * (size_t)c + 64);
  hgl_status stt = HGL_OK;
  char* base = static_cast<char*>(buffer_get(g->solver, bytes, &stt));
  if (!base) return stt;
  sm->R = base + oR;
  sm->P = base + oP;
  sm->Q = base + oQ;
  sm->Z = precond ? base + oZ : nullptr;
  sm->X = mode == HGL_FP64 ? nullptr : base + oX;
  if (mode != HGL_FP64) {
    sm->Fh = reinterpret_cast<float*>(base + oFh);
    sm->Fl = reinterpret_cast<float*>(base + oFl);
    sm->Fl16 = reinterpret_cast<bf16_t*>(base + oFl16);
    sm->s_hi = reinterpret_cast<float*>(base + oSc);
    sm->s_lo = sm->s_hi + g->n;
    sm->t_hi = sm->s_lo + g->n;
    sm->t_lo = sm->t_hi + g->m;
  }
  double* v = reinterpret_cast<double*>(base + oVec);
  CgState& S = sm->S;
  S.c = c;
  S.b2 = v;
  S.rr = v + c;
  S.rz = v + 2 * c;
  S.alpha = v + 3 * c;
  S.beta = v + 4 * c;
  S.target = v + 5 * c;
  S.relres = v + 6 * c;
  int32_t* iv = reinterpret_cast<int32_t*>(base + oInt);
  S.active = iv;
  S.iters = iv + c;
  S.bad = iv + 2 * c;
  S.run_flag = iv + 3 * c;
  S.done = reinterpret_cast<unsigned*>(iv + 3 * c + 4);
  S.need = iv + 3 * c + 8;
  sm->int_bytes = sizeof(int32_t) * 4 * (size_t)c + 64;
  sm->int_base = iv;
  // partials: two arrays of max(rows) x c
  const int rows = solver_partial_rows(g);
  double* pa = static_cast<double*>(buffer_get(g->partials, sizeof(double) * 2 * (size_t)rows * c, &stt));
  if (!pa) return stt;
  sm->pa = pa;
  sm->pb = pa + (size_t)rows * c;
  return HGL_OK;
}

int solver_partial_rows(const hgl_graph* g) { return std::max(op_partial_rows(g), g->num_sms * 4); }

// One CG iteration (Eqs. 16-20) on panels of type TP (search direction) / TV (others).
template <class TP, class TV>
hgl_status cg_iteration(hgl_graph* g, const SolverMem& sm, double lam, TV* Xs, int64_t ldx, int xdt, int vdt,
                        const hgl_precond* P, cudaStream_t st) {
  const CgState& S = sm.S;
  const int c = sm.c;
  const int64_t ldp = xdt == HGL_FP64 ? sm.ld64 : (xdt == HGL_BF16 ? sm.ld16 : sm.ld32);
  const int64_t ldv = vdt == HGL_FP64 ? sm.ld64 : sm.ld32;
  OpCall cl{};
  cl.g = g;
  cl.xdt = xdt;
  cl.zdt = vdt;
  cl.X = sm.P;
  cl.ldx = ldp;
  cl.Z = sm.Q;
  cl.ldz = ldv;
  cl.c = c;
  cl.a = 1.0 + lam;
  cl.b = -1.0;
  cl.epi = EPI_DOT_XZ;
  cl.partials = sm.pa;
  cl.run_flag = S.run_flag;
  cl.chunk_cols = g->chunk_cols;
  int rows = 0;
  HGL_TRY(op_launch(cl, st, &rows));
  HGL_TRY(cg_reduce<RED_ALPHA>(sm.pa, nullptr, rows, S, st));
  VecGrid vg = vec_grid(g, c, sizeof(TV));
  dim3 grid(vg.gx, vg.gy);
  HGL_PROFILED(HGL_PROF_VECTOR, hgl::count_launch(); HGL_LG_SWITCH(vg.lg, (k_cg_update_xr<TP, TV, LG><<<grid, VEC_THREADS, 0, st>>>(
                           g->n, c, static_cast<const TP*>(sm.P), ldp, static_cast<const TV*>(sm.Q), ldv, Xs, ldx,
                           static_cast<TV*>(sm.R), ldv, S.alpha, sm.pa, S.run_flag))));
  HGL_CHECK_CUDA(cudaGetLastError());
  const TV* zsrc = static_cast<const TV*>(sm.R);
  int rows_b = 0;
  if (P) {
    HGL_TRY(precond_apply_launch(P, g, sm.R, ldv, sm.Z, ldv, c, vdt, sm.pb, st, &rows_b, S.run_flag));
    zsrc = static_cast<const TV*>(sm.Z);
  }
  HGL_TRY(cg_reduce_beta(sm.pa, vg.gx, P ? sm.pb : nullptr, rows_b, S, st));
  HGL_PROFILED(HGL_PROF_VECTOR, hgl::count_launch(); HGL_LG_SWITCH(vg.lg, (k_cg_update_p<TP, TV, LG><<<grid, VEC_THREADS, 0, st>>>(
                           g->n, c, zsrc, ldv, static_cast<TP*>(sm.P), ldp, S.beta, S.run_flag))));
  HGL_CHECK_CUDA(cudaGetLastError());
  return HGL_OK;
}

hgl_status cg_reduce_beta(double* pa, int rows_a, double* pb, int rows_b, const CgState& S, cudaStream_t st) {
  if (!pb || rows_b == rows_a) return cg_reduce<RED_BETA>(pa, pb, rows_a, S, st);
  // rows differ: pad the shorter array with zeros (pb may be padded in place since it
  // is sized for the maximum row count)
  const int rows = std::max(rows_a, rows_b);
  const int c = S.c;
  if (rows_b < rows) {
    HGL_CHECK_CUDA(cudaMemsetAsync(pb + (size_t)rows_b * c, 0, sizeof(double) * (size_t)(rows - rows_b) * c, st));
  } else {
    HGL_CHECK_CUDA(cudaMemsetAsync(pa + (size_t)rows_a * c, 0, sizeof(double) * (size_t)(rows - rows_a) * c, st));
  }
  return cg_reduce<RED_BETA>(pa, pb, rows, S, st);
}

template <class TP, class TV>
hgl_status run_cg_loop(hgl_graph* g, const SolverMem& sm, double lam, TV* Xs, int64_t ldx, int xdt, int vdt,
                       const hgl_precond* P, int max_iter, int first_batch, cudaStream_t st, int* done_iters) {
  int it = 0;
  int32_t flag = 1;
  // Small problems launch a Chebyshev-bound batch of iterations between host checks
  // (kernels of converged iterations return at once); large ones check after every
  // iteration, where one host round trip is negligible next to an iteration.
  const bool large = (double)g->n * sm.c >= (double)(1 << 24);
  int batch = large ? 1 : std::max(1, std::min(first_batch, max_iter));
  while (it < max_iter) {
    const int todo = std::min(batch, max_iter - it);
    for (int k = 0; k < todo; ++k) HGL_TRY((cg_iteration<TP, TV>(g, sm, lam, Xs, ldx, xdt, vdt, P, st)));
    it += todo;
    HGL_CHECK_CUDA(cudaMemcpyAsync(&flag, sm.S.run_flag, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    HGL_CHECK_CUDA(cudaStreamSynchronize(st));
    if (flag == 0) break;
    batch = large ? 1 : 4;
  }
  *done_iters = it;
  return HGL_OK;
}

// Chebyshev bound for kappa(M) <= (1+lam)/lam, reduction `tol` (+2 for rounding).
int cg_iteration_bound(double lam, double tol) {
  if (!(lam > 0) || !(tol > 0) || tol >= 1) return 8;
  const double kappa = (1.0 + lam) / lam;
  const double rate = (std::sqrt(kappa) + 1.0) / (std::sqrt(kappa) - 1.0);
  return (int)std::ceil(std::log(2.0 / tol) / std::log(rate)) + 2;
}

hgl_status true_residual(hgl_graph* g, const SolverMem& sm, double lam, double gy, const double* Y, int64_t ldy,
                         const double* F, int64_t ldf, void* Rout, int rdt, int64_t ldr, cudaStream_t st) {
  OpCall cl{};
  cl.g = g;
  cl.xdt = HGL_FP64;
  cl.zdt = rdt;
  cl.X = F;
  cl.ldx = ldf;
  cl.Z = Rout;
  cl.ldz = ldr;
  cl.c = sm.c;
  cl.a = -(1.0 + lam);
  cl.b = 1.0;
  cl.epi = EPI_RESID;
  cl.Y = Y;
  cl.ldy = ldy;
  cl.gy = gy;
  cl.partials = sm.pa;
  cl.chunk_cols = g->chunk_cols;
  int rows = 0;
  HGL_TRY(op_launch(cl, st, &rows));
  return cg_reduce<RED_RESID>(sm.pa, nullptr, rows, sm.S, st);
}

hgl_status fill_stats(const CgState& S, int c, int refinements, double tol, double* relres_out,
                      int32_t* iters_out, hgl_solve_stats* stats, cudaStream_t st, hgl_status* verdict) {
  if (relres_out)
    HGL_CHECK_CUDA(cudaMemcpyAsync(relres_out, S.relres, sizeof(double) * c, cudaMemcpyDeviceToDevice, st));
  if (iters_out)
    HGL_CHECK_CUDA(cudaMemcpyAsync(iters_out, S.iters, sizeof(int32_t) * c, cudaMemcpyDeviceToDevice, st));
  std::vector<double> rel(c);
  std::vector<int32_t> bad(c), its(c);
  HGL_CHECK_CUDA(cudaMemcpyAsync(rel.data(), S.relres, sizeof(double) * c, cudaMemcpyDeviceToHost, st));
  HGL_CHECK_CUDA(cudaMemcpyAsync(bad.data(), S.bad, sizeof(int32_t) * c, cudaMemcpyDeviceToHost, st));
  HGL_CHECK_CUDA(cudaMemcpyAsync(its.data(), S.iters, sizeof(int32_t) * c, cudaMemcpyDeviceToHost, st));
  HGL_CHECK_CUDA(cudaStreamSynchronize(st));
  int max_it = 0;
  for (int j = 0; j < c; ++j) max_it = std::max(max_it, (int)its[j]);
  int conv = 0, nbad = 0;
  double mx = 0.0;
  for (int j = 0; j < c; ++j) {
    if (!std::isfinite(rel[j])) nbad++;
    if (rel[j] <= tol) conv++;
    if (rel[j] > mx || !std::isfinite(rel[j])) mx = rel[j];
    if (bad[j] && !(rel[j] <= tol)) nbad++;
  }
  hgl_status v = HGL_OK;
  if (nbad > 0) v = record_error(HGL_ERR_NONFINITE, "non-finite value or CG breakdown in %d column(s)", nbad);
  else if (conv < c) v = record_error(HGL_ERR_NOT_CONVERGED, "%d of %d columns missed the tolerance", c - conv, c);
  if (stats) {
    stats->status = v;
    stats->iters = max_it;
    stats->refinements = refinements;
    stats->converged = conv;
    stats->relres_max = mx;
  }
  *verdict = v;
  return HGL_OK;
}

hgl_status cg_solve_impl(hgl_graph* g, const double* w, double lam, double gy, const double* Y, int64_t ldy, double* F,
                         int64_t ldf, int c, const hgl_precond* P, const hgl_solve_opts& o, double* relres_out,
                         int32_t* iters_out, hgl_solve_stats* stats, cudaStream_t st, bool degrees_ready,
                         SolveExtras* extras) {
  const int mode = o.dtype;
  const double tol = o.tol > 0 ? o.tol : 1e-10;
  const int max_iter = o.max_iter > 0 ? o.max_iter : 1000;
  const bool warm = (o.flags & HGL_SOLVE_WARM_START) != 0;
  SolverMem sm;
  HGL_TRY(solver_layout(g, c, mode, P != nullptr, &sm));
  const CgState& S = sm.S;
  // active flags, iteration counts, breakdown flags, run flag and the last-block counter
  HGL_CHECK_CUDA(cudaMemsetAsync(sm.int_base, 0, sm.int_bytes, st));
  if (!degrees_ready) HGL_TRY(degrees_launch(g, w, st));
  if (P) HGL_TRY(precond_check(P, g, lam));

  int rows = 0;
  HGL_TRY((panel_dot<double, double>(g, c, Y, ldy, Y, ldy, gy * gy, sm.pa, st, &rows)));
  HGL_TRY(cg_reduce<RED_B2>(sm.pa, nullptr, rows, S, st));
  hgl::count_launch(); k_set_target<<<(c + 255) / 256, 256, 0, st>>>(S, tol * tol);
  HGL_CHECK_CUDA(cudaGetLastError());
  if (!warm) HGL_CHECK_CUDA(cudaMemset2DAsync(F, sizeof(double) * ldf, 0, sizeof(double) * c, g->n, st));

  hgl_status verdict = HGL_OK;
  if (mode == HGL_FP64) {
    double* R = static_cast<double*>(sm.R);
    if (warm) {
      HGL_TRY(true_residual(g, sm, lam, gy, Y, ldy, F, ldf, R, HGL_FP64, sm.ld64, st));
    } else {
      HGL_TRY((panel_scale<double, double, false>(g, c, Y, ldy, gy, R, sm.ld64, nullptr, st, nullptr)));
    }
    int rows_b = 0;
    const double* zsrc = R;
    if (P) {
      HGL_TRY(precond_apply_launch(P, g, R, sm.ld64, sm.Z, sm.ld64, c, HGL_FP64, sm.pb, st, &rows_b, nullptr));
      zsrc = static_cast<const double*>(sm.Z);
    }
    HGL_TRY((panel_dot<double, double>(g, c, R, sm.ld64, R, sm.ld64, 1.0, sm.pa, st, &rows)));
    HGL_CHECK_CUDA(cudaMemcpy2DAsync(sm.P, sizeof(double) * sm.ld64, zsrc, sizeof(double) * sm.ld64,
                                     sizeof(double) * c, g->n, cudaMemcpyDeviceToDevice, st));
    if (P && rows_b != rows) {
      // fold to a common row count (pa from panel_dot, pb from the preconditioner)
      const int mx = std::max(rows, rows_b);
      if (rows < mx) HGL_CHECK_CUDA(cudaMemsetAsync(sm.pa + (size_t)rows * c, 0, sizeof(double) * (size_t)(mx - rows) * c, st));
      if (rows_b < mx) HGL_CHECK_CUDA(cudaMemsetAsync(sm.pb + (size_t)rows_b * c, 0, sizeof(double) * (size_t)(mx - rows_b) * c, st));
      rows = mx;
    }
    HGL_TRY(cg_reduce<RED_INIT>(sm.pa, P ? sm.pb : nullptr, rows, S, st));
    int done = 0;
    if (extras && extras->fixed_iters > 0) {
      // capture mode: a fixed number of iterations, converged columns exit on the device
      for (int k = 0; k < extras->fixed_iters; ++k)
        HGL_TRY((cg_iteration<double, double>(g, sm, lam, F, ldf, HGL_FP64, HGL_FP64, P, st)));
    } else {
      HGL_TRY((run_cg_loop<double, double>(g, sm, lam, F, ldf, HGL_FP64, HGL_FP64, P, max_iter,
                                           cg_iteration_bound(lam, tol), st, &done)));
    }
    HGL_TRY(true_residual(g, sm, lam, gy, Y, ldy, F, ldf, sm.Q, HGL_FP64, sm.ld64, st));
    if (extras) extras->state = S;
    if (extras && extras->fixed_iters > 0) return HGL_OK;
    HGL_TRY(fill_stats(S, c, 0, tol, relres_out, iters_out, stats, st, &verdict));
    return verdict;
  }

  // mixed precision: FP64 refinement around an FP32-arithmetic CG.  With BF16 search
  // directions the inner CG still reaches FP32 rates: alpha comes from the stored p and
  // its product M p, and x and r move along that same p, so r stays the residual of x;
  // rounding p to BF16 (2^-9 relative) only perturbs which direction is taken, and the
  // loss of conjugacy that causes is far below what the inner tolerance needs.
  const double inner_tol = o.inner_tol > 0 ? o.inner_tol : 1e-5;
  const int max_refine = o.max_refine > 0 ? o.max_refine : 8;
  float* R32 = static_cast<float*>(sm.R);
  float* X32 = static_cast<float*>(sm.X);
  // the iterate F lives as an FP32 pair (hi, lo) during refinement; the residual is
  // formed from the pair in pair arithmetic (FP64-accurate, no FP64 arithmetic)
  // Compact residual: the gather passes read F's low part (and store the intermediate's)
  // in BF16, which adds at most 2^-32 ||F_j|| <= 2^-32 / lam ||gy y_j|| to a column's
  // residual (||F_j|| <= ||gy y_j|| / lam since M >= lam I); taken when that is below
  // tol / 64, i.e. where it cannot move a convergence decision.
  const bool compact = tol >= 64.0 * 0x1p-32 / lam;
  bf16_t* Fl16 = compact ? sm.Fl16 : nullptr;
  HGL_TRY(df_split_scalings(g, sm.s_hi, sm.s_lo, sm.t_hi, sm.t_lo, st));
  HGL_TRY(df_panel_op(g, 0, c, F, ldf, sm.Fh, sm.Fl, sm.ld32, nullptr, st, nullptr, Fl16, sm.ld16));
  // FP64-accurate residual from the pair; with a guard, skipped (launches and
  // reduction) when *guard == 0, leaving the previous relres in place
  auto residual = [&](const int32_t* guard) -> hgl_status {
    int rr_rows = 0;
    HGL_TRY(df_residual(g, sm.s_hi, sm.s_lo, sm.t_hi, sm.t_lo, sm.Fh, sm.Fl, sm.ld32, Y, ldy, -(1.0 + lam), 1.0, gy,
                        c, R32, sm.pa, st, &rr_rows, guard, extras ? extras->edge_tf : nullptr,
                        extras ? extras->edge_ldtf : 0, extras ? extras->edge_ex : nullptr, Fl16, sm.ld16));
    CgState Sg = S;
    Sg.guard = guard;
    return cg_reduce<RED_RESID>(sm.pa, nullptr, rr_rows, Sg, st);
  };
  // FP32 estimate of the same residual from the high part alone (the FP32 operator with
  // the residual epilogue, no pair arithmetic: about 0.4x the cost).  Its error, a few
  // units of 2^-24 of ||lam Y|| times (1 + 2(1+lam)/lam) (||F|| <= ||lam Y|| / lam),
  // enters the first correction; the solve starts from it when that error is well
  // below tol.  It never ends a solve: every convergence decision and every reported
  // residual comes from the pair residual.
  const bool cheap_first = tol >= 4.0 * 0x1p-24 * (1.0 + 2.0 * (1.0 + lam) / lam);
  auto residual_f32 = [&]() -> hgl_status {
    OpCall cl{};
    cl.g = g;
    cl.xdt = HGL_FP32;
    cl.zdt = HGL_FP32;
    cl.X = sm.Fh;
    cl.ldx = sm.ld32;
    cl.Z = R32;
    cl.ldz = sm.ld32;
    cl.c = c;
    cl.a = -(1.0 + lam);
    cl.b = 1.0;
    cl.epi = EPI_RESID;
    cl.Y = Y;
    cl.ldy = ldy;
    cl.gy = gy;
    cl.partials = sm.pa;
    cl.chunk_cols = g->chunk_cols;
    int rows = 0;
    HGL_TRY(op_launch(cl, st, &rows));
    return cg_reduce<RED_RESID>(sm.pa, nullptr, rows, S, st);
  };
  // one refinement sweep: inner targets, z0 = P^-1 r, CG on M d = r in FP32 (host-checked
  // batches, or `fixed` iterations with device-side early exit), F += d in the pair.
  // Guarded sweeps (captured solves) skip their expensive launches when no column
  // needs them (S.need, set by k_inner_targets).
  auto sweep = [&](double floor, int fixed, int budget, int* done, bool guarded) -> hgl_status {
    const int32_t* guard = guarded ? S.need : nullptr;
    if (guarded) HGL_CHECK_CUDA(cudaMemsetAsync(S.need, 0, sizeof(int32_t), st));
    hgl::count_launch();
    k_inner_targets<<<(c + 255) / 256, 256, 0, st>>>(S, tol, floor);
    HGL_CHECK_CUDA(cudaGetLastError());
    if (guarded) {
      HGL_PROFILED(HGL_PROF_VECTOR, hgl::count_launch();
                   k_zero_panel<<<g->num_sms * 8, 256, 0, st>>>(g->n, c, X32, sm.ld32, guard));
      HGL_CHECK_CUDA(cudaGetLastError());
    } else {
      HGL_CHECK_CUDA(cudaMemset2DAsync(X32, sizeof(float) * sm.ld32, 0, sizeof(float) * c, g->n, st));
    }
    int rows_b = 0;
    const float* zsrc = R32;
    if (P) {
      HGL_TRY(precond_apply_launch(P, g, R32, sm.ld32, sm.Z, sm.ld32, c, HGL_FP32, sm.pb, st, &rows_b, guard));
      zsrc = static_cast<const float*>(sm.Z);
    }
    if (mode == HGL_BF16) {
      HGL_TRY((panel_scale<float, bf16_t, false>(g, c, zsrc, sm.ld32, 1.0, static_cast<bf16_t*>(sm.P), sm.ld16,
                                                 nullptr, st, nullptr, guard)));
    } else if (guarded) {
      HGL_TRY((panel_scale<float, float, false>(g, c, zsrc, sm.ld32, 1.0, static_cast<float*>(sm.P), sm.ld32,
                                                nullptr, st, nullptr, guard)));
    } else {
      HGL_CHECK_CUDA(cudaMemcpy2DAsync(sm.P, sizeof(float) * sm.ld32, zsrc, sizeof(float) * sm.ld32,
                                       sizeof(float) * c, g->n, cudaMemcpyDeviceToDevice, st));
    }
    int drows = 0;
    HGL_TRY((panel_dot<float, float>(g, c, R32, sm.ld32, R32, sm.ld32, 1.0, sm.pa, st, &drows, guard)));
    if (P && rows_b != drows) {
      const int mx = std::max(drows, rows_b);
      if (drows < mx)
        HGL_CHECK_CUDA(cudaMemsetAsync(sm.pa + (size_t)drows * c, 0, sizeof(double) * (size_t)(mx - drows) * c, st));
      if (rows_b < mx)
        HGL_CHECK_CUDA(cudaMemsetAsync(sm.pb + (size_t)rows_b * c, 0, sizeof(double) * (size_t)(mx - rows_b) * c, st));
      drows = mx;
    }
    HGL_TRY(cg_reduce<RED_INIT>(sm.pa, P ? sm.pb : nullptr, drows, S, st));
    if (fixed > 0) {
      for (int k = 0; k < fixed; ++k) {
        if (mode == HGL_BF16)
          HGL_TRY((cg_iteration<bf16_t, float>(g, sm, lam, X32, sm.ld32, HGL_BF16, HGL_FP32, P, st)));
        else
          HGL_TRY((cg_iteration<float, float>(g, sm, lam, X32, sm.ld32, HGL_FP32, HGL_FP32, P, st)));
      }
      *done = fixed;
    } else {
      const int first = cg_iteration_bound(lam, floor) + 1;
      if (mode == HGL_BF16) {
        HGL_TRY((run_cg_loop<bf16_t, float>(g, sm, lam, X32, sm.ld32, HGL_BF16, HGL_FP32, P, budget, first, st,
                                            done)));
      } else {
        HGL_TRY((run_cg_loop<float, float>(g, sm, lam, X32, sm.ld32, HGL_FP32, HGL_FP32, P, budget, first, st,
                                           done)));
      }
    }
    return df_panel_op(g, 1, c, nullptr, 0, sm.Fh, sm.Fl, sm.ld32, X32, st, guard, Fl16, sm.ld16);
  };

  if (extras && extras->fixed_iters > 0) {
    // capture mode: a fixed launch sequence without host reads -- the residual, then
    // guarded sweeps (the first ones of the eager loop) each followed by a guarded
    // residual; a sweep runs, on the device's decision, only when the previous one fell
    // short of tol.  One sweep (FP32 or BF16 search directions) reaches about 1e-7
    // times the starting relres and at most the inner floor, so two suffice.
    // Statistics stay on the device.
    const double floor = inner_tol;
    const int nsweeps = 2;
    int done = 0;
    HGL_TRY(cheap_first ? residual_f32() : residual(nullptr));
    for (int sw = 0; sw < nsweeps; ++sw) {
      HGL_TRY(sweep(floor, extras->fixed_iters, 0, &done, true));
      // after an FP32 estimate the pair residual runs even when the sweep was skipped:
      // the estimate is never the reported relres
      HGL_TRY(residual(sw == 0 && cheap_first ? nullptr : S.need));
    }
    HGL_TRY(df_panel_op(g, 2, c, F, ldf, sm.Fh, sm.Fl, sm.ld32, nullptr, st));
    extras->f32 = sm.Fh;
    extras->ld32 = sm.ld32;
    extras->state = S;
    return HGL_OK;
  }

  // eager: sweep until every column meets tol (host-checked), iterations counted on
  // the device across sweeps
  int total = 0, sweeps = 0;
  bool cheap = cheap_first;
  std::vector<double> rel(c), b2(c);
  for (;;) {
    HGL_TRY(cheap ? residual_f32() : residual(nullptr));
    HGL_CHECK_CUDA(cudaMemcpyAsync(rel.data(), S.relres, sizeof(double) * c, cudaMemcpyDeviceToHost, st));
    HGL_CHECK_CUDA(cudaMemcpyAsync(b2.data(), S.b2, sizeof(double) * c, cudaMemcpyDeviceToHost, st));
    HGL_CHECK_CUDA(cudaStreamSynchronize(st));
    bool all = true;
    for (int j = 0; j < c; ++j)
      if (b2[j] > 0 && !(rel[j] <= tol)) all = false;
    if (cheap) {
      cheap = false;
      if (all) continue;  // converged by the estimate: confirm with the pair residual
    }
    if (all || sweeps >= max_refine || total >= max_iter) break;
    int done = 0;
    HGL_TRY(sweep(inner_tol, 0, max_iter - total, &done, false));
    total += done;
    ++sweeps;
  }
  if (sweeps > 0) HGL_TRY(df_panel_op(g, 2, c, F, ldf, sm.Fh, sm.Fl, sm.ld32, nullptr, st));
  if (extras) {
    extras->f32 = sm.Fh;
    extras->ld32 = sm.ld32;
    extras->state = S;
  }
  HGL_TRY(fill_stats(S, c, sweeps > 0 ? sweeps - 1 : 0, tol, relres_out, iters_out, stats, st, &verdict));
  if (P) HGL_TRY(precond_tc_status(const_cast<hgl_precond*>(P), st));
  return verdict;
}

hgl_status panel_dot_launch(const hgl_graph* g, int c, int dt, const void* A, int64_t lda, const void* B, int64_t ldb,
                            double* partials, cudaStream_t st, int* rows, const int32_t* run_flag) {
  if (dt == HGL_FP64)
    return panel_dot<double, double>(g, c, (const double*)A, lda, (const double*)B, ldb, 1.0, partials, st, rows,
                                     run_flag);
  if (dt == HGL_FP32)
    return panel_dot<float, float>(g, c, (const float*)A, lda, (const float*)B, ldb, 1.0, partials, st, rows,
                                   run_flag);
  return record_error(HGL_ERR_INVALID_ARG, "dot panels must be FP64 or FP32");
}

hgl_status panel_norm2(const hgl_graph* g, const double* F, int64_t ldf, int c, cudaStream_t st, double* out) {
  return panel_inner(g, F, ldf, F, ldf, c, st, out);
}

hgl_status panel_inner(const hgl_graph* g, const double* A, int64_t lda, const double* B, int64_t ldb, int c,
                       cudaStream_t st, double* out) {
  hgl_graph* gg = const_cast<hgl_graph*>(g);
  VecGrid vg = vec_grid(g, c, 8);
  hgl_status stt = HGL_OK;
  double* part = static_cast<double*>(buffer_get(gg->partials, sizeof(double) * 2 * (size_t)std::max(op_partial_rows(g), g->num_sms * 4) * c, &stt));
  if (!part) return stt;
  int rows = 0;
  HGL_TRY((panel_dot<double, double>(g, c, A, lda, B, ldb, 1.0, part, st, &rows)));
  std::vector<double> h((size_t)rows * c);
  HGL_CHECK_CUDA(cudaMemcpyAsync(h.data(), part, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, st));
  HGL_CHECK_CUDA(cudaStreamSynchronize(st));
  double s = 0.0;
  for (double x : h) s += x;
  (void)vg;
  *out = s;
  return HGL_OK;
}

}  // namespace hgl

extern "C" hgl_status hgl_cg_solve(const hgl_graph* g, const double* w, double lam, const double* Y, int64_t ldy,
                                   double* F, int64_t ldf, int32_t c, const hgl_precond* precond,
                                   const hgl_solve_opts* opts, double* relres, int32_t* iters,
                                   hgl_solve_stats* stats, void* stream) {
  if (!g || !w) return hgl::record_error(HGL_ERR_INVALID_ARG, "graph or w is NULL");
  if (c < 1) return hgl::record_error(HGL_ERR_INVALID_ARG, "c must be >= 1");
  if (!(lam > 0.0)) return hgl::record_error(HGL_ERR_INVALID_ARG, "lam must be positive");
  HGL_TRY(hgl::check_panel(Y, ldy, c, 8, "Y"));
  HGL_TRY(hgl::check_panel(F, ldf, c, 8, "F"));
  hgl_solve_opts o{};
  o.tol = 1e-10;
  o.max_iter = 1000;
  o.dtype = HGL_FP64;
  if (opts) o = *opts;
  if (o.dtype != HGL_FP64 && o.dtype != HGL_FP32 && o.dtype != HGL_BF16)
    return hgl::record_error(HGL_ERR_INVALID_ARG, "unknown solve dtype");
  return hgl::cg_solve_impl(const_cast<hgl_graph*>(g), w, lam, lam, Y, ldy, F, ldf, c, precond, o, relres, iters, stats,
                            hgl::as_stream(stream), false, nullptr);
}
