// adjoint.cu -- hgl_adjoint_grad: the w-gradient of a loss that depends on w through
// the ranking solve (Eq. 6), by the adjoint method.
//
// With M(w) F = lam Y, differentiating gives dF = -M^-1 (dM) F and dM/dw_e =
// -dTheta/dw_e.  For a loss gradient G = dL/dF the chain rule term is therefore
//   <G, dF/dw_e> = d/dw_e tr(Z^T Theta(w) F),   Z = M^-1 G   (M is symmetric),
// one more batched CG solve with the same operator and the bilinear form of the
// Eq. 4 gradient.  Nothing of the forward solve is stored but F: the adjoint solve
// runs its own recurrences.
#include "precond.cuh"
#include "solver.cuh"

extern "C" hgl_status hgl_adjoint_grad(hgl_graph* g, const double* w, double lam, const double* F,
                                       const double* G, double* Z, int64_t ld, int32_t c,
                                       const hgl_precond* precond, const hgl_solve_opts* opts, double* grad,
                                       hgl_solve_stats* stats, void* stream) {
  using namespace hgl;
  if (!g || !w || !F || !G || !Z || !grad || !opts) return record_error(HGL_ERR_INVALID_ARG, "NULL argument");
  if (c < 1) return record_error(HGL_ERR_INVALID_ARG, "c must be >= 1");
  if (!(lam > 0.0)) return record_error(HGL_ERR_INVALID_ARG, "lam must be positive");
  HGL_TRY(check_panel(F, ld, c, 8, "F"));
  HGL_TRY(check_panel(G, ld, c, 8, "G"));
  HGL_TRY(check_panel(Z, ld, c, 8, "Z"));
  if (Z == F || Z == G) return record_error(HGL_ERR_INVALID_ARG, "Z must not alias F or G");
  cudaStream_t st = as_stream(stream);
  HGL_TRY(degrees_launch(g, w, st));
  // adjoint system M Z = G: the right-hand-side multiplier is 1, the operator that of lam
  const hgl_status solved = cg_solve_impl(g, w, lam, 1.0, G, ld, Z, ld, c, precond, *opts, nullptr, nullptr, stats,
                                          st, true, nullptr);
  if (solved != HGL_OK && solved != HGL_ERR_NOT_CONVERGED) return solved;
  // grad = + d tr(Z^T Theta F)/dw (the weight-gradient kernels with the Theta term's sign flipped, mu = 0)
  HGL_TRY(weight_grad_launch(g, w, F, Z, ld, c, HGL_FP64, 0.0, 0, grad, st, -1.0));
  HGL_CHECK_CUDA(cudaStreamSynchronize(st));
  return solved;
}

// tr(F^T Delta F) with Delta = I - Theta(w) (the first term of the objective of Eq. 4),
// and Delta F itself (the loss's F-gradient is 2 Delta F).
extern "C" hgl_status hgl_laplacian_quadratic(hgl_graph* g, const double* w, const double* F, int64_t ldf,
                                              double* DF, int64_t lddf, int32_t c, double* value, void* stream) {
  using namespace hgl;
  if (!g || !w || !F || !DF || !value) return record_error(HGL_ERR_INVALID_ARG, "NULL argument");
  if (c < 1) return record_error(HGL_ERR_INVALID_ARG, "c must be >= 1");
  HGL_TRY(check_panel(F, ldf, c, 8, "F"));
  HGL_TRY(check_panel(DF, lddf, c, 8, "DF"));
  if (DF == F) return record_error(HGL_ERR_INVALID_ARG, "DF must not alias F");
  cudaStream_t st = as_stream(stream);
  HGL_TRY(degrees_launch(g, w, st));
  OpCall cl{};
  cl.g = g;
  cl.xdt = HGL_FP64;
  cl.zdt = HGL_FP64;
  cl.X = F;
  cl.ldx = ldf;
  cl.Z = DF;
  cl.ldz = lddf;
  cl.c = c;
  cl.a = 1.0;
  cl.b = -1.0;
  cl.epi = EPI_PLAIN;
  HGL_TRY(op_launch(cl, st, nullptr));
  return panel_inner(g, F, ldf, DF, lddf, c, st, value);
}
