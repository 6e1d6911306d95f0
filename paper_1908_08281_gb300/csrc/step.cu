// step.cu -- hgl_adaptive_step: one outer iteration of the alternation of Section 2
// (F at fixed w by Eq. 6, then w at fixed F by the constrained steepest descent of
// Eqs. 4-5).
#include <algorithm>
#include <cmath>
#include <vector>

#include "solver.cuh"

namespace hgl {

hgl_status project_launch(double* w, const double* grad, double eta, int64_t m, double* work, int sms,
                          cudaStream_t st, int max_steps);
size_t project_work_doubles(int64_t m, int sms);

namespace {

constexpr int RED_THREADS = 256;

// partial sums of sum_e t_e ex_e (tr F^T Theta F), ||w||^2 and ||w - w_old||^2
__global__ void k_step_sums(int64_t m, const double* __restrict__ t, const double* __restrict__ ex,
                            const double* __restrict__ w_old, const double* __restrict__ w_new,
                            double* __restrict__ part) {
  __shared__ double red[3][RED_THREADS / 32];
  double a = 0.0, b = 0.0, d = 0.0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x) {
    a += t[e] * ex[e];
    b += w_old[e] * w_old[e];
    const double x = w_new[e] - w_old[e];
    d += x * x;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
    d += __shfl_xor_sync(0xffffffffu, d, o);
  }
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = a;
    red[1][threadIdx.x >> 5] = b;
    red[2][threadIdx.x >> 5] = d;
  }
  __syncthreads();
  if (threadIdx.x < 3) {
    double s = 0.0;
    for (int i = 0; i < RED_THREADS / 32; ++i) s += red[threadIdx.x][i];
    part[blockIdx.x * 3 + threadIdx.x] = s;
  }
}

}  // namespace

hgl_status adaptive_step_impl(hgl_graph* g, double* w, const hgl_step_opts& o, const double* Y, int64_t ldy,
                              double* F, int64_t ldf, int c, hgl_step_stats* stats, cudaStream_t st) {
  const int64_t m = g->m;
  const int sms = g->num_sms;
  const int red_blocks = (int)std::max<int64_t>(1, std::min<int64_t>((m + RED_THREADS - 1) / RED_THREADS, sms * 2));
  // step buffer: grad[m] | w_old[m] | projection work | sums
  const size_t pw = project_work_doubles(m, sms);
  hgl_status stt = HGL_OK;
  // misc is used by the gradient (ex, phi); the step keeps its vectors in `step`
  double* buf = static_cast<double*>(buffer_get(g->step, sizeof(double) * (2 * (size_t)m + pw + 3 * red_blocks + 8), &stt));
  if (!buf) return stt;
  double* grad = buf;
  double* w_old = grad + m;
  double* pwork = w_old + m;
  double* part = pwork + pw;

  HGL_TRY(degrees_launch(g, w, st));
  hgl_precond* P = nullptr;
  if (o.route == HGL_ROUTE_BR) {
    HGL_TRY(precond_build(g, w, o.lam, o.block_ptr, o.nblocks, o.k, o.p, o.q, o.seed, HGL_BF16, st, &P, true));
  }
  hgl_solve_opts so = o.solve;
  so.flags |= HGL_SOLVE_WARM_START;
  hgl_solve_stats ss{};
  SolveExtras ext;
  hgl_status solve_status = cg_solve_impl(g, w, o.lam, o.lam, Y, ldy, F, ldf, c, P, so, nullptr, nullptr, &ss, st, true,
                                          &ext);
  if (P) hgl_precond_destroy(P);
  if (solve_status != HGL_OK && solve_status != HGL_ERR_NOT_CONVERGED) return solve_status;

  // gradient at the solve's F (degrees are still those of the current w)
  // mixed modes differentiate at the FP32 high part of F (FP32 arithmetic); FP64 mode at F
  if (ext.f32)
    HGL_TRY(weight_grad_launch(g, w, ext.f32, nullptr, ext.ld32, c, HGL_FP32, o.mu, 0, grad, st));
  else
    HGL_TRY(weight_grad_launch(g, w, F, nullptr, ldf, c, HGL_FP64, o.mu, 0, grad, st));
  // ||F||^2 for the objective
  HGL_CHECK_CUDA(cudaMemcpyAsync(w_old, w, sizeof(double) * m, cudaMemcpyDeviceToDevice, st));
  HGL_TRY(project_launch(w, grad, o.eta, m, pwork, sms, st, 0));
  const double* ex = static_cast<const double*>(g->misc.ptr);
  hgl::count_launch(); k_step_sums<<<red_blocks, RED_THREADS, 0, st>>>(m, g->t, ex, w_old, w, part);
  HGL_CHECK_CUDA(cudaGetLastError());
  std::vector<double> hp(3 * (size_t)red_blocks);
  HGL_CHECK_CUDA(cudaMemcpyAsync(hp.data(), part, sizeof(double) * hp.size(), cudaMemcpyDeviceToHost, st));
  double fnorm2 = 0.0;
  HGL_TRY(panel_norm2(g, F, ldf, c, st, &fnorm2));
  HGL_CHECK_CUDA(cudaStreamSynchronize(st));
  double tr = 0.0, w2 = 0.0, dw2 = 0.0;
  for (int b = 0; b < red_blocks; ++b) {
    tr += hp[3 * b];
    w2 += hp[3 * b + 1];
    dw2 += hp[3 * b + 2];
  }
  if (stats) {
    stats->solve = ss;
    stats->objective = fnorm2 - tr + o.mu * w2;
    stats->dw_norm = std::sqrt(dw2);
  }
  return solve_status;
}

}  // namespace hgl

extern "C" hgl_status hgl_adaptive_step(hgl_graph* g, double* w, const hgl_step_opts* opts, const double* Y,
                                        int64_t ldy, double* F, int64_t ldf, int32_t c, hgl_step_stats* stats,
                                        void* stream) {
  if (!g || !w || !opts) return hgl::record_error(HGL_ERR_INVALID_ARG, "NULL argument");
  if (c < 1) return hgl::record_error(HGL_ERR_INVALID_ARG, "c must be >= 1");
  if (!(opts->lam > 0.0) || opts->mu < 0.0 || !(opts->eta >= 0.0))
    return hgl::record_error(HGL_ERR_INVALID_ARG, "need lam > 0, mu >= 0, eta >= 0");
  if (opts->route != HGL_ROUTE_CG && opts->route != HGL_ROUTE_BR)
    return hgl::record_error(HGL_ERR_INVALID_ARG, "unknown route");
  HGL_TRY(hgl::check_panel(Y, ldy, c, 8, "Y"));
  HGL_TRY(hgl::check_panel(F, ldf, c, 8, "F"));
  return hgl::adaptive_step_impl(g, w, *opts, Y, ldy, F, ldf, c, stats, hgl::as_stream(stream));
}
