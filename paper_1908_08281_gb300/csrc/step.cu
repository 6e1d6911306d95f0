// step.cu -- hgl_adaptive_step: one outer iteration of the alternation of Section 2
// (F at fixed w by Eq. 6, then w at fixed F by the constrained steepest descent of
// Eqs. 4-5).
#include <algorithm>
#include <cmath>
#include <vector>

#include "precond.cuh"
#include "solver.cuh"

namespace hgl {

hgl_status project_launch(double* w, const double* grad, double eta, int64_t m, double* work, int sms,
                          cudaStream_t st, int max_steps);
hgl_status project_finish(double* w, int64_t m, double* work, int sms, cudaStream_t st, bool* continued);
size_t project_work_doubles(int64_t m, int sms);
hgl_status active_set_launch(double* w, const double* grad, double eta, int64_t m, double* work, int sms,
                             cudaStream_t st);
size_t active_set_work_doubles(int64_t m, int sms);

namespace {
// work of the weight step: the projection's or the active-set step's, whichever is larger
size_t step_work_doubles(int64_t m, int sms) {
  return std::max(project_work_doubles(m, sms), active_set_work_doubles(m, sms));
}
}  // namespace

namespace {

constexpr int RED_THREADS = 256;

// Mixed-precision solves hand the weight gradient its first pass: the pair residual at
// the final F writes t * (H^T s F) and the per-hyperedge sums of squares (graph
// buffers, sized here on the eager call and reused by the captured one).
hgl_status request_edges(hgl_graph* g, int c, SolveExtras* ext) {
  hgl_status stt = HGL_OK;
  const int64_t ld = (c + 3) / 4 * 4;
  float* tf = static_cast<float*>(buffer_get(g->edge_tf, sizeof(float) * (size_t)g->m * ld, &stt));
  if (!tf) return stt;
  double* gv = grad_vectors(g, &stt);
  if (!gv) return stt;
  ext->edge_tf = tf;
  ext->edge_ldtf = ld;
  ext->edge_ex = gv;
  return HGL_OK;
}

// The gradient at the solve's F: from the pair residual's first pass in mixed modes,
// else from F itself.
hgl_status step_gradient(hgl_graph* g, const double* w, const SolveExtras& ext, const double* F, int64_t ldf, int c,
                         double mu, double* grad, cudaStream_t st) {
  if (ext.f32 && ext.edge_tf)
    return weight_grad_from_edges(g, w, ext.edge_tf, ext.edge_ldtf, ext.f32, ext.ld32, c, mu, 0, grad, st);
  if (ext.f32) return weight_grad_launch(g, w, ext.f32, nullptr, ext.ld32, c, HGL_FP32, mu, 0, grad, st);
  return weight_grad_launch(g, w, F, nullptr, ldf, c, HGL_FP64, mu, 0, grad, st);
}

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

hgl_status adaptive_step_eager(hgl_graph* g, double* w, const hgl_step_opts& o, const double* Y, int64_t ldy,
                               double* F, int64_t ldf, int c, hgl_step_stats* stats, cudaStream_t st) {
  const int64_t m = g->m;
  const int sms = g->num_sms;
  const int red_blocks = (int)std::max<int64_t>(1, std::min<int64_t>((m + RED_THREADS - 1) / RED_THREADS, sms * 2));
  // step buffer: grad[m] | w_old[m] | projection work | sums
  const size_t pw = step_work_doubles(m, sms);
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
  hgl_status solve_status = HGL_OK;
  if (o.route == HGL_ROUTE_BCG) {
    // block CG over groups of k columns (FP64); per-group iterations and per-column
    // relres come back through a small device buffer
    const int G = (c + o.k - 1) / o.k;
    void* sbuf = nullptr;
    HGL_CHECK_CUDA(cudaMalloc(&sbuf, sizeof(double) * c + sizeof(int32_t) * G));
    double* d_rel = static_cast<double*>(sbuf);
    int32_t* d_it = reinterpret_cast<int32_t*>(d_rel + c);
    solve_status = hgl_block_cg_solve(g, w, o.lam, Y, ldy, F, ldf, c, o.k, so.tol > 0 ? so.tol : 1e-10,
                                      so.max_iter > 0 ? so.max_iter : 1000, HGL_SOLVE_WARM_START, d_rel, d_it, st);
    std::vector<double> rel(c);
    std::vector<int32_t> its(G);
    cudaError_t ce = cudaMemcpy(rel.data(), d_rel, sizeof(double) * c, cudaMemcpyDeviceToHost);
    if (ce == cudaSuccess) ce = cudaMemcpy(its.data(), d_it, sizeof(int32_t) * G, cudaMemcpyDeviceToHost);
    cudaFree(sbuf);
    if (ce != cudaSuccess) return cuda_error(ce, "block CG statistics", __FILE__, __LINE__);
    ss.status = solve_status;
    for (int j = 0; j < c; ++j) {
      ss.relres_max = std::max(ss.relres_max, rel[j]);
      ss.converged += rel[j] <= so.tol ? 1 : 0;
    }
    for (int i = 0; i < G; ++i) ss.iters = std::max(ss.iters, its[i]);
  } else {
    if (so.dtype != HGL_FP64) {
      const hgl_status er = request_edges(g, c, &ext);
      if (er != HGL_OK) {
        if (P) hgl_precond_destroy(P);
        return er;
      }
    }
    solve_status = cg_solve_impl(g, w, o.lam, o.lam, Y, ldy, F, ldf, c, P, so, nullptr, nullptr, &ss, st, true, &ext);
  }
  if (P) hgl_precond_destroy(P);
  if (solve_status != HGL_OK && solve_status != HGL_ERR_NOT_CONVERGED) return solve_status;

  // gradient at the solve's F (degrees are still those of the current w): mixed modes
  // at F's pair through the last pair residual's first pass, FP64 mode at F
  HGL_TRY(step_gradient(g, w, ext, F, ldf, c, o.mu, grad, st));
  // ||F||^2 for the objective
  HGL_CHECK_CUDA(cudaMemcpyAsync(w_old, w, sizeof(double) * m, cudaMemcpyDeviceToDevice, st));
  if (o.flags & HGL_STEP_ACTIVE_SET)
    HGL_TRY(active_set_launch(w, grad, o.eta, m, pwork, sms, st));
  else
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

// ---- captured step (HGL_STEP_GRAPH) -----------------------------------------------
//
// The step's launches -- degrees, the block rSVD rebuild (route BR), the solve with a
// fixed launch sequence (one refinement sweep, a fixed count of CG iterations from
// which converged columns exit on the device), the gradient, a fixed number of
// projection steps and the statistics' partial sums -- are captured once into a CUDA
// graph and replayed by every later call with the same pointers and options.  The
// Omega seed is read from a device word written before each replay.  The statistics
// are read after the replay; a projection that had not settled within the fixed steps
// is finished there.  The graph is captured again if a work buffer it uses has moved.

constexpr int GRAPH_PROJ_STEPS = 48;

struct StepGraph {
  // the call the graph replays
  double* w = nullptr;
  const double* Y = nullptr;
  int64_t ldy = 0;
  double* F = nullptr;
  int64_t ldf = 0;
  int c = 0;
  double lam = 0, mu = 0, eta = 0;
  int route = 0;
  int flags = 0;
  hgl_solve_opts solve{};
  std::vector<int64_t> bp;
  int k = 0, p = 0, q = 0;
  // resources
  PrecondPlan* plan = nullptr;
  cudaStream_t cs = nullptr;
  cudaGraphExec_t exec = nullptr;
  uint64_t* seed_dev = nullptr;
  std::vector<std::pair<const Buffer*, void*>> deps;
  std::vector<ProfEvent> prof;
  unsigned long long launches = 0;
  // device state read after a replay
  CgState S{};
  double* part = nullptr;
  int red_blocks = 0;
  double* fpart = nullptr;
  int frows = 0;
  double* pwork = nullptr;
  int fixed_iters = 0;

  bool matches(const double* w_, const hgl_step_opts& o, const double* Y_, int64_t ldy_, const double* F_,
               int64_t ldf_, int c_) const {
    if (w_ != w || Y_ != Y || ldy_ != ldy || F_ != F || ldf_ != ldf || c_ != c) return false;
    if (o.lam != lam || o.mu != mu || o.eta != eta || o.route != route || o.flags != flags) return false;
    if (o.solve.tol != solve.tol || o.solve.max_iter != solve.max_iter || o.solve.dtype != solve.dtype ||
        o.solve.inner_tol != solve.inner_tol || o.solve.max_refine != solve.max_refine ||
        o.solve.flags != solve.flags)
      return false;
    if (route == HGL_ROUTE_BR) {
      if (o.k != k || o.p != p || o.q != q || o.nblocks + 1 != (int)bp.size()) return false;
      for (int b = 0; b <= o.nblocks; ++b)
        if (o.block_ptr[b] != bp[b]) return false;
    }
    return true;
  }
  bool deps_moved() const {
    for (const auto& d : deps)
      if (d.first->ptr != d.second) return true;
    return false;
  }
};

void step_graph_destroy(StepGraph* sg) {
  if (!sg) return;
  if (sg->exec) cudaGraphExecDestroy(sg->exec);
  if (sg->cs) cudaStreamDestroy(sg->cs);
  if (sg->seed_dev) cudaFree(sg->seed_dev);
  precond_plan_destroy(sg->plan);
  prof_graph_release(sg->prof);
  delete sg;
}

namespace {

// The launch-only body of a captured step (no host reads, no allocations: every work
// buffer was sized by the eager call that created the StepGraph).
hgl_status step_body_captured(hgl_graph* g, StepGraph* sg, const hgl_step_opts& o, cudaStream_t st) {
  double* w = sg->w;
  const int c = sg->c;
  const int64_t m = g->m;
  const int sms = g->num_sms;
  const int red_blocks = (int)std::max<int64_t>(1, std::min<int64_t>((m + RED_THREADS - 1) / RED_THREADS, sms * 2));
  const size_t pw = step_work_doubles(m, sms);
  hgl_status stt = HGL_OK;
  double* buf = static_cast<double*>(buffer_get(g->step, sizeof(double) * (2 * (size_t)m + pw + 3 * red_blocks + 8), &stt));
  if (!buf) return stt;
  double* grad = buf;
  double* w_old = grad + m;
  double* pwork = w_old + m;
  double* part = pwork + pw;

  HGL_TRY(degrees_launch(g, w, st));
  const hgl_precond* P = nullptr;
  if (sg->route == HGL_ROUTE_BR) {
    HGL_TRY(precond_plan_compute(g, sg->plan, o.seed, sg->seed_dev, st));
    P = precond_plan_handle(sg->plan);
  }
  hgl_solve_opts so = o.solve;
  so.flags |= HGL_SOLVE_WARM_START;
  SolveExtras ext;
  ext.fixed_iters = sg->fixed_iters;
  if (so.dtype != HGL_FP64) HGL_TRY(request_edges(g, c, &ext));
  HGL_TRY(cg_solve_impl(g, w, o.lam, o.lam, sg->Y, sg->ldy, sg->F, sg->ldf, c, P, so, nullptr, nullptr, nullptr, st,
                        true, &ext));
  HGL_TRY(step_gradient(g, w, ext, sg->F, sg->ldf, c, o.mu, grad, st));
  HGL_CHECK_CUDA(cudaMemcpyAsync(w_old, w, sizeof(double) * m, cudaMemcpyDeviceToDevice, st));
  if (o.flags & HGL_STEP_ACTIVE_SET)
    HGL_TRY(active_set_launch(w, grad, o.eta, m, pwork, sms, st));
  else
    HGL_TRY(project_launch(w, grad, o.eta, m, pwork, sms, st, GRAPH_PROJ_STEPS));
  const double* ex = static_cast<const double*>(g->misc.ptr);
  hgl::count_launch();
  k_step_sums<<<red_blocks, RED_THREADS, 0, st>>>(m, g->t, ex, w_old, w, part);
  HGL_CHECK_CUDA(cudaGetLastError());
  // ||F||^2 partials into the solver's reduction buffer (idle after the solve)
  double* fpart = static_cast<double*>(g->partials.ptr);
  int frows = 0;
  HGL_TRY(panel_dot_launch(g, c, HGL_FP64, sg->F, sg->ldf, sg->F, sg->ldf, fpart, st, &frows));
  sg->S = ext.state;
  sg->part = part;
  sg->red_blocks = red_blocks;
  sg->fpart = fpart;
  sg->frows = frows;
  sg->pwork = pwork;
  return HGL_OK;
}

hgl_status step_capture(hgl_graph* g, StepGraph* sg, const hgl_step_opts& o) {
  if (sg->exec) {
    cudaGraphExecDestroy(sg->exec);
    sg->exec = nullptr;
  }
  prof_graph_release(sg->prof);
  const unsigned long long l0 = hgl_launch_count();
  prof_capture_begin(&sg->prof);
  HGL_CHECK_CUDA(cudaStreamBeginCapture(sg->cs, cudaStreamCaptureModeThreadLocal));
  hgl_status body = step_body_captured(g, sg, o, sg->cs);
  cudaGraph_t graph = nullptr;
  const cudaError_t ec = cudaStreamEndCapture(sg->cs, &graph);
  prof_capture_end();
  sg->launches = hgl_launch_count() - l0;
  uncount_launch(sg->launches);
  if (body != HGL_OK || ec != cudaSuccess || !graph) {
    if (graph) cudaGraphDestroy(graph);
    (void)cudaGetLastError();
    prof_graph_release(sg->prof);
    if (body != HGL_OK) return body;
    return cuda_error(ec != cudaSuccess ? ec : cudaErrorUnknown, "cudaStreamEndCapture(adaptive step)", __FILE__,
                      __LINE__);
  }
  const cudaError_t ei = cudaGraphInstantiate(&sg->exec, graph, 0);
  cudaGraphDestroy(graph);
  if (ei != cudaSuccess) {
    sg->exec = nullptr;
    return cuda_error(ei, "cudaGraphInstantiate(adaptive step)", __FILE__, __LINE__);
  }
  sg->deps.clear();
  for (const Buffer* b : {&g->step, &g->solver, &g->partials, &g->scratch, &g->scratch2, &g->misc, &g->edge_tf})
    sg->deps.emplace_back(b, b->ptr);
  if (sg->plan) {
    hgl_precond* P = const_cast<hgl_precond*>(precond_plan_handle(sg->plan));
    sg->deps.emplace_back(&P->cbuf, P->cbuf.ptr);
    sg->deps.emplace_back(&P->pbuf, P->pbuf.ptr);
  }
  return HGL_OK;
}

hgl_status step_replay(hgl_graph* g, StepGraph* sg, const hgl_step_opts& o, hgl_step_stats* stats, cudaStream_t st) {
  uint64_t seed = o.seed;
  HGL_CHECK_CUDA(cudaMemcpyAsync(sg->seed_dev, &seed, sizeof(seed), cudaMemcpyHostToDevice, st));
  HGL_CHECK_CUDA(cudaGraphLaunch(sg->exec, st));
  count_launch((unsigned)sg->launches);
  HGL_CHECK_CUDA(cudaStreamSynchronize(st));
  prof_graph_add(sg->prof);
  if (sg->plan) HGL_TRY(precond_plan_check(sg->plan, st));
  bool continued = false;
  if (!(o.flags & HGL_STEP_ACTIVE_SET)) HGL_TRY(project_finish(sg->w, g->m, sg->pwork, g->num_sms, st, &continued));
  if (continued) {
    // the projection was finished after the replay: recompute the step's sums
    const double* ex = static_cast<const double*>(g->misc.ptr);
    const double* w_old = sg->pwork - g->m;
    hgl::count_launch();
    k_step_sums<<<sg->red_blocks, RED_THREADS, 0, st>>>(g->m, g->t, ex, w_old, sg->w, sg->part);
    HGL_CHECK_CUDA(cudaGetLastError());
  }
  hgl_solve_stats ss{};
  hgl_status verdict = HGL_OK;
  const double tol = o.solve.tol > 0 ? o.solve.tol : 1e-10;
  // a mixed-precision solve ran its second sweep when the flag is still set
  int32_t need = 0;
  if (sg->solve.dtype != HGL_FP64)
    HGL_CHECK_CUDA(cudaMemcpyAsync(&need, sg->S.need, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  HGL_TRY(fill_stats(sg->S, sg->c, 0, tol, nullptr, nullptr, &ss, st, &verdict));
  ss.refinements = need;
  std::vector<double> hp(3 * (size_t)sg->red_blocks), hf((size_t)sg->frows * sg->c);
  HGL_CHECK_CUDA(cudaMemcpyAsync(hp.data(), sg->part, sizeof(double) * hp.size(), cudaMemcpyDeviceToHost, st));
  HGL_CHECK_CUDA(cudaMemcpyAsync(hf.data(), sg->fpart, sizeof(double) * hf.size(), cudaMemcpyDeviceToHost, st));
  HGL_CHECK_CUDA(cudaStreamSynchronize(st));
  double tr = 0.0, w2 = 0.0, dw2 = 0.0, fnorm2 = 0.0;
  for (int b = 0; b < sg->red_blocks; ++b) {
    tr += hp[3 * b];
    w2 += hp[3 * b + 1];
    dw2 += hp[3 * b + 2];
  }
  for (double x : hf) fnorm2 += x;
  if (stats) {
    stats->solve = ss;
    stats->objective = fnorm2 - tr + o.mu * w2;
    stats->dw_norm = std::sqrt(dw2);
  }
  return verdict;
}

}  // namespace

hgl_status adaptive_step_impl(hgl_graph* g, double* w, const hgl_step_opts& o, const double* Y, int64_t ldy,
                              double* F, int64_t ldf, int c, hgl_step_stats* stats, cudaStream_t st) {
  if (!(o.flags & HGL_STEP_GRAPH)) return adaptive_step_eager(g, w, o, Y, ldy, F, ldf, c, stats, st);
  if (o.solve.dtype != HGL_FP64 && o.solve.dtype != HGL_FP32 && o.solve.dtype != HGL_BF16)
    return record_error(HGL_ERR_INVALID_ARG, "unknown solve dtype");
  if (o.route == HGL_ROUTE_BCG) return record_error(HGL_ERR_INVALID_ARG, "the block CG route runs eagerly");
  StepGraph*& sg = g->step_graph;
  if (!sg || !sg->matches(w, o, Y, ldy, F, ldf, c)) {
    // a new call pattern: run it eagerly (which also sizes every work buffer the graph
    // will use), then set up the graph's own resources; the next call captures
    step_graph_destroy(sg);
    sg = nullptr;
    const hgl_status s = adaptive_step_eager(g, w, o, Y, ldy, F, ldf, c, stats, st);
    if (s != HGL_OK && s != HGL_ERR_NOT_CONVERGED) return s;
    StepGraph* ng = new (std::nothrow) StepGraph();
    if (!ng) return record_error(HGL_ERR_OOM, "host allocation failed");
    ng->w = w;
    ng->Y = Y;
    ng->ldy = ldy;
    ng->F = F;
    ng->ldf = ldf;
    ng->c = c;
    ng->lam = o.lam;
    ng->mu = o.mu;
    ng->eta = o.eta;
    ng->route = o.route;
    ng->flags = o.flags;
    ng->solve = o.solve;
    const double floor = o.solve.inner_tol > 0 ? o.solve.inner_tol : 1e-5;
    ng->fixed_iters = cg_iteration_bound(o.lam, o.solve.dtype == HGL_FP64 ? (o.solve.tol > 0 ? o.solve.tol : 1e-10)
                                                                           : floor) + 4;
    hgl_status e = HGL_OK;
    if (o.route == HGL_ROUTE_BR) {
      ng->bp.assign(o.block_ptr, o.block_ptr + o.nblocks + 1);
      ng->k = o.k;
      ng->p = o.p;
      ng->q = o.q;
      e = precond_plan_create(g, o.lam, o.block_ptr, o.nblocks, o.k, o.p, o.q, HGL_BF16, true, st, &ng->plan);
      if (e == HGL_OK)
        e = precond_reserve(const_cast<hgl_precond*>(precond_plan_handle(ng->plan)), c,
                            o.solve.dtype == HGL_FP64 ? HGL_FP64 : HGL_FP32);
    }
    if (e == HGL_OK) {
      const cudaError_t ce = cudaMalloc(&ng->seed_dev, sizeof(uint64_t));
      if (ce != cudaSuccess) e = cuda_error(ce, "cudaMalloc(seed word)", __FILE__, __LINE__);
    }
    if (e == HGL_OK) {
      const cudaError_t ce = cudaStreamCreateWithFlags(&ng->cs, cudaStreamNonBlocking);
      if (ce != cudaSuccess) e = cuda_error(ce, "cudaStreamCreate(capture)", __FILE__, __LINE__);
    }
    if (e != HGL_OK) {
      step_graph_destroy(ng);
      return e;
    }
    sg = ng;
    return s;
  }
  if (!sg->exec || sg->deps_moved()) HGL_TRY(step_capture(g, sg, o));
  return step_replay(g, sg, o, stats, st);
}

}  // namespace hgl

extern "C" hgl_status hgl_adaptive_step(hgl_graph* g, double* w, const hgl_step_opts* opts, const double* Y,
                                        int64_t ldy, double* F, int64_t ldf, int32_t c, hgl_step_stats* stats,
                                        void* stream) {
  if (!g || !w || !opts) return hgl::record_error(HGL_ERR_INVALID_ARG, "NULL argument");
  if (c < 1) return hgl::record_error(HGL_ERR_INVALID_ARG, "c must be >= 1");
  if (!(opts->lam > 0.0) || opts->mu < 0.0 || !(opts->eta >= 0.0))
    return hgl::record_error(HGL_ERR_INVALID_ARG, "need lam > 0, mu >= 0, eta >= 0");
  if (opts->route != HGL_ROUTE_CG && opts->route != HGL_ROUTE_BR && opts->route != HGL_ROUTE_BCG)
    return hgl::record_error(HGL_ERR_INVALID_ARG, "unknown route");
  if (opts->route == HGL_ROUTE_BCG && opts->solve.dtype != HGL_FP64)
    return hgl::record_error(HGL_ERR_INVALID_ARG, "the block CG route is FP64");
  HGL_TRY(hgl::check_panel(Y, ldy, c, 8, "Y"));
  HGL_TRY(hgl::check_panel(F, ldf, c, 8, "F"));
  return hgl::adaptive_step_impl(g, w, *opts, Y, ldy, F, ldf, c, stats, hgl::as_stream(stream));
}

extern "C" hgl_status hgl_step_precond(const hgl_graph* g, const hgl_precond** out) {
  if (!g || !out) return hgl::record_error(HGL_ERR_INVALID_ARG, "graph or out is NULL");
  *out = nullptr;
  const hgl::StepGraph* sg = g->step_graph;
  if (!sg || !sg->plan)
    return hgl::record_error(HGL_ERR_INVALID_ARG, "no captured block-rSVD step has been set up on this graph");
  *out = hgl::precond_plan_handle(sg->plan);
  return HGL_OK;
}
