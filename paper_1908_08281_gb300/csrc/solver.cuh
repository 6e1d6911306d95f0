// solver.cuh -- internals shared by the CG solver, the preconditioner and the
// adaptive step.
#pragma once

#include "hgl_internal.cuh"
#include "vec_kernels.cuh"

namespace hgl {

struct VecGrid {
  int lg = 32, gx = 1, gy = 1;
};

// Launch shape of the row-parallel panel kernels for c columns of `elt`-byte elements.
VecGrid vec_grid(const hgl_graph* g, int c, int elt);

struct SolverMem {
  CgState S{};
  void* R = nullptr;  // residual
  void* P = nullptr;  // search direction
  void* Q = nullptr;  // M p
  void* Z = nullptr;  // preconditioned residual
  void* X = nullptr;  // mixed modes: correction D
  double* pa = nullptr;
  double* pb = nullptr;
  int c = 0;
  int64_t ld64 = 0, ld32 = 0, ld16 = 0;
  void* int_base = nullptr;  // per-column int32 state and flags (zeroed per solve)
  size_t int_bytes = 0;
  float *Fh = nullptr, *Fl = nullptr;          // mixed modes: F as an FP32 pair
  bf16_t* Fl16 = nullptr;                      // mixed modes: F's low part in BF16 (compact residual)
  float *s_hi = nullptr, *s_lo = nullptr;      // mixed modes: scalings as FP32 pairs
  float *t_hi = nullptr, *t_lo = nullptr;
};

// Optional outputs of a solve: in mixed modes the FP32 high part of F (valid until
// the next solve on the graph).
struct SolveExtras {
  // out (mixed modes): the FP32 high part of F, valid until the next solve on the graph
  const float* f32 = nullptr;
  int64_t ld32 = 0;
  // out: the per-column device state (relres, iterations, breakdown flags)
  CgState state{};
  // in (mixed modes, optional): every pair residual also writes t * (H^T s F) in FP32
  // to edge_tf (m x c, row stride edge_ldtf) and per hyperedge the sum of squares of
  // H^T s F over the columns to edge_ex -- the weight gradient's first pass at the
  // solve's final F (the last residual of a solve is taken at the returned F)
  float* edge_tf = nullptr;
  int64_t edge_ldtf = 0;
  double* edge_ex = nullptr;
  // in: > 0 selects capture mode -- a fixed launch sequence without host reads (one
  // refinement sweep in mixed modes, this many CG iterations with device-side early
  // exit); the caller reads the statistics after running it (fill_stats on `state`)
  int fixed_iters = 0;
};

// Per-column statistics and the verdict of a finished solve from its device state.
// Synchronises the stream.
hgl_status fill_stats(const CgState& S, int c, int refinements, double tol, double* relres_out,
                      int32_t* iters_out, hgl_solve_stats* stats, cudaStream_t st, hgl_status* verdict);

hgl_status df_split_scalings(const hgl_graph* g, float* s_hi, float* s_lo, float* t_hi, float* t_lo, cudaStream_t st);
// guard (optional device flag): the kernels return at once when *guard == 0
// Fl16 (optional): SPLIT and ACCUMULATE also store the low part rounded to BF16
hgl_status df_panel_op(const hgl_graph* g, int op, int c, double* F, int64_t ldf, float* Fh, float* Fl, int64_t ld32,
                       const float* D, cudaStream_t st, const int32_t* guard = nullptr, bf16_t* Fl16 = nullptr,
                       int64_t ld16 = 0);
// Fl16 (optional): the compact residual, gathering F's low part from its BF16 copy
hgl_status df_residual(hgl_graph* g, const float* s_hi, const float* s_lo, const float* t_hi, const float* t_lo,
                       const float* Fh, const float* Fl, int64_t ld32, const double* Y, int64_t ldy, double a,
                       double b, double gy, int c, float* R, double* partials, cudaStream_t st, int* rows,
                       const int32_t* guard = nullptr, float* tf = nullptr, int64_t ldtf = 0,
                       double* ex = nullptr, const bf16_t* Fl16 = nullptr, int64_t ld16 = 0);

hgl_status cg_reduce_beta(double* pa, int rows_a, double* pb, int rows_b, const CgState& S, cudaStream_t st);

// Solves M F = gy Y with M = (1 + lam) I - Theta (gy = lam for the ranking system of
// Eq. 6, gy = 1 for the adjoint system M Z = G); relative residuals are taken against
// ||gy y_j||.
hgl_status cg_solve_impl(hgl_graph* g, const double* w, double lam, double gy, const double* Y, int64_t ldy, double* F,
                         int64_t ldf, int c, const hgl_precond* P, const hgl_solve_opts& o, double* relres_out,
                         int32_t* iters_out, hgl_solve_stats* stats, cudaStream_t st, bool degrees_ready,
                         SolveExtras* extras);

int cg_iteration_bound(double lam, double tol);

// The same gradient (Zb = F, FP32 panel) from a first pass already done: TF = t * (H^T s F)
// (m x c FP32, row stride ldtf) and ex[e] = ||(H^T s F)_e||^2 in the graph's gradient
// vectors (as a pair residual with SolveExtras::edge_tf writes them).
hgl_status weight_grad_from_edges(hgl_graph* g, const double* w, const float* TF, int64_t ldtf, const float* F,
                                  int64_t ld, int c, double mu, int flags, double* grad, cudaStream_t st);
// The graph's gradient vectors (ex[m], phi[n]); allocates on first use.
double* grad_vectors(hgl_graph* g, hgl_status* st);
// grad = -theta_sign * d tr(Zb^T Theta F)/dw + 2 mu w (Zb = NULL: Zb = F), at fixed panels.
hgl_status weight_grad_launch(hgl_graph* g, const double* w, const void* F, const void* Zb, int64_t ld, int c,
                              int dtype, double mu, int flags, double* grad, cudaStream_t st,
                              double theta_sign = 1.0);

// per-column partial sums of A.B for panels of type dt (FP64 or FP32); rows in *rows
hgl_status panel_dot_launch(const hgl_graph* g, int c, int dt, const void* A, int64_t lda, const void* B, int64_t ldb,
                            double* partials, cudaStream_t st, int* rows, const int32_t* run_flag = nullptr);

// A block rSVD plan for one block layout: created once (allocates, uploads metadata,
// synchronous), computed any number of times (kernel launches only; capturable), its
// handle reused by every compute.
struct PrecondPlan;
hgl_status precond_plan_create(const hgl_graph* g, double lam, const int64_t* bp, int32_t nb, int32_t k, int32_t p,
                               int32_t q, int gemm_dtype, bool own_space, cudaStream_t st, PrecondPlan** out);
hgl_status precond_plan_compute(const hgl_graph* g, PrecondPlan* pl, uint64_t seed, const uint64_t* seed_dev,
                                cudaStream_t st);
hgl_status precond_plan_check(PrecondPlan* pl, cudaStream_t st);
const hgl_precond* precond_plan_handle(const PrecondPlan* pl);
void precond_plan_destroy(PrecondPlan* pl);
// Grow the apply's work space for c-column panels of `dt` (so that applies allocate nothing).
hgl_status precond_reserve(hgl_precond* P, int c, int dt);

hgl_status precond_build(const hgl_graph* g, const double* w, double lam, const int64_t* block_ptr, int32_t nblocks,
                         int32_t k, int32_t p, int32_t q, uint64_t seed, int gemm_dtype, cudaStream_t st,
                         hgl_precond** out, bool degrees_ready);

// sum over all entries of F*F (FP64 panel), deterministic; synchronises the stream.
hgl_status panel_norm2(const hgl_graph* g, const double* F, int64_t ldf, int c, cudaStream_t st, double* out);
// Algorithm 1 (Rayleigh-Ritz, FP64) on the symmetric parts of nb dense matrices at once,
// Omega drawn for global rows v0s[b] ..; Ritz vectors to rows v0s[b] - qrow0 .. of Qout
// (k columns), values to ev[b * k ..].
hgl_status dense_rsvd_batch_fp64(int nb, const double* const* Ls, const int64_t* ldls, const int64_t* v0s,
                                 const int64_t* sizes, int k, int p, int q, uint64_t seed, Buffer& space,
                                 double* Qout, int64_t qrow0, double* ev, cudaStream_t st);
// sum over all entries of A*B (FP64 panels), deterministic; synchronises the stream.
hgl_status panel_inner(const hgl_graph* g, const double* A, int64_t lda, const double* B, int64_t ldb, int c,
                       cudaStream_t st, double* out);

// Preconditioner hooks (rsvd.cu).  Z = P^-1 R on panels of `dt` (FP64 or FP32) and,
// when partials_rz is given, per-column partial sums of R.Z (row count in *rows).
hgl_status precond_check(const hgl_precond* P, const hgl_graph* g, double lam);
// Rows of each of the solver's two FP64 partial-sum arrays (row stride c).
int solver_partial_rows(const hgl_graph* g);

hgl_status precond_apply_launch(const hgl_precond* P, const hgl_graph* g, const void* R, int64_t ldr, void* Z,
                                int64_t ldz, int c, int dt, double* partials_rz, cudaStream_t st, int* rows,
                                const int32_t* run_flag);

}  // namespace hgl
