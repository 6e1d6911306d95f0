// resid_df.cu -- launches of the pair-arithmetic residual (df_kernels.cuh): the
// mixed-precision solver keeps its FP64 iterate F as two FP32 panels (hi, lo) and
// recomputes lam Y - M F from them to ~48 significant bits; hgl_selftest_pair_split.
#include <algorithm>

#include "df_kernels.cuh"
#include "solver.cuh"
#include "theta_kernels.cuh"

namespace hgl {

hgl_status df_split_scalings(const hgl_graph* g, float* s_hi, float* s_lo, float* t_hi, float* t_lo,
                             cudaStream_t st) {
  count_launch(2);
  df::k_split_vec<<<g->num_sms * 4, 256, 0, st>>>(g->n, g->s, s_hi, s_lo);
  df::k_split_vec<<<g->num_sms * 4, 256, 0, st>>>(g->m, g->t, t_hi, t_lo);
  HGL_CHECK_CUDA(cudaGetLastError());
  return HGL_OK;
}

hgl_status df_panel_op(const hgl_graph* g, int op, int c, double* F, int64_t ldf, float* Fh, float* Fl, int64_t ld32,
                       const float* D, cudaStream_t st, const int32_t* guard, bf16_t* Fl16, int64_t ld16) {
  const int blocks = g->num_sms * 8;
  count_launch();
  if (op == df::SPLIT)
    df::k_panel<df::SPLIT><<<blocks, 256, 0, st>>>(g->n, c, F, ldf, Fh, Fl, ld32, D, guard, Fl16, ld16);
  else if (op == df::ACCUMULATE)
    df::k_panel<df::ACCUMULATE><<<blocks, 256, 0, st>>>(g->n, c, F, ldf, Fh, Fl, ld32, D, guard, Fl16, ld16);
  else
    df::k_panel<df::COMBINE><<<blocks, 256, 0, st>>>(g->n, c, F, ldf, Fh, Fl, ld32, D, guard, nullptr, 0);
  HGL_CHECK_CUDA(cudaGetLastError());
  return HGL_OK;
}

// R = fl32(gy Y + a F + b Theta F) with F = Fh + Fl; partials of R.R (rows returned).
// With Fl16 (the low part of F rounded to BF16, row stride ld16) the gather passes read
// it and store the intermediate's low part in BF16 too: 6 bytes per gathered element
// instead of 8, at most 2^-32 ||F|| of added error (see df_kernels.cuh).
hgl_status df_residual(hgl_graph* g, const float* s_hi, const float* s_lo, const float* t_hi, const float* t_lo,
                       const float* Fh, const float* Fl, int64_t ld32, const double* Y, int64_t ldy, double a,
                       double b, double gy, int c, float* R, double* partials, cudaStream_t st, int* rows,
                       const int32_t* guard, float* tf, int64_t ldtf, double* ex, const bf16_t* Fl16,
                       int64_t ld16) {
  constexpr int E = 4;
  const int nvec = (c + E - 1) / E;
  int lg = 1, nv = 1;
  const int tuned = tuned_chunk_vecs(g, Fl16 ? TUNE_PAIR16 : TUNE_PAIR, c);
  pick_tile(std::min(nvec, tuned > 0 ? tuned : 32), &lg, &nv);
  const int cc = lg * nv * E;
  hgl_status stt = HGL_OK;
  float* Th = static_cast<float*>(buffer_get(g->scratch, sizeof(float) * 2 * (size_t)g->m * cc, &stt));
  if (!Th) return stt;
  float* Tl = Th + (size_t)g->m * cc;
  bf16_t* Tl16 = reinterpret_cast<bf16_t*>(Tl);
  // grids capped at the blocks resident at once (one wave; warps stride over rows)
  auto grid_edge = [&](const void* fn) {
    const int64_t cap = (int64_t)g->num_sms * std::min(8, resident_blocks(fn, df::THREADS, 0));
    return (int)(g->nheavy + std::max<int64_t>(1, std::min<int64_t>((g->m - g->nheavy + 7) / 8, cap)));
  };
  auto grid_vertex = [&](const void* fn) {
    const int64_t cap = (int64_t)g->num_sms * std::min(8, resident_blocks(fn, df::THREADS, 0));
    return (int)std::max<int64_t>(1, std::min<int64_t>((g->n + 7) / 8, cap));
  };
  int grid2 = 1;
  ProfScope prof(HGL_PROF_RESIDUAL, st);
  for (int c0 = 0; c0 < c; c0 += cc) {
    const int cw = std::min(cc, c - c0);
#define HGL_DF_LAUNCH(LG_, NV_, LO_, FLO, TLO, LDFLO)                                                           \
  {                                                                                                               \
    count_launch(2);                                                                                              \
    const int grid1 = grid_edge(reinterpret_cast<const void*>(df::k_edge<LG_, NV_, LO_>));                         \
    grid2 = grid_vertex(reinterpret_cast<const void*>(df::k_vertex<LG_, NV_, LO_>));                               \
    df::k_edge<LG_, NV_, LO_><<<grid1, df::THREADS, 0, st>>>(g->m, g->csc_ptr, g->csc_idx, g->edge_order,         \
                                                             g->nheavy, s_hi, s_lo, t_hi, t_lo, Fh, ld32, FLO,    \
                                                             LDFLO, c0, cw, Th, TLO, (int64_t)cc, guard, tf,      \
                                                             ldtf, ex);                                           \
    df::k_vertex<LG_, NV_, LO_><<<grid2, df::THREADS, 0, st>>>(g->n, g->csr_ptr, g->csr_idx, s_hi, s_lo, Th, TLO, \
                                                               (int64_t)cc, Fh, Fl, ld32, Y, ldy, a, b, gy, c0,   \
                                                               cw, c, R, ld32, partials, guard);                  \
  }
#define HGL_DF_CASE(LG_, NV_)                                                                                     \
  else if (lg == LG_ && nv == NV_) {                                                                              \
    if (Fl16)                                                                                                     \
      HGL_DF_LAUNCH(LG_, NV_, bf16_t, Fl16, Tl16, ld16)                                                           \
    else                                                                                                          \
      HGL_DF_LAUNCH(LG_, NV_, float, Fl, Tl, ld32)                                                                \
  }
    if (false) {
    }
    HGL_DF_CASE(1, 1) HGL_DF_CASE(2, 1) HGL_DF_CASE(4, 1) HGL_DF_CASE(8, 1) HGL_DF_CASE(16, 1) HGL_DF_CASE(32, 1)
    HGL_DF_CASE(32, 2) HGL_DF_CASE(32, 4)
#undef HGL_DF_CASE
#undef HGL_DF_LAUNCH
    HGL_CHECK_CUDA(cudaGetLastError());
  }
  *rows = grid2;
  return HGL_OK;
}

namespace {

__global__ void k_pair_selftest(int64_t len, const double* __restrict__ x, float* __restrict__ hi,
                                float* __restrict__ lo, double* __restrict__ back) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < len; i += (int64_t)gridDim.x * blockDim.x) {
    const df::f2 p = df::split_bits(x[i]);
    hi[i] = p.hi;
    lo[i] = p.lo;
    back[i] = df::f2d_bits(p.hi) + df::f2d_bits(p.lo);
  }
}

}  // namespace
}  // namespace hgl

// The solver's FP64 <-> FP32-pair conversions on given values (a test of the bit-field
// conversions against their FP64 definitions).
extern "C" hgl_status hgl_selftest_pair_split(const double* x, int64_t len, float* hi, float* lo, double* back,
                                              void* stream) {
  if (len < 0 || (len > 0 && (!x || !hi || !lo || !back)))
    return hgl::record_error(HGL_ERR_INVALID_ARG, "NULL array or negative length");
  if (len == 0) return HGL_OK;
  cudaStream_t st = hgl::as_stream(stream);
  hgl::count_launch();
  hgl::k_pair_selftest<<<(unsigned)std::min<int64_t>((len + 255) / 256, 4096), 256, 0, st>>>(len, x, hi, lo, back);
  HGL_CHECK_CUDA(cudaGetLastError());
  return HGL_OK;
}
