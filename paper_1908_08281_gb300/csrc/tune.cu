// tune.cu -- hgl_tune_operator: pick the column chunk of the gather passes by timing.
//
// The operator apply and the pair-arithmetic residual process the right-hand-side
// columns in chunks; a wide chunk reads each gathered row in one long burst, a narrow
// one keeps the gathered slice of the panel in L2 but re-reads the index arrays per
// chunk.  Which wins depends on n, m, c, the panel type and the degree distribution,
// so the chunk is chosen by timing every supported width on the graph itself.  The
// choice is stored in the graph and used by later calls; untuned graphs use a fixed
// default, so results never depend on timing unless the caller asks for tuning.
#include <algorithm>

#include "solver.cuh"
#include "theta_launch.cuh"

namespace hgl {
namespace {

struct DevMem {
  void* p = nullptr;
  ~DevMem() {
    if (p) cudaFree(p);
  }
};

template <class F>
hgl_status time_ms(cudaStream_t st, F&& run, float* ms) {
  cudaEvent_t a = nullptr, b = nullptr;
  HGL_CHECK_CUDA(cudaEventCreate(&a));
  HGL_CHECK_CUDA(cudaEventCreate(&b));
  hgl_status s = run();  // warm
  if (s == HGL_OK) {
    cudaEventRecord(a, st);
    for (int r = 0; r < 2 && s == HGL_OK; ++r) s = run();
    cudaEventRecord(b, st);
    cudaEventSynchronize(b);
    cudaEventElapsedTime(ms, a, b);
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return s;
}

}  // namespace
}  // namespace hgl

extern "C" hgl_status hgl_tune_operator(hgl_graph* g, const double* w, int32_t c, hgl_dtype dtype,
                                        int32_t* chunk_cols, int32_t* pair_chunk_cols, int32_t* grid_policy,
                                        void* stream) {
  using namespace hgl;
  if (!g || !w) return record_error(HGL_ERR_INVALID_ARG, "graph or w is NULL");
  if (c < 1) return record_error(HGL_ERR_INVALID_ARG, "c must be >= 1");
  if (dtype != HGL_FP64 && dtype != HGL_FP32 && dtype != HGL_BF16)
    return record_error(HGL_ERR_INVALID_ARG, "unknown dtype");
  cudaStream_t st = as_stream(stream);
  HGL_TRY(degrees_launch(g, w, st));
  const size_t elt = dtype_size(dtype);
  const int E = (int)(16 / elt);
  const int64_t ld = (c + E - 1) / E * E;
  const int nvec = (c + E - 1) / E;
  // the variant the CG iteration launches: Z = M X with the column partials of X.Z,
  // Z in FP32 for BF16 search directions
  const int zdt = dtype == HGL_BF16 ? HGL_FP32 : dtype;
  const size_t zelt = dtype_size(zdt);
  const int64_t ldz = (c + (int)(16 / zelt) - 1) / (int)(16 / zelt) * (int)(16 / zelt);
  DevMem X, Z, part;
  HGL_CHECK_CUDA(cudaMalloc(&X.p, elt * (size_t)g->n * ld));
  HGL_CHECK_CUDA(cudaMalloc(&Z.p, zelt * (size_t)g->n * ldz));
  HGL_CHECK_CUDA(cudaMalloc(&part.p, sizeof(double) * (size_t)op_partial_rows(g) * c));
  HGL_CHECK_CUDA(cudaMemsetAsync(X.p, 0x3F, elt * (size_t)g->n * ld, st));  // finite, normal values

  // operator apply: chunk widths of 1 .. 128 vectors per row (each a distinct tile;
  // up to 8 vectors the row-per-group kernels, above them the member-parallel ones)
  int best = 0;
  float best_ms = 0.f;
  for (int vecs : {1, 2, 4, 8, 16, 32, 64, 128}) {
    const int cand = std::min(vecs, nvec);
    OpCall cl{};
    cl.g = g;
    cl.xdt = dtype;
    cl.zdt = zdt;
    cl.X = X.p;
    cl.ldx = ld;
    cl.Z = Z.p;
    cl.ldz = ldz;
    cl.c = c;
    cl.a = 1.5;
    cl.b = -1.0;
    cl.epi = EPI_DOT_XZ;
    cl.partials = static_cast<double*>(part.p);
    cl.chunk_cols = cand * E;
    float ms = 0.f;
    HGL_TRY(time_ms(st, [&] { return op_launch(cl, st, nullptr); }, &ms));
    if (best == 0 || ms < best_ms) {
      best = cand;
      best_ms = ms;
    }
    if (cand == nvec) break;
  }
  g->tuned_chunk[tune_key(dtype, c)] = best;
  if (chunk_cols) *chunk_cols = best * E;
  // grid policy at that chunk: the blocks resident at once (one wave) or eight per SM,
  // timed with the same variant
  {
    OpCall cl{};
    cl.g = g;
    cl.xdt = dtype;
    cl.zdt = zdt;
    cl.X = X.p;
    cl.ldx = ld;
    cl.Z = Z.p;
    cl.ldz = ldz;
    cl.c = c;
    cl.a = 1.5;
    cl.b = -1.0;
    cl.epi = EPI_DOT_XZ;
    cl.partials = static_cast<double*>(part.p);
    // the two grids are often within a few percent: alternate them three times, keep
    // each one's best time, and leave the one-wave default unless eight per SM wins
    // by more than 3%
    float ms[2] = {0.f, 0.f};
    for (int rep = 0; rep < 3; ++rep)
      for (int pol = 0; pol < 2; ++pol) {
        g->tuned_chunk[tune_key(TUNE_GRID + dtype, c)] = pol;
        float t = 0.f;
        HGL_TRY(time_ms(st, [&] { return op_launch(cl, st, nullptr); }, &t));
        ms[pol] = rep == 0 ? t : std::min(ms[pol], t);
      }
    g->tuned_chunk[tune_key(TUNE_GRID + dtype, c)] = ms[1] < 0.97f * ms[0] ? 1 : 0;
  }
  if (grid_policy) *grid_policy = g->tuned_chunk[tune_key(TUNE_GRID + dtype, c)];

  // pair-arithmetic residual (used by the FP32 / BF16 solvers): 4-float vectors
  if (dtype != HGL_FP64) {
    const int64_t ld32 = (c + 3) / 4 * 4, ld64 = (c + 1) / 2 * 2;
    const int pvec = (c + 3) / 4;
    DevMem Fh, Fl, Y, R, sc, part;
    HGL_CHECK_CUDA(cudaMalloc(&Fh.p, 4 * (size_t)g->n * ld32));
    HGL_CHECK_CUDA(cudaMalloc(&Fl.p, 4 * (size_t)g->n * ld32));
    HGL_CHECK_CUDA(cudaMalloc(&R.p, 4 * (size_t)g->n * ld32));
    HGL_CHECK_CUDA(cudaMalloc(&Y.p, 8 * (size_t)g->n * ld64));
    HGL_CHECK_CUDA(cudaMalloc(&sc.p, 4 * 2 * (size_t)(g->n + g->m)));
    const int rows = std::max(op_partial_rows(g), g->num_sms * 8);
    HGL_CHECK_CUDA(cudaMalloc(&part.p, 8 * (size_t)rows * c));
    HGL_CHECK_CUDA(cudaMemsetAsync(Fh.p, 0x3F, 4 * (size_t)g->n * ld32, st));
    HGL_CHECK_CUDA(cudaMemsetAsync(Fl.p, 0, 4 * (size_t)g->n * ld32, st));
    HGL_CHECK_CUDA(cudaMemsetAsync(Y.p, 0, 8 * (size_t)g->n * ld64, st));
    float* s_hi = static_cast<float*>(sc.p);
    float* s_lo = s_hi + g->n;
    float* t_hi = s_lo + g->n;
    float* t_lo = t_hi + g->m;
    HGL_TRY(df_split_scalings(g, s_hi, s_lo, t_hi, t_lo, st));
    // both variants: the full pair and the compact one (F's low part gathered in BF16)
    const int64_t ld16 = (c + 7) / 8 * 8;
    DevMem Fl16;
    HGL_CHECK_CUDA(cudaMalloc(&Fl16.p, 2 * (size_t)g->n * ld16));
    HGL_CHECK_CUDA(cudaMemsetAsync(Fl16.p, 0, 2 * (size_t)g->n * ld16, st));
    for (int variant = 0; variant < 2; ++variant) {
      const bf16_t* lo16 = variant ? static_cast<const bf16_t*>(Fl16.p) : nullptr;
      int pbest = 0;
      float pbest_ms = 0.f;
      const uint64_t key = tune_key(variant ? TUNE_PAIR16 : TUNE_PAIR, c);
      for (int vecs : {8, 16, 32, 64, 128}) {
        const int cand = std::min(vecs, pvec);
        g->tuned_chunk[key] = cand;
        float ms = 0.f;
        int r_rows = 0;
        HGL_TRY(time_ms(st, [&] {
          return df_residual(g, s_hi, s_lo, t_hi, t_lo, static_cast<float*>(Fh.p), static_cast<float*>(Fl.p), ld32,
                             static_cast<double*>(Y.p), ld64, -1.5, 1.0, 0.5, c, static_cast<float*>(R.p),
                             static_cast<double*>(part.p), st, &r_rows, nullptr, nullptr, 0, nullptr, lo16, ld16);
        }, &ms));
        if (pbest == 0 || ms < pbest_ms) {
          pbest = cand;
          pbest_ms = ms;
        }
        if (cand == pvec) break;
      }
      g->tuned_chunk[key] = pbest;
      if (pair_chunk_cols && variant == 0) *pair_chunk_cols = pbest * 4;
    }
  } else if (pair_chunk_cols) {
    *pair_chunk_cols = 0;
  }
  HGL_CHECK_CUDA(cudaStreamSynchronize(st));
  return HGL_OK;
}
