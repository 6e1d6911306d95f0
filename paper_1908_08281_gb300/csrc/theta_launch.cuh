// theta_launch.cuh -- host-side launch of the two operator passes over column chunks.
#pragma once

#include "theta_kernels.cuh"

namespace hgl {

// Default chunk width in 16-byte vectors per row (512 bytes of X per row).
inline int default_chunk_vecs() { return 32; }

// Blocks of the hyperedge pass: one per heavy hyperedge, then enough for the light
// rows, capped at the blocks that are resident at once (per_sm per SM, at most 8) so
// that the light part runs in a single wave; warps stride over the remaining rows.
inline int edge_grid(const hgl_graph* g, int per_sm = 8) {
  const int64_t light = g->m_large - g->nheavy;
  int64_t need = (light + OP_WARPS - 1) / OP_WARPS;
  int64_t cap = (int64_t)g->num_sms * (per_sm < 8 ? per_sm : 8);
  return (int)(g->nheavy + (need < cap ? (need > 0 ? need : 1) : cap));
}

// Blocks of the vertex pass (also the row count of its reduction partials); the
// default is the largest grid any instantiation uses.
inline int vertex_grid(const hgl_graph* g, int per_sm = 8) {
  int64_t need = (g->n + OP_WARPS - 1) / OP_WARPS;
  int64_t cap = (int64_t)g->num_sms * (per_sm < 8 ? per_sm : 8);
  return (int)(need < cap ? (need > 0 ? need : 1) : cap);
}

template <class TX, class TT, class TZ, int EPI>
hgl_status op_launch_typed(const OpCall& cl, cudaStream_t st, int* grid2_out) {
  hgl_graph* g = const_cast<hgl_graph*>(cl.g);
  constexpr int E = 16 / (int)sizeof(TX);
  const int nvec = (cl.c + E - 1) / E;
  const int tuned = tuned_chunk_vecs(g, cl.xdt, cl.c);
  int chunk_vec = cl.chunk_cols > 0 ? (cl.chunk_cols + E - 1) / E : (tuned > 0 ? tuned : default_chunk_vecs());
  if (chunk_vec > nvec) chunk_vec = nvec;
  if (chunk_vec < 1) chunk_vec = 1;
  if (cl.scratch) {
    // narrow the chunk to the largest tile whose m x chunk panel fits the given scratch
    const int64_t rows = g->m_large > 0 ? g->m_large : 1;
    const size_t per_vec = (size_t)rows * E * sizeof(TT);
    const size_t cap = per_vec ? cl.scratch_bytes / per_vec : 0;
    if (cap < 1)
      return record_error(HGL_ERR_INVALID_ARG, "m = %lld is too large for the %zu-byte scratch",
                          (long long)g->m, cl.scratch_bytes);
    int fit = cap >= 128 ? 128 : (cap >= 64 ? 64 : 1);
    if (cap < 64)
      while (fit * 2 <= (int)cap && fit < 32) fit *= 2;
    if (chunk_vec > fit) chunk_vec = fit;
  }
  int lg = 1, nv = 1;
  pick_tile(chunk_vec, &lg, &nv);
  const int cc = lg * nv * E;
  hgl_status stt = HGL_OK;
  const size_t trows = (size_t)(g->m_large > 0 ? g->m_large : 1);
  TT* Tp = cl.scratch ? static_cast<TT*>(cl.scratch)
                      : static_cast<TT*>(buffer_get(g->scratch, sizeof(TT) * trows * (size_t)cc, &stt));
  if (!Tp) return stt;
  int grid2 = vertex_grid(g);
  using A = typename AccOf<TX>::type;
  const A* sA = scal_s<A>(g);
  const A* tA = scal_t<A>(g);
  const SmallTerms<A> smt{g->scsr_ptr, g->scsr_v, scal_coef<A>(g), scal_diag<A>(g)};
  const bool edge_pass = g->m_large > 0;
  const bool eight_per_sm = tuned_chunk_vecs(g, TUNE_GRID + cl.xdt, cl.c) == 1;
  auto per_sm = [&](const void* fn) { return eight_per_sm ? 8 : resident_blocks(fn, OP_THREADS, 0); };
  ProfScope prof(cl.epi == EPI_RESID ? HGL_PROF_OPRESID : HGL_PROF_OPERATOR, st);
  const TX* X = static_cast<const TX*>(cl.X);
  TZ* Z = static_cast<TZ*>(cl.Z);
  for (int c0 = 0; c0 < cl.c; c0 += cc) {
    const int cw = cl.c - c0 < cc ? cl.c - c0 : cc;
#define HGL_EDGE_CASE(LG_, NV_)                                                                        \
  else if (lg == LG_ && nv == NV_) {                                                                   \
    auto fn = k_edge_pass<TX, TT, LG_, NV_>;                                                           \
    const int gr = edge_grid(g, per_sm(reinterpret_cast<const void*>(fn)));    \
    hgl::count_launch();                                                                               \
    fn<<<gr, OP_THREADS, 0, st>>>(g->m_large, g->csc_ptr, g->csc_idx, g->edge_order, g->nheavy, sA,    \
                                  tA, X, cl.ldx, c0, cw, Tp, (int64_t)cc, cl.run_flag);                \
  }
#define HGL_VERTEX_CASE(LG_, NV_)                                                                      \
  else if (lg == LG_ && nv == NV_) {                                                                   \
    auto fn = k_vertex_pass<TX, TT, TZ, LG_, NV_, EPI>;                                                \
    grid2 = vertex_grid(g, per_sm(reinterpret_cast<const void*>(fn)));         \
    hgl::count_launch();                                                                               \
    fn<<<grid2, OP_THREADS, 0, st>>>(g->n, g->lcsr_ptr, g->lcsr_idx, smt, sA, Tp, (int64_t)cc, X,      \
                                     cl.ldx, Z,                                                        \
                                     cl.ldz, c0, cw, cl.c, cl.a, cl.b, cl.Y, cl.ldy, cl.gy, cl.partials, \
                                     cl.run_flag);                                                     \
  }
#define HGL_EDGE_ROWS(LG_)                                                                             \
  else if (lg == LG_) {                                                                                \
    auto fn = k_edge_rows<TX, TT, LG_>;                                                                \
    const int gr = edge_grid(g, per_sm(reinterpret_cast<const void*>(fn)));    \
    hgl::count_launch();                                                                               \
    fn<<<gr, OP_THREADS, 0, st>>>(g->m_large, g->csc_ptr, g->csc_idx, g->edge_order, g->nheavy, sA,    \
                                  tA, X, cl.ldx, c0, cw, Tp, (int64_t)cc, cl.run_flag);                \
  }
#define HGL_VERTEX_ROWS(LG_)                                                                           \
  else if (lg == LG_) {                                                                                \
    auto fn = k_vertex_rows<TX, TT, TZ, LG_, EPI>;                                                     \
    grid2 = vertex_grid(g, per_sm(reinterpret_cast<const void*>(fn)));         \
    hgl::count_launch();                                                                               \
    fn<<<grid2, OP_THREADS, 0, st>>>(g->n, g->lcsr_ptr, g->lcsr_idx, smt, sA, Tp, (int64_t)cc, X,      \
                                     cl.ldx, Z,                                                        \
                                     cl.ldz, c0, cw, cl.c, cl.a, cl.b, cl.Y, cl.ldy, cl.gy, cl.partials, \
                                     cl.run_flag);                                                     \
  }
    if (nv == 1 && lg <= 8) {
      // narrow chunk: one row per group of lanes
      if (!edge_pass) {
      }
      HGL_FOR_EACH_ROW_LG(HGL_EDGE_ROWS)
      if (false) {
      }
      HGL_FOR_EACH_ROW_LG(HGL_VERTEX_ROWS)
    } else {
      if (!edge_pass) {
      }
      HGL_FOR_EACH_WIDE_TILE(HGL_EDGE_CASE)
      if (false) {
      }
      HGL_FOR_EACH_WIDE_TILE(HGL_VERTEX_CASE)
    }
#undef HGL_EDGE_CASE
#undef HGL_VERTEX_CASE
#undef HGL_EDGE_ROWS
#undef HGL_VERTEX_ROWS
    HGL_CHECK_CUDA(cudaGetLastError());
  }
  if (grid2_out) *grid2_out = grid2;
  return HGL_OK;
}

hgl_status op_launch_fp64(const OpCall& cl, cudaStream_t st, int* grid2);
hgl_status op_launch_fp32(const OpCall& cl, cudaStream_t st, int* grid2);
hgl_status op_launch_bf16(const OpCall& cl, cudaStream_t st, int* grid2);

}  // namespace hgl
