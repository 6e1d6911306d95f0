// hgl_internal.cuh -- shared internals of libhgl (not part of the ABI).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <map>
#include <vector>
#include <string>

#include "../../include/hgl.h"

// A graph handle: the two compressed layouts of H plus per-graph work buffers.
// Work buffers grow on demand and are reused; calls on one handle are serial.
namespace hgl {

struct Buffer {
  void* ptr = nullptr;
  size_t bytes = 0;
};

// Returns a device buffer of at least `bytes` (contents undefined), or nullptr after
// recording HGL_ERR_OOM / HGL_ERR_CUDA in *st.
void* buffer_get(Buffer& b, size_t bytes, hgl_status* st);
void buffer_free(Buffer& b);

hgl_status record_error(hgl_status s, const char* fmt, ...);
hgl_status cuda_error(cudaError_t e, const char* what, const char* file, int line);

int device_sm_count();

// Blocks of kernel `fn` that fit on one SM at `threads` threads and `smem` bytes of
// dynamic shared memory (occupancy API, cached per kernel and device; 1 on failure).
int resident_blocks(const void* fn, int threads, size_t smem);

constexpr int TUNE_PAIR = 7;
// tune_key(TUNE_PAIR16, c) -> chunk of the compact pair residual (BF16 low parts)
constexpr int TUNE_PAIR16 = 8;
// tune_key(TUNE_GRID + panel kind, c) -> grid policy of the operator's gather passes:
// 1 = eight blocks per SM (several waves), otherwise the blocks resident at once
constexpr int TUNE_GRID = 16;
inline uint64_t tune_key(int kind, int c) { return ((uint64_t)kind << 32) | (uint32_t)c; }
// Tuned chunk in vectors for (kind, c), or 0.
inline int tuned_chunk_vecs(const hgl_graph* g, int kind, int c);

// Rows (hyperedges) longer than this go to a whole thread block in the gather passes.
constexpr int64_t HEAVY_ROW = 128;
// Hyperedges of at most this many members skip the operator's intermediate: the vertex
// pass reads their other members' rows directly.  Per hyperedge of size d that costs
// d (d - 1) row reads instead of d reads, one intermediate row written and d read.
constexpr int SMALL_EDGE = 3;

// Process-wide count of kernels launched by the library (diagnostics).
void count_launch(unsigned n = 1);
void uncount_launch(unsigned long long n);  // launches recorded by a capture, not run
struct StepGraph;
void step_graph_destroy(StepGraph* sg);

// Kernel timing: while profiling is enabled, ProfScope records an event pair on the
// stream around the launches made in its lifetime.  While a stream capture of this
// thread has a sink installed, every ProfScope instead records its pair as event
// nodes of the graph (cudaEventRecordExternal) into the sink, whose times are added
// to the totals after each replay (prof_graph_add).
bool profiling();
int prof_begin(int family, cudaStream_t st);
void prof_end(int token, cudaStream_t st);
struct ProfEvent {
  int family;
  cudaEvent_t start, stop;
};
void prof_capture_begin(std::vector<ProfEvent>* sink);
void prof_capture_end();
bool prof_capturing();
void prof_graph_add(const std::vector<ProfEvent>& recs);   // device synchronised by the caller
void prof_graph_release(std::vector<ProfEvent>& recs);
// Time the statements (launches) passed as the macro's trailing argument on stream `st`.
#define HGL_PROFILED(FAM, ...)                 \
  do {                                         \
    ::hgl::ProfScope hgl_prof_scope_(FAM, st); \
    __VA_ARGS__;                               \
  } while (0)
struct ProfScope {
  int token;
  cudaStream_t st;
  ProfScope(int family, cudaStream_t s)
      : token(profiling() || prof_capturing() ? prof_begin(family, s) : -1), st(s) {}
  ~ProfScope() {
    if (token != -1) prof_end(token, st);
  }
};

}  // namespace hgl

struct hgl_graph {
  int64_t n = 0, m = 0, nnz = 0;
  int device = 0;
  int num_sms = 0;
  int64_t* csc_ptr = nullptr;  // m+1
  int32_t* csc_idx = nullptr;  // nnz, members of each hyperedge ascending
  int64_t* csr_ptr = nullptr;  // n+1
  int32_t* csr_idx = nullptr;  // nnz, hyperedges of each vertex ascending
  int32_t* de = nullptr;       // m
  double* dv = nullptr;        // n   (for the w of the last degrees call)
  double* s = nullptr;         // n   dv^-1/2 (0 where dv <= 0)
  double* t = nullptr;         // m   w / de
  float* s32 = nullptr;        // n   s rounded to FP32 (scalings of the FP32/BF16 kernels)
  float* t32 = nullptr;        // m   t rounded to FP32
  hgl::Buffer scratch;         // m x chunk intermediate panel of the operator
  hgl::Buffer scratch2;        // second intermediate panel (bilinear gradient)
  hgl::Buffer partials;        // per-block reduction partials
  hgl::Buffer solver;          // CG panels and per-column state
  hgl::Buffer misc;            // gradient vectors (ex[m], phi[n])
  hgl::Buffer step;            // adaptive-step vectors (grad, w_old, projection work)
  hgl::Buffer rsvd;            // block rSVD work space (dense blocks, bases, Grams)
  hgl::Buffer edge_tf;         // m x c FP32 t * (H^T s F) from the pair residual, for the gradient
  int block_product = HGL_BLOCKS_AUTO;  // route of the rSVD's products Theta_bb S
  int chunk_cols = 0;          // operator column chunk (0 = library default)
  // hyperedges in decreasing size order; the first nheavy (size > HEAVY_ROW) are
  // processed by a whole thread block each, the rest by one warp each in this order
  int32_t* edge_order = nullptr;  // m
  int64_t nheavy = 0;
  // Split of Theta for the operator: hyperedges with more than SMALL_EDGE members (the
  // first m_large of edge_order) go through the m_large x chunk intermediate, indexed
  // by their position in edge_order (their slot); smaller ones enter the vertex pass
  // directly as vertex-to-vertex terms t_e s_v X[v] (and a diagonal term).
  int64_t m_large = 0;
  int64_t* lcsr_ptr = nullptr;  // n+1
  int32_t* lcsr_idx = nullptr;  // slots of each vertex's large hyperedges, hyperedge order
  int64_t* scsr_ptr = nullptr;  // n+1
  int32_t* scsr_v = nullptr;    // per vertex, over its small hyperedges: the other members
  int32_t* scsr_e = nullptr;    //   and the hyperedge they share
  double* scoef = nullptr;      // t_e s_v per small entry (for the w of the last degrees call)
  float* scoef32 = nullptr;
  double* sdiag = nullptr;      // n: s_v^2 sum of t_e over the small hyperedges of v
  float* sdiag32 = nullptr;
  // column chunk (in 16-byte vectors per row) chosen by hgl_tune_operator, keyed by
  // (panel kind, c); kind = HGL_FP64/FP32/BF16 for the operator, TUNE_PAIR for the
  // pair-arithmetic residual
  std::map<uint64_t, int> tuned_chunk;
  // the captured CUDA graph of hgl_adaptive_step (HGL_STEP_GRAPH), if any
  hgl::StepGraph* step_graph = nullptr;
};

#define HGL_CHECK_CUDA(call)                                                   \
  do {                                                                         \
    cudaError_t e_ = (call);                                                   \
    if (e_ != cudaSuccess) return ::hgl::cuda_error(e_, #call, __FILE__, __LINE__); \
  } while (0)

#define HGL_TRY(expr)                                      \
  do {                                                     \
    hgl_status hgl_try_status_ = (expr);                   \
    if (hgl_try_status_ != HGL_OK) return hgl_try_status_; \
  } while (0)

namespace hgl {

inline cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

inline bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// Panel argument check: device pointer 16-byte aligned, ld >= c, ld * elt % 16 == 0.
inline hgl_status check_panel(const void* p, int64_t ld, int32_t c, size_t elt, const char* name) {
  if (p == nullptr) return record_error(HGL_ERR_INVALID_ARG, "%s is NULL", name);
  if (!aligned16(p)) return record_error(HGL_ERR_INVALID_ARG, "%s is not 16-byte aligned", name);
  if (ld < c) return record_error(HGL_ERR_INVALID_ARG, "leading dimension of %s is below c", name);
  if ((ld * (int64_t)elt) % 16 != 0)
    return record_error(HGL_ERR_INVALID_ARG, "leading dimension of %s times element size is not a multiple of 16 bytes", name);
  return HGL_OK;
}

inline size_t dtype_size(int dt) { return dt == HGL_FP64 ? 8 : (dt == HGL_FP32 ? 4 : 2); }

// ---------------------------------------------------------------------------
// operator internals (theta.cu)
// ---------------------------------------------------------------------------

// Epilogues of the vertex pass of the operator.
enum Epilogue : int {
  EPI_PLAIN = 0,   // Z = a X + b s (H T)
  EPI_DOT_XZ = 1,  // same, plus per-column partial sums of X.Z      (CG: p^T M p)
  EPI_RESID = 2,   // Z = gy Y + a X + b s (H T), plus partial sums of Z.Z (residual)
};

struct OpCall {
  const hgl_graph* g;
  int xdt;          // element type of X (HGL_FP64/FP32/BF16)
  int zdt;          // element type of Z
  const void* X; int64_t ldx;
  void* Z; int64_t ldz;
  int32_t c;
  double a, b;
  int epi;
  const double* Y; int64_t ldy; double gy;   // EPI_RESID only (FP64 Y)
  double* partials;  // EPI_DOT_XZ / EPI_RESID: [grid2 x c] FP64 partial sums (row stride c)
  const int32_t* run_flag;  // optional device flag: kernels return at once when *run_flag == 0
  int chunk_cols;   // 0 = default column chunk
  void* scratch;        // optional caller-provided intermediate panel (nullptr = graph-owned buffer)
  size_t scratch_bytes; // its capacity; the column chunk is narrowed to fit
};

// Launch both passes of the operator over all column chunks.  Returns the number of
// blocks of the vertex pass (the row count of `partials`) in *grid2.
hgl_status op_launch(const OpCall& call, cudaStream_t st, int* grid2);

// Blocks the vertex pass will use (for sizing `partials`).
int op_partial_rows(const hgl_graph* g);

// Recompute dv, s, t for w into the graph's vectors.
hgl_status degrees_launch(const hgl_graph* g, const double* w, cudaStream_t st);

}  // namespace hgl

namespace hgl {
// The scalings s = dv^-1/2 and t = w/de in the accumulation type A of a kernel: FP64
// kernels read the FP64 vectors, FP32 ones the FP32 copies (the same values the
// kernels would get by rounding on every load, without an FP64 conversion per gather).
template <class A> inline const A* scal_s(const hgl_graph* g);
template <> inline const double* scal_s<double>(const hgl_graph* g) { return g->s; }
template <> inline const float* scal_s<float>(const hgl_graph* g) { return g->s32; }
template <class A> inline const A* scal_coef(const hgl_graph* g);
template <> inline const double* scal_coef<double>(const hgl_graph* g) { return g->scoef; }
template <> inline const float* scal_coef<float>(const hgl_graph* g) { return g->scoef32; }
template <class A> inline const A* scal_diag(const hgl_graph* g);
template <> inline const double* scal_diag<double>(const hgl_graph* g) { return g->sdiag; }
template <> inline const float* scal_diag<float>(const hgl_graph* g) { return g->sdiag32; }
template <class A> inline const A* scal_t(const hgl_graph* g);
template <> inline const double* scal_t<double>(const hgl_graph* g) { return g->t; }
template <> inline const float* scal_t<float>(const hgl_graph* g) { return g->t32; }
}  // namespace hgl

inline int hgl::tuned_chunk_vecs(const hgl_graph* g, int kind, int c) {
  auto it = g->tuned_chunk.find(tune_key(kind, c));
  return it == g->tuned_chunk.end() ? 0 : it->second;
}
