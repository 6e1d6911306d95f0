// api.cu -- status strings, error recording, work buffers, graph queries and the
// degree/scaling kernel (Section 2: dv = H w, de = H^T 1; Eq. 1 scalings).
#include <atomic>
#include <cstdarg>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "hgl_internal.cuh"

namespace hgl {

static thread_local char g_last_error[512] = "";
static std::atomic<unsigned long long> g_launches{0};

void count_launch(unsigned n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
void uncount_launch(unsigned long long n) { g_launches.fetch_sub(n, std::memory_order_relaxed); }

namespace {
struct ProfRecord {
  int family;
  cudaEvent_t start, stop;
};
std::mutex g_prof_mutex;
std::atomic<bool> g_prof_on{false};
std::vector<ProfRecord> g_prof_records;   // recorded, not yet read
std::vector<cudaEvent_t> g_prof_pool;     // free events
double g_prof_ms[HGL_PROF_FAMILIES] = {};
int64_t g_prof_count[HGL_PROF_FAMILIES] = {};

cudaEvent_t pool_get() {
  if (!g_prof_pool.empty()) {
    cudaEvent_t e = g_prof_pool.back();
    g_prof_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

// fold finished records into the totals (caller holds the mutex, device synchronised)
void prof_drain() {
  for (auto& r : g_prof_records) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, r.start, r.stop) == cudaSuccess) {
      g_prof_ms[r.family] += ms;
      g_prof_count[r.family] += 1;
    }
    g_prof_pool.push_back(r.start);
    g_prof_pool.push_back(r.stop);
  }
  g_prof_records.clear();
}
}  // namespace

bool profiling() { return g_prof_on.load(std::memory_order_relaxed); }

static thread_local std::vector<ProfEvent>* t_capture_sink = nullptr;

void prof_capture_begin(std::vector<ProfEvent>* sink) { t_capture_sink = sink; }
void prof_capture_end() { t_capture_sink = nullptr; }
bool prof_capturing() { return t_capture_sink != nullptr; }

// tokens >= 0 index the pending records; tokens <= -2 index the capture sink
int prof_begin(int family, cudaStream_t st) {
  std::lock_guard<std::mutex> lock(g_prof_mutex);
  ProfRecord r{family, pool_get(), pool_get()};
  if (!r.start || !r.stop) return -1;
  if (t_capture_sink) {
    if (cudaEventRecordWithFlags(r.start, st, cudaEventRecordExternal) != cudaSuccess) return -1;
    t_capture_sink->push_back(ProfEvent{family, r.start, r.stop});
    return -2 - ((int)t_capture_sink->size() - 1);
  }
  if (cudaEventRecord(r.start, st) != cudaSuccess) return -1;
  g_prof_records.push_back(r);
  return (int)g_prof_records.size() - 1;
}

void prof_end(int token, cudaStream_t st) {
  std::lock_guard<std::mutex> lock(g_prof_mutex);
  if (token <= -2) {
    const int i = -2 - token;
    if (t_capture_sink && i < (int)t_capture_sink->size())
      cudaEventRecordWithFlags((*t_capture_sink)[i].stop, st, cudaEventRecordExternal);
    return;
  }
  if (token >= 0 && token < (int)g_prof_records.size()) cudaEventRecord(g_prof_records[token].stop, st);
}

void prof_graph_add(const std::vector<ProfEvent>& recs) {
  if (!profiling()) return;
  std::lock_guard<std::mutex> lock(g_prof_mutex);
  for (const auto& r : recs) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, r.start, r.stop) == cudaSuccess) {
      g_prof_ms[r.family] += ms;
      g_prof_count[r.family] += 1;
    } else {
      (void)cudaGetLastError();
    }
  }
}

void prof_graph_release(std::vector<ProfEvent>& recs) {
  std::lock_guard<std::mutex> lock(g_prof_mutex);
  for (const auto& r : recs) {
    g_prof_pool.push_back(r.start);
    g_prof_pool.push_back(r.stop);
  }
  recs.clear();
}

hgl_status record_error(hgl_status s, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_last_error, sizeof(g_last_error), fmt, ap);
  va_end(ap);
  return s;
}

hgl_status cuda_error(cudaError_t e, const char* what, const char* file, int line) {
  const char* f = strrchr(file, '/');
  f = f ? f + 1 : file;
  record_error(e == cudaErrorMemoryAllocation ? HGL_ERR_OOM : HGL_ERR_CUDA, "%s failed: %s (%s:%d)", what,
               cudaGetErrorString(e), f, line);
  return e == cudaErrorMemoryAllocation ? HGL_ERR_OOM : HGL_ERR_CUDA;
}

void* buffer_get(Buffer& b, size_t bytes, hgl_status* st) {
  if (bytes == 0) bytes = 16;
  if (b.bytes >= bytes) return b.ptr;
  if (b.ptr) {
    cudaError_t e = cudaFree(b.ptr);
    b.ptr = nullptr;
    b.bytes = 0;
    if (e != cudaSuccess) {
      *st = cuda_error(e, "cudaFree(work buffer)", __FILE__, __LINE__);
      return nullptr;
    }
  }
  size_t want = bytes + bytes / 8;  // headroom for slightly larger later calls
  cudaError_t e = cudaMalloc(&b.ptr, want);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    b.ptr = nullptr;
    *st = cuda_error(e, "cudaMalloc(work buffer)", __FILE__, __LINE__);
    return nullptr;
  }
  b.bytes = want;
  return b.ptr;
}

void buffer_free(Buffer& b) {
  if (b.ptr) cudaFree(b.ptr);
  b.ptr = nullptr;
  b.bytes = 0;
}

int resident_blocks(const void* fn, int threads, size_t smem) {
  static std::mutex mu;
  static std::map<std::tuple<const void*, int, int, size_t>, int> cache;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 1;
  const auto key = std::make_tuple(fn, dev, threads, smem);
  std::lock_guard<std::mutex> lock(mu);
  auto it = cache.find(key);
  if (it != cache.end()) return it->second;
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, threads, smem) != cudaSuccess || nb < 1) {
    (void)cudaGetLastError();
    nb = 1;
  }
  cache[key] = nb;
  return nb;
}

int device_sm_count() {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 1;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 1;
  return sms > 0 ? sms : 1;
}

// dv_v = sum_{e in row v} w_e (row order), s_v = dv^-1/2 or 0;  t_e = w_e / de_e.
__global__ void k_degrees(int64_t n, int64_t m, const int64_t* __restrict__ csr_ptr,
                          const int32_t* __restrict__ csr_idx, const int32_t* __restrict__ de,
                          const double* __restrict__ w, double* __restrict__ dv,
                          double* __restrict__ s, double* __restrict__ t, float* __restrict__ s32,
                          float* __restrict__ t32) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += stride) {
    double acc = 0.0;
    for (int64_t i = csr_ptr[v], end = csr_ptr[v + 1]; i < end; ++i) acc += w[csr_idx[i]];
    dv[v] = acc;
    const double sv = acc > 0.0 ? 1.0 / sqrt(acc) : 0.0;
    s[v] = sv;
    s32[v] = (float)sv;
  }
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m; e += stride) {
    const double te = w[e] / (double)de[e];
    t[e] = te;
    t32[e] = (float)te;
  }
}

// The operator's small-hyperedge terms at the current scalings: per entry (v, e) of a
// vertex u the coefficient t_e s_v, per vertex s_u^2 times the sum of t_e over its small
// hyperedges (hyperedge order).
__global__ void k_small_coef(int64_t n, const int64_t* __restrict__ csr_ptr, const int32_t* __restrict__ csr_idx,
                             const int32_t* __restrict__ de, const int64_t* __restrict__ sptr,
                             const int32_t* __restrict__ sv, const int32_t* __restrict__ se,
                             const double* __restrict__ s, const double* __restrict__ t,
                             double* __restrict__ coef, float* __restrict__ coef32, double* __restrict__ diag,
                             float* __restrict__ diag32) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < n; u += stride) {
    double d = 0.0;
    for (int64_t i = csr_ptr[u], end = csr_ptr[u + 1]; i < end; ++i) {
      const int32_t e = csr_idx[i];
      if (de[e] <= SMALL_EDGE) d += t[e];
    }
    const double su = s[u];
    diag[u] = su * su * d;
    diag32[u] = (float)(su * su * d);
    for (int64_t k = sptr[u], end = sptr[u + 1]; k < end; ++k) {
      const double cf = t[se[k]] * s[sv[k]];
      coef[k] = cf;
      coef32[k] = (float)cf;
    }
  }
}

hgl_status degrees_launch(const hgl_graph* g, const double* w, cudaStream_t st) {
  int blocks = g->num_sms * 8;
  hgl::count_launch(); k_degrees<<<blocks, 256, 0, st>>>(g->n, g->m, g->csr_ptr, g->csr_idx, g->de, w, g->dv, g->s, g->t,
                                                         g->s32, g->t32);
  HGL_CHECK_CUDA(cudaGetLastError());
  hgl::count_launch();
  k_small_coef<<<blocks, 256, 0, st>>>(g->n, g->csr_ptr, g->csr_idx, g->de, g->scsr_ptr, g->scsr_v, g->scsr_e, g->s,
                                       g->t, g->scoef, g->scoef32, g->sdiag, g->sdiag32);
  HGL_CHECK_CUDA(cudaGetLastError());
  return HGL_OK;
}

}  // namespace hgl

extern "C" {

const char* hgl_status_string(hgl_status s) {
  switch (s) {
    case HGL_OK: return "HGL_OK";
    case HGL_ERR_INVALID_ARG: return "HGL_ERR_INVALID_ARG";
    case HGL_ERR_INDEX_RANGE: return "HGL_ERR_INDEX_RANGE";
    case HGL_ERR_DUPLICATE_MEMBER: return "HGL_ERR_DUPLICATE_MEMBER";
    case HGL_ERR_EMPTY_EDGE: return "HGL_ERR_EMPTY_EDGE";
    case HGL_ERR_OOM: return "HGL_ERR_OOM";
    case HGL_ERR_CUDA: return "HGL_ERR_CUDA";
    case HGL_ERR_NOT_CONVERGED: return "HGL_ERR_NOT_CONVERGED";
    case HGL_ERR_TIMEOUT: return "HGL_ERR_TIMEOUT";
    case HGL_ERR_NONFINITE: return "HGL_ERR_NONFINITE";
    default: return "HGL_ERR_UNKNOWN";
  }
}

const char* hgl_last_error(void) { return hgl::g_last_error; }

int32_t hgl_version(void) { return 100; }

uint64_t hgl_launch_count(void) { return hgl::g_launches.load(std::memory_order_relaxed); }

hgl_status hgl_profile_enable(int32_t on) {
  std::lock_guard<std::mutex> lock(hgl::g_prof_mutex);
  if (on) {
    HGL_CHECK_CUDA(cudaDeviceSynchronize());
    hgl::prof_drain();
    for (int f = 0; f < HGL_PROF_FAMILIES; ++f) {
      hgl::g_prof_ms[f] = 0.0;
      hgl::g_prof_count[f] = 0;
    }
  }
  hgl::g_prof_on.store(on != 0);
  return HGL_OK;
}

hgl_status hgl_profile_read(int32_t family, double* ms_total, int64_t* launches) {
  if (family < 0 || family >= HGL_PROF_FAMILIES) return hgl::record_error(HGL_ERR_INVALID_ARG, "unknown family");
  std::lock_guard<std::mutex> lock(hgl::g_prof_mutex);
  HGL_CHECK_CUDA(cudaDeviceSynchronize());
  hgl::prof_drain();
  if (ms_total) *ms_total = hgl::g_prof_ms[family];
  if (launches) *launches = hgl::g_prof_count[family];
  return HGL_OK;
}

void hgl_graph_destroy(hgl_graph* g) {
  if (g) hgl::step_graph_destroy(g->step_graph);
  if (!g) return;
  cudaFree(g->csc_ptr);
  cudaFree(g->csc_idx);
  cudaFree(g->csr_ptr);
  cudaFree(g->csr_idx);
  cudaFree(g->de);
  cudaFree(g->dv);
  cudaFree(g->s);
  cudaFree(g->t);
  cudaFree(g->s32);
  cudaFree(g->t32);
  cudaFree(g->edge_order);
  cudaFree(g->lcsr_ptr);
  cudaFree(g->lcsr_idx);
  cudaFree(g->scsr_ptr);
  cudaFree(g->scsr_v);
  cudaFree(g->scsr_e);
  cudaFree(g->scoef);
  cudaFree(g->scoef32);
  cudaFree(g->sdiag);
  cudaFree(g->sdiag32);
  hgl::buffer_free(g->scratch);
  hgl::buffer_free(g->scratch2);
  hgl::buffer_free(g->partials);
  hgl::buffer_free(g->solver);
  hgl::buffer_free(g->misc);
  hgl::buffer_free(g->step);
  hgl::buffer_free(g->rsvd);
  hgl::buffer_free(g->edge_tf);
  delete g;
}

hgl_status hgl_graph_info(const hgl_graph* g, int64_t* n, int64_t* m, int64_t* nnz) {
  if (!g) return hgl::record_error(HGL_ERR_INVALID_ARG, "graph is NULL");
  if (n) *n = g->n;
  if (m) *m = g->m;
  if (nnz) *nnz = g->nnz;
  return HGL_OK;
}

hgl_status hgl_graph_export(const hgl_graph* g, int64_t* csc_ptr, int32_t* csc_idx, int64_t* csr_ptr,
                            int32_t* csr_idx, int32_t* de, void* stream) {
  if (!g) return hgl::record_error(HGL_ERR_INVALID_ARG, "graph is NULL");
  cudaStream_t st = hgl::as_stream(stream);
  if (csc_ptr)
    HGL_CHECK_CUDA(cudaMemcpyAsync(csc_ptr, g->csc_ptr, sizeof(int64_t) * (g->m + 1), cudaMemcpyDeviceToDevice, st));
  if (csc_idx)
    HGL_CHECK_CUDA(cudaMemcpyAsync(csc_idx, g->csc_idx, sizeof(int32_t) * g->nnz, cudaMemcpyDeviceToDevice, st));
  if (csr_ptr)
    HGL_CHECK_CUDA(cudaMemcpyAsync(csr_ptr, g->csr_ptr, sizeof(int64_t) * (g->n + 1), cudaMemcpyDeviceToDevice, st));
  if (csr_idx)
    HGL_CHECK_CUDA(cudaMemcpyAsync(csr_idx, g->csr_idx, sizeof(int32_t) * g->nnz, cudaMemcpyDeviceToDevice, st));
  if (de) HGL_CHECK_CUDA(cudaMemcpyAsync(de, g->de, sizeof(int32_t) * g->m, cudaMemcpyDeviceToDevice, st));
  return HGL_OK;
}

hgl_status hgl_degrees(const hgl_graph* g, const double* w, double* dv, double* s, double* t, void* stream) {
  if (!g || !w) return hgl::record_error(HGL_ERR_INVALID_ARG, "graph or w is NULL");
  cudaStream_t st = hgl::as_stream(stream);
  HGL_TRY(hgl::degrees_launch(g, w, st));
  if (dv) HGL_CHECK_CUDA(cudaMemcpyAsync(dv, g->dv, sizeof(double) * g->n, cudaMemcpyDeviceToDevice, st));
  if (s) HGL_CHECK_CUDA(cudaMemcpyAsync(s, g->s, sizeof(double) * g->n, cudaMemcpyDeviceToDevice, st));
  if (t) HGL_CHECK_CUDA(cudaMemcpyAsync(t, g->t, sizeof(double) * g->m, cudaMemcpyDeviceToDevice, st));
  return HGL_OK;
}

}  // extern "C"
