// noalloc.cu -- hgl_apply_theta_noalloc: the operator apply of hgl_apply_theta for
// callers that must not allocate device memory during the call.
//
// hgl_apply_theta keeps its m x chunk intermediate panel in a buffer that the graph
// handle allocates with cudaMalloc on first use (and re-allocates when a larger
// chunk is needed).  Some callers cannot let that happen inside the call: programs
// that hand all device memory to their own pool or run under a fixed memory budget,
// and latency-sensitive loops that cannot afford the implicit synchronisation of a
// cudaMalloc/cudaFree.  This variant uses instead a fixed scratch array that lives in
// the library's own device image, so the call itself allocates nothing.
#include <mutex>

#include "hgl_internal.cuh"

namespace hgl {
namespace {

// 32 MiB of intermediate-panel scratch.  Every GPU that loads libhgl holds it until
// the process exits.  It caps the column chunk so that the m x chunk panel fits;
// the narrowest chunk takes 16 bytes per hyperedge for FP64 and FP32 panels and 32
// bytes for BF16 panels, so a call needs m <= 2,097,152 (FP64, FP32) or
// m <= 1,048,576 (BF16).
constexpr size_t kNoAllocScratchBytes = size_t(32) << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_addr_mutex;
void* g_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device.  In host code the
// array's name is only a host-side stand-in, so the address is looked up once per
// device with that device current, and cached.
hgl_status scratch_address(void** out) {
  int dev = 0;
  HGL_CHECK_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return record_error(HGL_ERR_INVALID_ARG, "device ordinal %d out of range", dev);
  std::lock_guard<std::mutex> lock(g_addr_mutex);
  if (!g_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_error(e, "cudaGetSymbolAddress(no-allocation scratch)", __FILE__, __LINE__);
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return HGL_OK;
}

}  // namespace
}  // namespace hgl

extern "C" hgl_status hgl_apply_theta_noalloc(const hgl_graph* g, const double* w, double a, double b,
                                              const void* X, int64_t ldx, void* Z, int64_t ldz, int32_t c,
                                              hgl_dtype dtype, void* stream) {
  if (!g || !w) return hgl::record_error(HGL_ERR_INVALID_ARG, "graph or w is NULL");
  if (c < 1) return hgl::record_error(HGL_ERR_INVALID_ARG, "c must be >= 1");
  if (dtype != HGL_FP64 && dtype != HGL_FP32 && dtype != HGL_BF16)
    return hgl::record_error(HGL_ERR_INVALID_ARG, "unknown dtype");
  const size_t elt = hgl::dtype_size(dtype);
  HGL_TRY(hgl::check_panel(X, ldx, c, elt, "X"));
  HGL_TRY(hgl::check_panel(Z, ldz, c, elt, "Z"));
  // one 16-byte vector of the intermediate panel per hyperedge is the narrowest chunk
  const size_t tt = dtype == HGL_FP64 ? 8 : 4;
  const size_t narrowest = (size_t)g->m * (16 / elt) * tt;
  if (narrowest > hgl::kNoAllocScratchBytes)
    return hgl::record_error(HGL_ERR_INVALID_ARG,
                             "m = %lld needs %zu bytes of scratch for the narrowest chunk; the limit is %zu",
                             (long long)g->m, narrowest, hgl::kNoAllocScratchBytes);
  void* scratch = nullptr;
  HGL_TRY(hgl::scratch_address(&scratch));
  cudaStream_t st = hgl::as_stream(stream);
  HGL_TRY(hgl::degrees_launch(g, w, st));
  hgl::OpCall cl{};
  cl.g = g;
  cl.xdt = dtype;
  cl.zdt = dtype;
  cl.X = X;
  cl.ldx = ldx;
  cl.Z = Z;
  cl.ldz = ldz;
  cl.c = c;
  cl.a = a;
  cl.b = b;
  cl.epi = hgl::EPI_PLAIN;
  cl.scratch = scratch;
  cl.scratch_bytes = hgl::kNoAllocScratchBytes;
  return hgl::op_launch(cl, st, nullptr);
}
