// theta.cu -- hgl_apply_theta: Z = a X + b Theta(w) X (Eq. 1), matrix-free.
#include "theta_launch.cuh"

namespace hgl {

int op_partial_rows(const hgl_graph* g) { return vertex_grid(g); }

hgl_status op_launch(const OpCall& cl, cudaStream_t st, int* grid2) {
  switch (cl.xdt) {
    case HGL_FP64: return op_launch_fp64(cl, st, grid2);
    case HGL_FP32: return op_launch_fp32(cl, st, grid2);
    case HGL_BF16: return op_launch_bf16(cl, st, grid2);
  }
  return record_error(HGL_ERR_INVALID_ARG, "unknown panel type");
}

}  // namespace hgl

extern "C" hgl_status hgl_apply_theta(const hgl_graph* g, const double* w, double a, double b, const void* X,
                                      int64_t ldx, void* Z, int64_t ldz, int32_t c, hgl_dtype dtype,
                                      void* stream) {
  if (!g || !w) return hgl::record_error(HGL_ERR_INVALID_ARG, "graph or w is NULL");
  if (c < 1) return hgl::record_error(HGL_ERR_INVALID_ARG, "c must be >= 1");
  if (dtype != HGL_FP64 && dtype != HGL_FP32 && dtype != HGL_BF16)
    return hgl::record_error(HGL_ERR_INVALID_ARG, "unknown dtype");
  const size_t elt = hgl::dtype_size(dtype);
  HGL_TRY(hgl::check_panel(X, ldx, c, elt, "X"));
  HGL_TRY(hgl::check_panel(Z, ldz, c, elt, "Z"));
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
  return hgl::op_launch(cl, st, nullptr);
}
