// placeholder until the block rSVD preconditioner lands
#include "solver.cuh"
namespace hgl {
hgl_status precond_check(const hgl_precond*, const hgl_graph*, double) {
  return record_error(HGL_ERR_INVALID_ARG, "preconditioner not available");
}
hgl_status precond_apply_launch(const hgl_precond*, const hgl_graph*, const void*, int64_t, void*, int64_t, int,
                                int, double*, cudaStream_t, int*, const int32_t*) {
  return record_error(HGL_ERR_INVALID_ARG, "preconditioner not available");
}
hgl_status precond_build(const hgl_graph*, const double*, double, const int64_t*, int32_t, int32_t, int32_t, int32_t,
                         uint64_t, int, cudaStream_t, hgl_precond**, bool) {
  return record_error(HGL_ERR_INVALID_ARG, "preconditioner not available");
}
}  // namespace hgl
extern "C" void hgl_precond_destroy(hgl_precond*) {}
extern "C" hgl_status hgl_block_rsvd(const hgl_graph*, const double*, double, const int64_t*, int32_t, int32_t,
                                     int32_t, int32_t, uint64_t, hgl_dtype, void*, hgl_precond** out) {
  if (out) *out = nullptr;
  return hgl::record_error(HGL_ERR_INVALID_ARG, "block rSVD not available");
}
extern "C" hgl_status hgl_precond_export(const hgl_precond*, int32_t, double*, double*, int32_t*, void*) {
  return hgl::record_error(HGL_ERR_INVALID_ARG, "block rSVD not available");
}
extern "C" hgl_status hgl_precond_apply(const hgl_precond*, const void*, int64_t, void*, int64_t, int32_t, hgl_dtype,
                                        void*) {
  return hgl::record_error(HGL_ERR_INVALID_ARG, "block rSVD not available");
}
