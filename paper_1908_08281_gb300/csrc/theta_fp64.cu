// theta_fp64.cu -- operator passes with FP64 X panels (FP64 accumulation).
#include "theta_launch.cuh"

namespace hgl {

hgl_status op_launch_fp64(const OpCall& cl, cudaStream_t st, int* grid2) {
  if (cl.zdt == HGL_FP64) {
    switch (cl.epi) {
      case EPI_PLAIN: return op_launch_typed<double, double, double, EPI_PLAIN>(cl, st, grid2);
      case EPI_DOT_XZ: return op_launch_typed<double, double, double, EPI_DOT_XZ>(cl, st, grid2);
      case EPI_RESID: return op_launch_typed<double, double, double, EPI_RESID>(cl, st, grid2);
    }
  } else if (cl.zdt == HGL_FP32 && cl.epi == EPI_RESID) {
    return op_launch_typed<double, double, float, EPI_RESID>(cl, st, grid2);
  }
  return record_error(HGL_ERR_INVALID_ARG, "unsupported operator variant (FP64 X)");
}

}  // namespace hgl
