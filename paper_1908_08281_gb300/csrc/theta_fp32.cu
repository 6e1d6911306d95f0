// theta_fp32.cu -- operator passes with FP32 X panels (FP32 accumulation, compensated dots).
#include "theta_launch.cuh"

namespace hgl {

hgl_status op_launch_fp32(const OpCall& cl, cudaStream_t st, int* grid2) {
  if (cl.zdt == HGL_FP32) {
    switch (cl.epi) {
      case EPI_PLAIN: return op_launch_typed<float, float, float, EPI_PLAIN>(cl, st, grid2);
      case EPI_DOT_XZ: return op_launch_typed<float, float, float, EPI_DOT_XZ>(cl, st, grid2);
      case EPI_RESID: return op_launch_typed<float, float, float, EPI_RESID>(cl, st, grid2);
    }
  }
  return record_error(HGL_ERR_INVALID_ARG, "unsupported operator variant (FP32 X)");
}

}  // namespace hgl
