// theta_bf16.cu -- operator passes with BF16 X panels (FP32 intermediate and accumulation).
#include "theta_launch.cuh"

namespace hgl {

hgl_status op_launch_bf16(const OpCall& cl, cudaStream_t st, int* grid2) {
  if (cl.zdt == HGL_BF16 && cl.epi == EPI_PLAIN)
    return op_launch_typed<bf16_t, float, bf16_t, EPI_PLAIN>(cl, st, grid2);
  if (cl.zdt == HGL_FP32 && cl.epi == EPI_DOT_XZ)
    return op_launch_typed<bf16_t, float, float, EPI_DOT_XZ>(cl, st, grid2);
  if (cl.zdt == HGL_FP32 && cl.epi == EPI_PLAIN)
    return op_launch_typed<bf16_t, float, float, EPI_PLAIN>(cl, st, grid2);
  return record_error(HGL_ERR_INVALID_ARG, "unsupported operator variant (BF16 X)");
}

}  // namespace hgl
