// selftest.cu -- hgl_selftest_wait_timeout: the bounded device wait of the tcgen05
// kernels, run against an mbarrier that nothing arrives on.
#include "hgl_internal.cuh"
#include "umma.cuh"

namespace hgl {
namespace {

// One warp: lane 0 initialises a barrier expecting one arrival that never comes and
// waits for its first phase with the given cycle limit; the wait gives up, records 1 in
// *err and returns false.  No memory operation is pending when the kernel ends.
__global__ void k_wait_selftest(unsigned long long limit_cycles, int* err) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    umma::mbar_init(&bar, 1);
    umma::fence_barrier_init();
    const bool done = umma::mbar_wait_limit(&bar, 0, err, limit_cycles);
    if (done) atomicExch(err, 2);  // impossible: nothing arrived
  }
  __syncwarp();
}

}  // namespace
}  // namespace hgl

extern "C" hgl_status hgl_selftest_wait_timeout(int64_t limit_cycles, void* stream) {
  if (limit_cycles < 1 || limit_cycles > (int64_t)8000000000ll)
    return hgl::record_error(HGL_ERR_INVALID_ARG, "limit_cycles must be in [1, 8e9]");
  cudaStream_t st = hgl::as_stream(stream);
  int* d_err = nullptr;
  HGL_CHECK_CUDA(cudaMalloc(&d_err, sizeof(int)));
  int h_err = 0;
  cudaError_t e = cudaMemsetAsync(d_err, 0, sizeof(int), st);
  if (e == cudaSuccess) {
    hgl::count_launch();
    hgl::k_wait_selftest<<<1, 32, 0, st>>>((unsigned long long)limit_cycles, d_err);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h_err, d_err, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(d_err);
  if (e != cudaSuccess) return hgl::cuda_error(e, "wait self-test", __FILE__, __LINE__);
  if (h_err == 1) return hgl::record_error(HGL_ERR_TIMEOUT, "the device wait gave up after %lld cycles (expected)",
                                           (long long)limit_cycles);
  return hgl::record_error(HGL_ERR_CUDA, "the device wait did not give up (status %d)", h_err);
}
