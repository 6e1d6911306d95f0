// precond.cuh -- the block preconditioner handle (built in rsvd.cu, applied in precond.cu).
#pragma once

#include <vector>

#include "hgl_internal.cuh"

struct hgl_precond {
  const hgl_graph* g = nullptr;
  int64_t n = 0;
  int nb = 0, k = 0, l = 0, lpad = 0;
  double lam = 0.0;
  int dtype = HGL_BF16;          // BF16: factors stored FP32; FP64: factors stored FP64
  std::vector<int64_t> bptr;     // host copy of the block boundaries
  std::vector<int32_t> kb;       // rank of each block (min(k, size))
  void* dev = nullptr;           // one allocation holding everything below
  void* Q = nullptr;             // n x k Ritz vectors, row v belongs to v's block
  double* gain = nullptr;        // nb x k
  double* ev = nullptr;          // nb x k eigenvalues (descending)
  int64_t* d_v0 = nullptr;       // nb + 1 block boundaries
  int32_t* d_rows = nullptr;     // nb
  int32_t* d_kb = nullptr;       // nb
  int32_t* unit_block = nullptr; // 64-row units used by the apply
  int32_t* unit_tile = nullptr;
  int nunits = 0;
  hgl::Buffer cbuf;              // apply scratch: diag(g) Q^T R, nb x k x c
};

namespace hgl {
hgl_status precond_gains_launch(hgl_precond* P, const double* ev_lpad, int lpad, cudaStream_t st);
}  // namespace hgl
