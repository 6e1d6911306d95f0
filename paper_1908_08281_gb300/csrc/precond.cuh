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
  // FP32 apply: projection slabs (block, first row) of up to PC_SLAB rows, the first
  // slab of every block (nb + 1 entries), and 128-row expansion tiles (block, tile)
  int32_t* slab_block = nullptr;
  int32_t* slab_row0 = nullptr;
  int32_t* blk_slab0 = nullptr;
  int nslabs = 0;
  int32_t* exp_block = nullptr;
  int32_t* exp_tile = nullptr;
  int nexp = 0;
  hgl::Buffer cbuf;              // apply scratch: diag(g) Q^T R, nb x k x c
  hgl::Buffer pbuf;              // FP32 apply scratch: per-slab partial projections
};

namespace hgl {
constexpr int PC_SLAB = 2048;  // block rows reduced by one projection CTA
constexpr int PC_TILE = 128;   // rows (and columns) of one expansion CTA
hgl_status precond_gains_launch(hgl_precond* P, const double* ev_lpad, int lpad, cudaStream_t st);
}  // namespace hgl
