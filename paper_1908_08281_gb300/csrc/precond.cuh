// precond.cuh -- the block preconditioner handle (built in rsvd.cu, applied in precond.cu).
#pragma once

#include <cuda.h>

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
  // tensor-core apply (FP32 factors, k <= 64): the factors split into TF32 pairs
  // hi + lo, row-major (n x kp) and transposed (kp x n4), rank padded to kp = 32 or 64
  bool tc = false;                // built for it
  bool tc_on = true;              // selected (hgl_precond_tensor_cores)
  int kp = 0;
  int64_t n4 = 0;
  float *Qh = nullptr, *Ql = nullptr, *QTh = nullptr, *QTl = nullptr;
  float* gain32 = nullptr;       // the gains in FP32 (nb x k)
  int32_t* blk_order = nullptr;  // blocks by decreasing size
  int32_t* d_err = nullptr;      // set by a tensor-core kernel that gave up a wait
  CUtensorMap mQh, mQl, mQTh, mQTl;
};

namespace hgl {
constexpr int PC_SLAB = 2048;  // block rows reduced by one projection CTA
constexpr int PC_TILE = 128;   // rows (and columns) of one expansion CTA
hgl_status precond_gains_launch(hgl_precond* P, const double* ev_lpad, int lpad, cudaStream_t st);

// 2-D tensor map over a row-major matrix (inner = elements per row, outer = rows).
hgl_status encode_map_2d(CUtensorMap* map, CUtensorMapDataType dt, const void* base, uint64_t inner, uint64_t outer,
                         uint64_t row_bytes, uint32_t box_inner, uint32_t box_outer, CUtensorMapSwizzle sw);

// Tensor-core apply (precond_tc.cu): whether P takes it, the split of the factors
// after a build, the maps over them, and the apply itself.
bool precond_tc_usable(const hgl_precond* P, const void* R, int64_t ldr, const void* Z, int64_t ldz);
hgl_status precond_tc_prepare(hgl_precond* P, cudaStream_t st);
// HGL_ERR_TIMEOUT (and the flag cleared) if a tensor-core apply gave up a wait since the
// last check.  Synchronises the stream.
hgl_status precond_tc_status(hgl_precond* P, cudaStream_t st);
hgl_status precond_tc_maps(hgl_precond* P);
// Z = P R on FP32 panels; when rz != nullptr also per-block partial sums of R.Z
// (nb rows of c, the identity r.z = r.r/(1+lam) + sum_i g_i (q_i.r)^2 per block).
hgl_status precond_tc_apply(hgl_precond* P, const float* R, int64_t ldr, float* Z, int64_t ldz, int c,
                            double* rz, cudaStream_t st, const int32_t* run_flag);
}  // namespace hgl
