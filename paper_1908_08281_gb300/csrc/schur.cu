// schur.cu -- hgl_schur_inverse: the nested 2 x 2 Schur-complement inverse of Section 3
// (Eqs. 12-14) with randomized-SVD inverses of the diagonal blocks and of the Schur
// complements, and nested tessellation of the diagonal blocks.
//
// For M = (1+lam) I - Theta on a contiguous vertex range, split in halves 1 | 2:
//   M^-1 = [[ Z1^-1,                 -M11^-1 M12 Z2^-1 ],
//           [ -Z2^-1 M21 M11^-1,      Z2^-1            ]]
//   Z1 = M11 - M12 M22^-1 M21 = (1+lam) I - (Theta11 + Theta12 M22^-1 Theta21),
//   Z2 = (1+lam) I - (Theta22 + Theta21 M11^-1 Theta12)          (M12 = -Theta12).
// Every inverted matrix has the form (1+lam) I - L with L symmetric positive
// semidefinite, and "inverted by randomized SVD" means exact on the subspace that
// Algorithm 1 (Rayleigh-Ritz form) captures for L and 1/(1+lam) on its complement:
//   ((1+lam) I - L)^-1 ~= I/(1+lam) + Q diag(l / ((1+lam)(1+lam-l))) Q^T.
// M11^-1 and M22^-1 come from the same scheme applied to the halves (nested
// tessellation) down to blocks of at most 2 r_min rows, which Algorithm 1 inverts
// directly.  The test matrix of a submatrix is the block preconditioner's Philox
// stream on the submatrix's global rows.
//
// The dense products (eight per split, each about 2 h^3 flops) run on the tcgen05
// tensor cores (HGL_FP32: kind::tf32 with every operand split into a TF32 pair and
// three products per pair, FP32 accumulation in TMEM, about 2^-21 relative per
// product) or on FP64 CUDA cores (HGL_FP64, for checking).  Algorithm 1 itself runs in
// FP64 either way (its products are nb x nb x (k + p), a small part of the work).
#include <algorithm>
#include <cstring>

#include "hgl_internal.cuh"
#include "rsvd_kernels.cuh"
#include "solver.cuh"
#include "umma.cuh"

namespace hgl {

hgl_status encode_map_2d(CUtensorMap* map, CUtensorMapDataType dt, const void* base, uint64_t inner, uint64_t outer,
                         uint64_t row_bytes, uint32_t box_inner, uint32_t box_outer, CUtensorMapSwizzle sw);

namespace {

// ---------------------------------------------------------------------------
// FP64 GEMM on CUDA cores: C = A op(B) (+ C0), row-major, op(B) = B (K x N) or, with
// transB, the transpose of B (N x K).  64 x 64 output tile per block, 4 x 4 per thread.
// ---------------------------------------------------------------------------
constexpr int DG_T = 64, DG_K = 16;

__global__ void __launch_bounds__(256)
k_dgemm(int64_t M, int64_t N, int64_t K, const double* __restrict__ A, int64_t lda, const double* __restrict__ B,
        int64_t ldb, int transB, const double* __restrict__ C0, int64_t ldc0, double* __restrict__ C, int64_t ldc) {
  __shared__ double sa[DG_K][DG_T + 1];
  __shared__ double sb[DG_K][DG_T + 1];
  const int64_t bm = (int64_t)blockIdx.y * DG_T, bn = (int64_t)blockIdx.x * DG_T;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  double acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
  for (int64_t k0 = 0; k0 < K; k0 += DG_K) {
    for (int q = threadIdx.x; q < DG_T * DG_K; q += blockDim.x) {
      const int m = q / DG_K, kk = q % DG_K;
      sa[kk][m] = (bm + m < M && k0 + kk < K) ? A[(bm + m) * lda + k0 + kk] : 0.0;
      if (transB) {
        sb[kk][m] = (bn + m < N && k0 + kk < K) ? B[(bn + m) * ldb + k0 + kk] : 0.0;
      } else {
        const int kr = q / DG_T, nn = q % DG_T;
        sb[kr][nn] = (bn + nn < N && k0 + kr < K) ? B[(k0 + kr) * ldb + bn + nn] : 0.0;
      }
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < DG_K; ++kk) {
      double av[4], bv[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) av[i] = sa[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) bv[j] = sb[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(av[i], bv[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int64_t r = bm + ty + 16 * i;
    if (r >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int64_t cc = bn + tx + 16 * j;
      if (cc < N) C[r * ldc + cc] = acc[i][j] + (C0 ? C0[r * ldc0 + cc] : 0.0);
    }
  }
}

// Qg[i, t] = Q[i, t] g_t with g = l / ((1+lam)(1+lam-l)) for the clipped Ritz values
// l = max(ev, 0) (the gains of the low-rank inverse).
__global__ void k_gain_cols(int64_t nb, int kb, const double* __restrict__ Q, const double* __restrict__ ev,
                            double lam, double* __restrict__ Qg) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nb * kb; q += (int64_t)gridDim.x * blockDim.x) {
    const int t = (int)(q % kb);
    const double l = fmax(ev[t], 0.0);
    Qg[q] = Q[q] * (l / ((1.0 + lam) * (1.0 + lam - l)));
  }
}

// out[i, i] += 1 / (1 + lam)
__global__ void k_add_diag(int64_t nb, double v, double* __restrict__ out, int64_t ldo) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nb; i += (int64_t)gridDim.x * blockDim.x)
    out[i * ldo + i] += v;
}

// A dense FP64 matrix (rows x cols, row-major) as a TF32 pair hi + lo in FP32 storage
// (hi = x rounded to TF32, lo = the remainder rounded to TF32), rows x ldk with zero
// padding up to ldk columns; with trans, the pair of the transpose (cols x ldk).
__global__ void k_split_pair(int64_t rows, int64_t cols, const double* __restrict__ X, int64_t ldx, int trans,
                             int64_t ldk, float* __restrict__ hi, float* __restrict__ lo) {
  const int64_t orows = trans ? cols : rows, icols = trans ? rows : cols;
  const int64_t total = orows * ldk;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = q / ldk, k = q % ldk;
    double x = 0.0;
    if (k < icols) x = trans ? X[k * ldx + r] : X[r * ldx + k];
    const float xf = (float)x;
    const float h = umma::tf32_round(xf);
    const float l = umma::tf32_round((float)(x - (double)h));
    hi[q] = h;
    lo[q] = l;
  }
}

}  // namespace
}  // namespace hgl

namespace hgl {
namespace {

// ---------------------------------------------------------------------------
// C = A B^T (+ C0) on tcgen05 (kind::tf32), A (M x Kp) and B (N x Kp) K-major FP32
// TF32 pairs: acc = Ah Bh + Ah Bl + Al Bh accumulated in FP32 in TMEM (the lo*lo term,
// ~2^-22 relative, is dropped).  Work unit = one 128 x 128 output tile; persistent
// CTAs stride over the units.  Warp 0: TMA producer (four 128 x 32 FP32 tiles per
// stage, 128-byte swizzle); warp 1: one elected lane issues the MMAs into a
// double-buffered 128 x 128 FP32 accumulator; warp 2: TMEM allocation; warps 4-7:
// epilogue (TMEM -> registers -> C in FP64, + C0).  Every wait is bounded (about 2 s)
// and records HGL_ERR_TIMEOUT's code in *err instead of hanging.
// ---------------------------------------------------------------------------
constexpr int TG_BM = 128, TG_BN = 128, TG_BK = 32, TG_STAGES = 3;
constexpr uint32_t TG_TILE = TG_BM * TG_BK * 4;   // 16 KB
constexpr uint32_t TG_STAGE = 4 * TG_TILE;        // Ah, Al, Bh, Bl
constexpr uint32_t TG_ACC_COLS = 128;
constexpr size_t TG_SMEM = 1024 + (size_t)TG_STAGES * TG_STAGE + 256;

struct TgArgs {
  int64_t M, N;
  int ktiles, tiles_n, nunits;
  const double* C0;
  int64_t ldc0;
  double* C;
  int64_t ldc;
  int* err;
};

__global__ void __launch_bounds__(256, 1)
k_gemm_tf32x3(const __grid_constant__ CUtensorMap mAh, const __grid_constant__ CUtensorMap mAl,
              const __grid_constant__ CUtensorMap mBh, const __grid_constant__ CUtensorMap mBl, TgArgs a) {
  using namespace umma;
  constexpr uint32_t IDESC = idesc_tf32_f32(TG_BM, TG_BN);
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + TG_STAGES * TG_STAGE);
  uint64_t* empty = full + TG_STAGES;
  uint64_t* acc_full = empty + TG_STAGES;  // 2
  uint64_t* acc_empty = acc_full + 2;      // 2
  uint64_t* mma_drain = acc_empty + 2;     // 1
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(mma_drain + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < TG_STAGES; ++s) {
      mbar_init(full + s, 1);
      mbar_init(empty + s, 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(acc_full + b, 1);
      mbar_init(acc_empty + b, 4);
    }
    mbar_init(mma_drain, 1);
    fence_barrier_init();
  }
  if (warp == 2) tmem_alloc(tmem_slot, 2 * TG_ACC_COLS);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      bool ok = true;
      ArmedPhases<TG_STAGES> armed;
      for (int u = blockIdx.x; u < a.nunits && ok; u += gridDim.x) {
        const int tm = u / a.tiles_n, tn = u % a.tiles_n;
        for (int kt = 0; kt < a.ktiles; ++kt) {
          if (!mbar_wait(empty + stage, phase ^ 1, a.err)) {
            ok = false;
            break;
          }
          uint8_t* s0 = smem + stage * TG_STAGE;
          mbar_arrive_expect_tx(full + stage, TG_STAGE);
          tma_load_2d(s0, &mAh, full + stage, kt * TG_BK, tm * TG_BM);
          tma_load_2d(s0 + TG_TILE, &mAl, full + stage, kt * TG_BK, tm * TG_BM);
          tma_load_2d(s0 + 2 * TG_TILE, &mBh, full + stage, kt * TG_BK, tn * TG_BN);
          tma_load_2d(s0 + 3 * TG_TILE, &mBl, full + stage, kt * TG_BK, tn * TG_BN);
          armed.p[stage] = (uint8_t)phase;
          if (++stage == TG_STAGES) {
            stage = 0;
            phase ^= 1;
          }
        }
      }
      if (*(volatile int*)a.err != 0) armed.drain(full);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      int stage = 0, acc = 0;
      uint32_t phase = 0, acc_phase = 0;
      bool ok = true;
      for (int u = blockIdx.x; u < a.nunits && ok; u += gridDim.x) {
        if (!mbar_wait(acc_empty + acc, acc_phase ^ 1, a.err)) break;
        tc_fence_after();
        const uint32_t d_tmem = tmem_base + (uint32_t)acc * TG_ACC_COLS;
        for (int kt = 0; kt < a.ktiles; ++kt) {
          if (!mbar_wait(full + stage, phase, a.err)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t s0 = smem_u32(smem + stage * TG_STAGE);
          const uint64_t ah = smem_desc_sw128(s0), al = smem_desc_sw128(s0 + TG_TILE);
          const uint64_t bh = smem_desc_sw128(s0 + 2 * TG_TILE), bl = smem_desc_sw128(s0 + 3 * TG_TILE);
#pragma unroll
          for (int kk = 0; kk < TG_BK / 8; ++kk) {
            // 8 TF32 elements (32 bytes) along K per MMA inside the 128-byte swizzled row
            const uint64_t off = (uint64_t)((kk * 32) >> 4);
            mma_tf32(d_tmem, ah + off, bh + off, IDESC, (kt > 0 || kk > 0) ? 1u : 0u);
            mma_tf32(d_tmem, ah + off, bl + off, IDESC, 1u);
            mma_tf32(d_tmem, al + off, bh + off, IDESC, 1u);
          }
          mma_commit(empty + stage);
          if (++stage == TG_STAGES) {
            stage = 0;
            phase ^= 1;
          }
        }
        if (!ok) break;
        mma_commit(acc_full + acc);
        if (++acc == 2) {
          acc = 0;
          acc_phase ^= 1;
        }
      }
      if (*(volatile int*)a.err != 0) {
        mma_commit(mma_drain);
        mbar_drain(mma_drain, 0);
      }
    }
  } else if (warp >= 4) {
    const int quarter = warp & 3;
    int acc = 0;
    uint32_t acc_phase = 0;
    for (int u = blockIdx.x; u < a.nunits; u += gridDim.x) {
      const int tm = u / a.tiles_n, tn = u % a.tiles_n;
      if (!mbar_wait(acc_full + acc, acc_phase, a.err)) break;
      tc_fence_after();
      const int64_t row = (int64_t)tm * TG_BM + quarter * 32 + lane;
      const uint32_t taddr = tmem_base + (uint32_t)acc * TG_ACC_COLS + ((uint32_t)(quarter * 32) << 16);
#pragma unroll 1
      for (int cb = 0; cb < TG_BN / 16; ++cb) {
        uint32_t r[16];
        tmem_ld16(taddr + cb * 16, r);
        tmem_ld_wait();
        if (row < a.M) {
          const int64_t c0 = (int64_t)tn * TG_BN + cb * 16;
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const int64_t col = c0 + j;
            if (col < a.N)
              a.C[row * a.ldc + col] = (double)__uint_as_float(r[j]) + (a.C0 ? a.C0[row * a.ldc0 + col] : 0.0);
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(acc_empty + acc);
      if (++acc == 2) {
        acc = 0;
        acc_phase ^= 1;
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 2) {
    tc_fence_after();
    tmem_dealloc(tmem_base, 2 * TG_ACC_COLS);
  }
}

}  // namespace
}  // namespace hgl

namespace hgl {
namespace {


inline int64_t rup64(int64_t x, int64_t a) { return (x + a - 1) / a * a; }
inline size_t dbytes(int64_t count) { return (size_t)rup64(count * (int64_t)sizeof(double), 256); }

struct SchurCtx {
  int dtype = HGL_FP64;
  double lam = 0.0;
  int r_min = 0, k = 0, p = 0, q = 0;
  uint64_t seed = 0;
  int sms = 0;
  cudaStream_t st = nullptr;
  Buffer split;   // Ah, Al, Bh, Bl (FP32) of the tensor-core products
  Buffer rsvd;    // Algorithm 1's work space
  int* err = nullptr;
};

// C (M x N) = A (M x K) op(B) (+ C0): tcgen05 3xTF32 for HGL_FP32 when every side is at
// least 128, else FP64 CUDA cores.
hgl_status dense_gemm(SchurCtx& cx, int64_t M, int64_t N, int64_t K, const double* A, int64_t lda, const double* B,
                      int64_t ldb, bool transB, const double* C0, int64_t ldc0, double* C, int64_t ldc) {
  if (cx.dtype == HGL_FP32 && M >= 128 && N >= 128 && K >= 128) {
    const int64_t Kp = rup64(K, TG_BK);
    const size_t an = (size_t)M * Kp, bn = (size_t)N * Kp;
    hgl_status s_ = HGL_OK;
    float* base = static_cast<float*>(buffer_get(cx.split, sizeof(float) * 2 * (an + bn) + 1024, &s_));
    if (!base) return s_;
    float *Ah = base, *Al = Ah + an, *Bh = Al + an, *Bl = Bh + bn;
    count_launch(2);
    k_split_pair<<<cx.sms * 8, 256, 0, cx.st>>>(M, K, A, lda, 0, Kp, Ah, Al);
    // B^T as K-major rows: B is K x N (transpose it) or already N x K
    if (transB)
      k_split_pair<<<cx.sms * 8, 256, 0, cx.st>>>(N, K, B, ldb, 0, Kp, Bh, Bl);
    else
      k_split_pair<<<cx.sms * 8, 256, 0, cx.st>>>(K, N, B, ldb, 1, Kp, Bh, Bl);
    HGL_CHECK_CUDA(cudaGetLastError());
    CUtensorMap mAh, mAl, mBh, mBl;
    const auto f32 = CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    const auto sw = CU_TENSOR_MAP_SWIZZLE_128B;
    HGL_TRY(encode_map_2d(&mAh, f32, Ah, (uint64_t)Kp, (uint64_t)M, (uint64_t)Kp * 4, TG_BK, TG_BM, sw));
    HGL_TRY(encode_map_2d(&mAl, f32, Al, (uint64_t)Kp, (uint64_t)M, (uint64_t)Kp * 4, TG_BK, TG_BM, sw));
    HGL_TRY(encode_map_2d(&mBh, f32, Bh, (uint64_t)Kp, (uint64_t)N, (uint64_t)Kp * 4, TG_BK, TG_BN, sw));
    HGL_TRY(encode_map_2d(&mBl, f32, Bl, (uint64_t)Kp, (uint64_t)N, (uint64_t)Kp * 4, TG_BK, TG_BN, sw));
    TgArgs a{};
    a.M = M;
    a.N = N;
    a.ktiles = (int)(Kp / TG_BK);
    a.tiles_n = (int)((N + TG_BN - 1) / TG_BN);
    a.nunits = (int)((M + TG_BM - 1) / TG_BM) * a.tiles_n;
    a.C0 = C0;
    a.ldc0 = ldc0;
    a.C = C;
    a.ldc = ldc;
    a.err = cx.err;
    HGL_CHECK_CUDA(cudaFuncSetAttribute(reinterpret_cast<const void*>(k_gemm_tf32x3),
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TG_SMEM));
    {
      ProfScope prof(HGL_PROF_SCHUR_GEMM, cx.st);
      count_launch();
      k_gemm_tf32x3<<<std::min(a.nunits, cx.sms), 256, TG_SMEM, cx.st>>>(mAh, mAl, mBh, mBl, a);
    }
    HGL_CHECK_CUDA(cudaGetLastError());
    return HGL_OK;
  }
  dim3 grid((unsigned)((N + DG_T - 1) / DG_T), (unsigned)((M + DG_T - 1) / DG_T));
  {
    ProfScope prof(HGL_PROF_SCHUR_GEMM, cx.st);
    count_launch();
    k_dgemm<<<grid, 256, 0, cx.st>>>(M, N, K, A, lda, B, ldb, transB ? 1 : 0, C0, ldc0, C, ldc);
  }
  HGL_CHECK_CUDA(cudaGetLastError());
  return HGL_OK;
}

// One node of the nested tessellation: rows [off, off + n) of the range (offsets into the
// dense Theta), its inverse in `out` (ld ldo), its halves' nodes (internal nodes).
struct Node {
  int64_t off = 0, n = 0;
  int level = 0;
  int child[2] = {-1, -1};
  double* out = nullptr;
  int64_t ldo = 0;
};

int build_tree(std::vector<Node>& nodes, int64_t off, int64_t n, int level, int r_min) {
  const int id = (int)nodes.size();
  nodes.push_back(Node{});
  nodes[id].off = off;
  nodes[id].n = n;
  nodes[id].level = level;
  if (n > 2 * (int64_t)r_min) {
    const int64_t h = n / 2;
    const int c0 = build_tree(nodes, off, h, level + 1, r_min);
    const int c1 = build_tree(nodes, off + h, n - h, level + 1, r_min);
    nodes[id].child[0] = c0;
    nodes[id].child[1] = c1;
  }
  return id;
}

// One item of a level's batched Algorithm 1: the matrix L (a leaf's diagonal block of
// Theta, or a Schur complement's L), its global first row, and where its low-rank
// inverse ((1+lam) I - L)^-1 goes.
struct Item {
  const double* L;
  int64_t ldl, v0, n;
  double* out;
  int64_t ldo;
};

// The level's inverses: Algorithm 1 on all items in one batch, then per item
// out = I/(1+lam) + (Q diag(g)) Q^T with g = l/((1+lam)(1+lam-l)), l = max(Ritz value, 0).
hgl_status lowrank_inverses(SchurCtx& cx, const std::vector<Item>& items, int64_t row0, double* Q, double* Qg,
                            double* ev) {
  const int nb = (int)items.size();
  std::vector<const double*> Ls(nb);
  std::vector<int64_t> ld(nb), v0(nb), sz(nb);
  for (int b = 0; b < nb; ++b) {
    Ls[b] = items[b].L;
    ld[b] = items[b].ldl;
    v0[b] = items[b].v0;
    sz[b] = items[b].n;
  }
  HGL_TRY(dense_rsvd_batch_fp64(nb, Ls.data(), ld.data(), v0.data(), sz.data(), cx.k, cx.p, cx.q, cx.seed, cx.rsvd,
                                Q, row0, ev, cx.st));
  for (int b = 0; b < nb; ++b) {
    const Item& it = items[b];
    // Q's columns past min(k, n) are zero, so all k columns can take part
    double* Qb = Q + (it.v0 - row0) * cx.k;
    double* Qgb = Qg + (it.v0 - row0) * cx.k;
    count_launch(3);
    k_gain_cols<<<cx.sms * 4, 256, 0, cx.st>>>(it.n, cx.k, Qb, ev + (size_t)b * cx.k, cx.lam, Qgb);
    // the low-rank outer product on CUDA cores in FP64 (n x n x k)
    dim3 grid((unsigned)((it.n + DG_T - 1) / DG_T), (unsigned)((it.n + DG_T - 1) / DG_T));
    k_dgemm<<<grid, 256, 0, cx.st>>>(it.n, it.n, cx.k, Qgb, cx.k, Qb, cx.k, 1, nullptr, 0, it.out, it.ldo);
    k_add_diag<<<(int)std::max<int64_t>(1, std::min<int64_t>((it.n + 255) / 256, cx.sms * 4)), 256, 0, cx.st>>>(
        it.n, 1.0 / (1.0 + cx.lam), it.out, it.ldo);
    HGL_CHECK_CUDA(cudaGetLastError());
  }
  return HGL_OK;
}

}  // namespace
}  // namespace hgl

extern "C" hgl_status hgl_schur_inverse(const hgl_graph* gc, const double* w, double lam, int64_t row0,
                                        int64_t nrows, int32_t r_min, int32_t k, int32_t p, int32_t q,
                                        uint64_t seed, hgl_dtype dtype, double* Minv, int64_t ldm, void* stream) {
  using namespace hgl;
  hgl_graph* g = const_cast<hgl_graph*>(gc);
  if (!g || !w || !Minv) return record_error(HGL_ERR_INVALID_ARG, "NULL argument");
  if (!(lam > 0.0)) return record_error(HGL_ERR_INVALID_ARG, "lam must be positive");
  if (row0 < 0 || nrows < 1 || row0 + nrows > g->n) return record_error(HGL_ERR_INVALID_ARG, "row range out of [0, n)");
  if (r_min < 1) return record_error(HGL_ERR_INVALID_ARG, "r_min must be >= 1");
  if (k < 1 || p < 0 || q < 0 || k + p > 96) return record_error(HGL_ERR_INVALID_ARG, "need k >= 1, p, q >= 0, k + p <= 96");
  if (dtype != HGL_FP64 && dtype != HGL_FP32) return record_error(HGL_ERR_INVALID_ARG, "dtype must be FP64 or FP32");
  if (ldm < nrows) return record_error(HGL_ERR_INVALID_ARG, "ldm must be >= nrows");
  if (nrows > 65536) return record_error(HGL_ERR_INVALID_ARG, "nrows must be <= 65536 (dense n x n work)");
  cudaStream_t st = as_stream(stream);
  HGL_TRY(degrees_launch(g, w, st));
  SchurCtx cx;
  cx.dtype = dtype;
  cx.lam = lam;
  cx.r_min = r_min;
  cx.k = k;
  cx.p = p;
  cx.q = q;
  cx.seed = seed;
  cx.sms = g->num_sms;
  cx.st = st;

  // the nested tessellation, its levels, and one arena: the dense Theta of the range,
  // every non-root node's inverse, one level's Schur-complement matrices, a product
  // temporary, and the Ritz vectors
  std::vector<Node> nodes;
  build_tree(nodes, 0, nrows, 0, r_min);
  int depth = 0;
  for (const Node& nd : nodes) depth = std::max(depth, nd.level);
  const int64_t ldt = rup64(nrows, 64), trows = rup64(nrows, 128);
  size_t bytes = dbytes(trows * ldt);
  for (size_t i = 1; i < nodes.size(); ++i) bytes += dbytes(nodes[i].n * nodes[i].n);
  std::vector<size_t> lvl_L(depth + 1, 0);
  int64_t maxX = 0;
  for (const Node& nd : nodes)
    if (nd.child[0] >= 0) {
      const int64_t h = nd.n / 2, h2 = nd.n - h;
      lvl_L[nd.level] += dbytes(h * h) + dbytes(h2 * h2);
      maxX = std::max(maxX, h * h2);
    }
  bytes += *std::max_element(lvl_L.begin(), lvl_L.end()) + dbytes(maxX) + 2 * dbytes(nrows * (int64_t)k) +
           dbytes((int64_t)nodes.size() * 2 * k) + 1024;
  char* arena = nullptr;
  HGL_CHECK_CUDA(cudaMalloc(reinterpret_cast<void**>(&arena), bytes));
  size_t top = 0;
  auto take = [&](int64_t count) {
    double* ptr = reinterpret_cast<double*>(arena + top);
    top += dbytes(count);
    return ptr;
  };
  double* T = take(trows * ldt);
  nodes[0].out = Minv;
  nodes[0].ldo = ldm;
  for (size_t i = 1; i < nodes.size(); ++i) {
    nodes[i].out = take(nodes[i].n * nodes[i].n);
    nodes[i].ldo = nodes[i].n;
  }
  const size_t lbase = top;
  top += *std::max_element(lvl_L.begin(), lvl_L.end());
  double* X = take(maxX);
  double* Q = take(nrows * (int64_t)k);
  double* Qg = take(nrows * (int64_t)k);
  double* ev = take((int64_t)nodes.size() * 2 * k);

  hgl_status s_ = HGL_OK;
  void* meta = nullptr;
  cudaError_t ce = cudaMalloc(reinterpret_cast<void**>(&cx.err), sizeof(int));
  if (ce == cudaSuccess) ce = cudaMemsetAsync(cx.err, 0, sizeof(int), st);
  if (ce == cudaSuccess) ce = cudaMalloc(&meta, 64);
  if (ce == cudaSuccess) {
    // the dense Theta of the range: the rSVD's block assembly with one block [row0, row0 + nrows)
    char hbuf[48] = {};
    const int64_t hm[3] = {row0, 0, 0};
    const int32_t im[3] = {(int32_t)nrows, 1, 1};
    memcpy(hbuf, hm, 24);
    memcpy(hbuf + 24, im, 12);
    ce = cudaMemcpyAsync(meta, hbuf, 36, cudaMemcpyHostToDevice, st);
    rsvd::Blocks B{};
    B.nb = 1;
    B.l = 1;
    B.lpad = 16;
    B.k = 1;
    B.ldA = ldt;
    B.Ktot = ldt;
    B.v0 = static_cast<const int64_t*>(meta);
    B.arow = B.v0 + 1;
    B.koff = B.v0 + 2;
    B.rows = reinterpret_cast<const int32_t*>(static_cast<char*>(meta) + 24);
    B.lb = B.rows + 1;
    B.kb = B.rows + 2;
    if (ce == cudaSuccess) {
      count_launch();
      rsvd::k_assemble<double, double><<<cx.sms * 8, 256, 0, st>>>(B, trows, g->csr_ptr, g->csr_idx, g->csc_ptr,
                                                                   g->csc_idx, g->s, g->t, T);
      ce = cudaGetLastError();
    }
  }
  if (ce != cudaSuccess) s_ = cuda_error(ce, "Schur inverse setup", __FILE__, __LINE__);

  // bottom-up: per level, the Schur complements of its internal nodes (from the next
  // level's inverses), one batch of Algorithm 1 for those and for the level's leaf
  // blocks, then the internal nodes' off-diagonal blocks
  for (int lv = depth; lv >= 0 && s_ == HGL_OK; --lv) {
    std::vector<Item> items;
    size_t ltop = lbase;
    for (const Node& nd : nodes) {
      if (nd.level != lv || s_ != HGL_OK) continue;
      const double* T11 = T + nd.off * ldt + nd.off;
      if (nd.child[0] < 0) {
        items.push_back(Item{T11, ldt, row0 + nd.off, nd.n, nd.out, nd.ldo});
        continue;
      }
      const int64_t h = nd.n / 2, h2 = nd.n - h;
      const double* T12 = T11 + h;
      const double* T21 = T11 + h * ldt;
      const double* T22 = T21 + h;
      const Node& c1 = nodes[nd.child[0]];
      const Node& c2 = nodes[nd.child[1]];
      double* L1 = reinterpret_cast<double*>(arena + ltop);
      ltop += dbytes(h * h);
      double* L2 = reinterpret_cast<double*>(arena + ltop);
      ltop += dbytes(h2 * h2);
      // L1 = T11 + (T12 M22^-1) T21,  L2 = T22 + (T21 M11^-1) T12
      s_ = dense_gemm(cx, h, h2, h2, T12, ldt, c2.out, c2.ldo, false, nullptr, 0, X, h2);
      if (s_ == HGL_OK) s_ = dense_gemm(cx, h, h, h2, X, h2, T21, ldt, false, T11, ldt, L1, h);
      if (s_ == HGL_OK) s_ = dense_gemm(cx, h2, h, h, T21, ldt, c1.out, c1.ldo, false, nullptr, 0, X, h);
      if (s_ == HGL_OK) s_ = dense_gemm(cx, h2, h2, h, X, h, T12, ldt, false, T22, ldt, L2, h2);
      items.push_back(Item{L1, h, row0 + nd.off, h, nd.out, nd.ldo});
      items.push_back(Item{L2, h2, row0 + nd.off + h, h2, nd.out + h * nd.ldo + h, nd.ldo});
    }
    if (s_ == HGL_OK && !items.empty()) s_ = lowrank_inverses(cx, items, row0, Q, Qg, ev);
    for (const Node& nd : nodes) {
      if (nd.level != lv || nd.child[0] < 0 || s_ != HGL_OK) continue;
      const int64_t h = nd.n / 2, h2 = nd.n - h;
      const double* T12 = T + nd.off * ldt + nd.off + h;
      const double* T21 = T + (nd.off + h) * ldt + nd.off;
      const Node& c1 = nodes[nd.child[0]];
      double* O12 = nd.out + h;
      double* O21 = nd.out + h * nd.ldo;
      const double* O22 = nd.out + h * nd.ldo + h;
      // -M11^-1 M12 Z2^-1 = (M11^-1 T12) Z2^-1,  -Z2^-1 M21 M11^-1 = (Z2^-1 T21) M11^-1
      s_ = dense_gemm(cx, h, h2, h, c1.out, c1.ldo, T12, ldt, false, nullptr, 0, X, h2);
      if (s_ == HGL_OK) s_ = dense_gemm(cx, h, h2, h2, X, h2, O22, nd.ldo, false, nullptr, 0, O12, nd.ldo);
      if (s_ == HGL_OK) s_ = dense_gemm(cx, h2, h, h2, O22, nd.ldo, T21, ldt, false, nullptr, 0, X, h);
      if (s_ == HGL_OK) s_ = dense_gemm(cx, h2, h, h, X, h, c1.out, c1.ldo, false, nullptr, 0, O21, nd.ldo);
    }
  }
  if (s_ == HGL_OK) {
    ce = cudaStreamSynchronize(st);
    int e = 0;
    if (ce == cudaSuccess) ce = cudaMemcpy(&e, cx.err, sizeof(int), cudaMemcpyDeviceToHost);
    if (ce != cudaSuccess) s_ = cuda_error(ce, "Schur inverse", __FILE__, __LINE__);
    else if (e != 0) s_ = record_error(HGL_ERR_TIMEOUT, "the tensor-core GEMM hit its wait limit");
  }
  cudaStreamSynchronize(st);
  if (meta) cudaFree(meta);
  if (cx.err) cudaFree(cx.err);
  cudaFree(arena);
  buffer_free(cx.split);
  buffer_free(cx.rsvd);
  return s_;
}
