// precond_tc.cu -- the block preconditioner apply (Section 3, Eq. 15) on tcgen05 tensor
// cores, for FP32 panels and FP32 factors of rank k <= 64:
//   C_b = diag(g_b) Q_b^T R_b          projection: contraction over the block's rows
//   Z_b = R_b / (1+lam) + Q_b C_b      expansion: contraction over the rank
// Both are dense products, so they run as kind::tf32 MMAs with FP32 accumulation in
// TMEM.  FP32 accuracy comes from splitting every operand x = hi + lo into two TF32
// numbers (hi = x rounded to TF32, lo = x - hi rounded to TF32) and summing the three
// products hi*hi + hi*lo + lo*hi: the dropped lo*lo term and the rounding of lo are
// ~2^-22 of x (the 3xTF32 scheme; Ootomo and Yokota, "Recovering single precision
// accuracy from Tensor Cores while surpassing the FP32 theoretical peak
// performance", 2022).  The factors are split once per build; R is split in the
// projection kernel while it is transposed into the MMA's K-major operand layout, and C
// is split by the projection's epilogue.
//
// The projection also returns, per block and column, r.z = r.r/(1+lam) + sum_i g_i
// (q_i.r)^2 (z = P r restricted to the block), so the PCG needs no separate pass over
// R and Z for its r.z dot product.
#include <algorithm>

#include "panel.cuh"
#include "precond.cuh"
#include "umma.cuh"

namespace hgl {
namespace {

using umma::mbar_arrive;
using umma::mbar_arrive_expect_tx;
using umma::mbar_init;
using umma::mbar_wait;
using umma::smem_desc_sw128;
using umma::smem_u32;
using umma::sw128_offset_f32;
using umma::tc_fence_after;
using umma::tc_fence_before;
using umma::tf32_round;
using umma::tma_load_2d;

constexpr int TC_THREADS = 256;
constexpr int PJ_ROWS = 32;   // block rows per projection step (one 128-byte TF32 K slice)
constexpr int PJ_COLS = 128;  // panel columns per projection unit (the MMA's M)
constexpr int EX_ROWS = 128;  // rows per expansion unit (the MMA's M)
constexpr int EX_COLS = 64;   // panel columns per expansion step (the MMA's N)

inline int64_t rup(int64_t x, int64_t a) { return (x + a - 1) / a * a; }

// Split of the factors: Q (n x k, row-major) -> Qh, Ql (n x KP) and QTh, QTl (KP x n4),
// zero beyond rank k and beyond row n.  One 32-row tile per iteration, transposed
// through shared memory so that both outputs are written along their rows.
template <int KP>
__global__ void __launch_bounds__(256)
k_tc_split(int64_t n, int64_t n4, int k, const float* __restrict__ Q, float* __restrict__ Qh,
           float* __restrict__ Ql, float* __restrict__ QTh, float* __restrict__ QTl) {
  __shared__ float th[KP][33], tl[KP][33];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  for (int64_t v0 = (int64_t)blockIdx.x * 32; v0 < n4; v0 += (int64_t)gridDim.x * 32) {
    for (int i = ty; i < 32; i += 8) {
      const int64_t v = v0 + i;
      for (int r = tx; r < KP; r += 32) {
        const float x = (v < n && r < k) ? Q[v * k + r] : 0.f;
        const float h = tf32_round(x);
        const float l = tf32_round(x - h);
        if (v < n) {
          Qh[v * KP + r] = h;
          Ql[v * KP + r] = l;
        }
        th[r][i] = h;
        tl[r][i] = l;
      }
    }
    __syncthreads();
    for (int r = ty; r < KP; r += 8) {
      const int64_t v = v0 + tx;
      if (v < n4) {
        QTh[(int64_t)r * n4 + v] = th[r][tx];
        QTl[(int64_t)r * n4 + v] = tl[r][tx];
      }
    }
    __syncthreads();
  }
}


// ---------------------------------------------------------------------------
// Projection.  Work unit = (block b, 128-column tile); units run in decreasing block
// size over persistent CTAs.  Per step of 32 block rows:
//   warp 0 (one lane): TMA of the R rows (32 x 128 FP32, unswizzled) into a ring of R
//          stages;
//   warp 3 (one lane): TMA of Q_b^T hi/lo (KP x 32, K-major, 128-byte swizzle) into a
//          ring of B stages (both rings deep enough to cover the DRAM latency: every
//          step waits on both streams);
//   warps 4-7 (thread t = panel column j): read column j of the staged rows, zero the
//          rows outside the block, accumulate r.r, split into TF32 hi + lo and write
//          them transposed (row t of a K-major 128 x 32 tile, 128-byte swizzle) into
//          a ring of two A stages (lo is left for the MMA to truncate to TF32: its
//          error, 2^-10 of lo, is 2^-21 of the element);
//   warp 1 (one lane): 4 K-substeps x 3 MMAs  D[j, i] += A[j, :] B[i, :]  (D = C^T, M =
//          128 columns, N = KP ranks, accumulated in TMEM over the whole block).
// Epilogue (warps 4-7, lane = column j): C[:, j] from TMEM, c_i = g_i C_ij split into
// TF32 hi/lo rows of Ch/Cl (layout [block][column][rank]), and r.z of column j.
struct PjArgs {
  const int32_t* blk_order;
  const int64_t* v0;
  const int32_t* rows;
  int nb, nct, c, k;
  const float* gain;  // FP32 copy, nb x k
  double inv1l;
  float* Ch;
  float* Cl;
  int64_t c128;
  double* rz;  // [nb][c] or nullptr
  const int32_t* run_flag;
  int* err;
};

constexpr int PJ_RSTAGES = 5;  // R stages (16 KB each)
constexpr int PJ_BSTAGES = 5;  // Q^T hi/lo stages (2 x KP x 128 bytes)
constexpr int PJ_ASTAGES = 2;  // built R^T hi/lo stages (32 KB each)
constexpr uint32_t PJ_R_BYTES = PJ_ROWS * PJ_COLS * 4;
constexpr uint32_t PJ_A_BYTES = PJ_COLS * 128;  // one split

template <int KP>
__host__ __device__ constexpr uint32_t pj_smem_bytes() {
  return 1024 + PJ_RSTAGES * PJ_R_BYTES + PJ_BSTAGES * 2 * KP * 128 + PJ_ASTAGES * 2 * PJ_A_BYTES + 256;
}

// One 32-row step of the builders: column t of the staged rows, rows [lo, hi) kept.
template <bool MASK>
__device__ __forceinline__ float pj_build(const float* __restrict__ stg, uint8_t* ah, uint8_t* al, int t, int lo,
                                          int hi) {
  float ss = 0.f;
#pragma unroll
  for (int g = 0; g < PJ_ROWS / 4; ++g) {
    float h[4], l[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int i = 4 * g + e;
      float x = stg[i * PJ_COLS + t];
      if (MASK && (i < lo || i >= hi)) x = 0.f;  // rows of the neighbouring blocks
      ss = fmaf(x, x, ss);
      h[e] = tf32_round(x);
      l[e] = x - h[e];
    }
    const uint32_t off = sw128_offset_f32(t, 4 * g);
    *reinterpret_cast<float4*>(ah + off) = make_float4(h[0], h[1], h[2], h[3]);
    *reinterpret_cast<float4*>(al + off) = make_float4(l[0], l[1], l[2], l[3]);
  }
  return ss;
}

template <int KP>
__global__ void __launch_bounds__(TC_THREADS, 1)
k_pc_proj_tc(const __grid_constant__ CUtensorMap mapR, const __grid_constant__ CUtensorMap mapQTh,
             const __grid_constant__ CUtensorMap mapQTl, PjArgs a) {
  if (a.run_flag && *a.run_flag == 0) return;
  constexpr uint32_t B_BYTES = KP * 128;  // per split
  constexpr uint32_t BS = 2 * B_BYTES;    // one B stage
  constexpr uint32_t AS = 2 * PJ_A_BYTES; // one A stage
  constexpr uint32_t ACC_COLS = KP;
  constexpr uint32_t TMEM_COLS = 2 * KP;
  constexpr uint32_t IDESC = umma::idesc_tf32_f32(PJ_COLS, KP);
  static_assert(PJ_R_BYTES % 1024 == 0 && BS % 1024 == 0 && AS % 1024 == 0, "stages must keep 1024-byte alignment");

  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* sR = smem;
  uint8_t* sB = sR + PJ_RSTAGES * PJ_R_BYTES;
  uint8_t* sA = sB + PJ_BSTAGES * BS;
  uint64_t* r_full = reinterpret_cast<uint64_t*>(sA + PJ_ASTAGES * AS);
  uint64_t* r_empty = r_full + PJ_RSTAGES;
  uint64_t* b_full = r_empty + PJ_RSTAGES;
  uint64_t* b_empty = b_full + PJ_BSTAGES;
  uint64_t* a_full = b_empty + PJ_BSTAGES;
  uint64_t* a_empty = a_full + PJ_ASTAGES;
  uint64_t* acc_full = a_empty + PJ_ASTAGES;  // 2
  uint64_t* acc_empty = acc_full + 2;           // 2
  uint64_t* mma_drain = acc_empty + 2;          // 1: the issuer's MMAs, after an error
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(mma_drain + 1);

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const int nunits = a.nb * a.nct;

  if (threadIdx.x == 0) {
    for (int s = 0; s < PJ_RSTAGES; ++s) {
      mbar_init(r_full + s, 1);
      mbar_init(r_empty + s, 4);  // one arrival per builder warp
    }
    for (int s = 0; s < PJ_BSTAGES; ++s) {
      mbar_init(b_full + s, 1);
      mbar_init(b_empty + s, 1);
    }
    for (int s = 0; s < PJ_ASTAGES; ++s) {
      mbar_init(a_full + s, 4);
      mbar_init(a_empty + s, 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(acc_full + b, 1);
      mbar_init(acc_empty + b, 4);
    }
    mbar_init(mma_drain, 1);
    umma::fence_barrier_init();
  }
  if (warp == 2) umma::tmem_alloc(tmem_slot, TMEM_COLS);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  // units in decreasing block size, dealt to the CTAs in rounds of gridDim.x that
  // alternate direction (every full odd round reversed), which evens out the CTAs' rows
  auto unit_rows = [&](int u, int& b, int& ct, int64_t& b0, int64_t& bend, int64_t& rs, int& nsteps) {
    const int G = (int)gridDim.x, r = u / G;
    if ((r & 1) && (r + 1) * G <= nunits) u = r * G + (G - 1 - (u - r * G));
    b = a.blk_order[u / a.nct];
    ct = u % a.nct;
    b0 = a.v0[b];
    bend = b0 + a.rows[b];
    rs = b0 & ~(int64_t)(PJ_ROWS - 1);
    nsteps = (int)((bend - rs + PJ_ROWS - 1) / PJ_ROWS);
  };

  if (warp == 0 || warp == 3) {
    // ---------------- TMA producers: R (warp 0), Q^T hi/lo (warp 3) ----------------
    if (lane == 0) {
      const bool rprod = warp == 0;
      const int nst = rprod ? PJ_RSTAGES : PJ_BSTAGES;
      uint64_t* full = rprod ? r_full : b_full;
      uint64_t* empty = rprod ? r_empty : b_empty;
      int stage = 0;
      uint32_t phase = 0;
      bool ok = true;
      umma::ArmedPhases<(PJ_RSTAGES > PJ_BSTAGES ? PJ_RSTAGES : PJ_BSTAGES)> armed;
      for (int u = blockIdx.x; u < nunits && ok; u += gridDim.x) {
        int b, ct, nsteps;
        int64_t b0, bend, rs;
        unit_rows(u, b, ct, b0, bend, rs, nsteps);
        for (int s = 0; s < nsteps; ++s) {
          if (!mbar_wait(empty + stage, phase ^ 1, a.err)) {
            ok = false;
            break;
          }
          armed.p[stage] = (uint8_t)phase;
          const int row = (int)(rs + (int64_t)s * PJ_ROWS);
          if (rprod) {
            mbar_arrive_expect_tx(full + stage, PJ_R_BYTES);
            tma_load_2d(sR + stage * PJ_R_BYTES, &mapR, full + stage, ct * PJ_COLS, row);
          } else {
            uint8_t* sb = sB + stage * BS;
            mbar_arrive_expect_tx(full + stage, BS);
            tma_load_2d(sb, &mapQTh, full + stage, row, 0);
            tma_load_2d(sb + B_BYTES, &mapQTl, full + stage, row, 0);
          }
          if (++stage == nst) {
            stage = 0;
            phase ^= 1;
          }
        }
      }
      if (*(volatile int*)a.err != 0) armed.drain(full);
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      int bstage = 0, astage = 0;
      uint32_t bphase = 0, aphase = 0;
      int acc = 0;
      uint32_t acc_phase = 0;
      bool ok = true;
      for (int u = blockIdx.x; u < nunits && ok; u += gridDim.x) {
        int b, ct, nsteps;
        int64_t b0, bend, rs;
        unit_rows(u, b, ct, b0, bend, rs, nsteps);
        if (!mbar_wait(acc_empty + acc, acc_phase ^ 1, a.err)) break;
        tc_fence_after();
        const uint32_t d_tmem = tmem_base + (uint32_t)acc * ACC_COLS;
        for (int s = 0; s < nsteps; ++s) {
          if (!mbar_wait(b_full + bstage, bphase, a.err) || !mbar_wait(a_full + astage, aphase, a.err)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t sa = smem_u32(sA + astage * AS), sb = smem_u32(sB + bstage * BS);
          const uint64_t ah = smem_desc_sw128(sa), al = smem_desc_sw128(sa + PJ_A_BYTES);
          const uint64_t bh = smem_desc_sw128(sb), bl = smem_desc_sw128(sb + B_BYTES);
#pragma unroll
          for (int kk = 0; kk < PJ_ROWS / 8; ++kk) {
            // 8 TF32 elements (32 bytes) along K per MMA inside the 128-byte swizzled row
            const uint64_t off = (uint64_t)((kk * 32) >> 4);
            umma::mma_tf32(d_tmem, ah + off, bh + off, IDESC, (s > 0 || kk > 0) ? 1u : 0u);
            umma::mma_tf32(d_tmem, ah + off, bl + off, IDESC, 1u);
            umma::mma_tf32(d_tmem, al + off, bh + off, IDESC, 1u);
          }
          umma::mma_commit(b_empty + bstage);
          umma::mma_commit(a_empty + astage);
          if (++bstage == PJ_BSTAGES) {
            bstage = 0;
            bphase ^= 1;
          }
          if (++astage == PJ_ASTAGES) {
            astage = 0;
            aphase ^= 1;
          }
        }
        if (!ok) break;
        umma::mma_commit(acc_full + acc);
        if (++acc == 2) {
          acc = 0;
          acc_phase ^= 1;
        }
      }
      if (*(volatile int*)a.err != 0) {
        umma::mma_commit(mma_drain);
        umma::mbar_drain(mma_drain, 0);
      }
    }
  } else if (warp >= 4) {
    // ---------------- operand builders, then the epilogue ----------------
    const int quarter = warp & 3;
    const int t = quarter * 32 + lane;  // A row = panel column of the unit
    int rstage = 0, astage = 0;
    uint32_t rphase = 0, aphase = 0;
    int acc = 0;
    uint32_t acc_phase = 0;
    bool ok = true;
    for (int u = blockIdx.x; u < nunits && ok; u += gridDim.x) {
      int b, ct, nsteps;
      int64_t b0, bend, rs;
      unit_rows(u, b, ct, b0, bend, rs, nsteps);
      double rr = 0.0;
      for (int s = 0; s < nsteps; ++s) {
        if (!mbar_wait(r_full + rstage, rphase, a.err) || !mbar_wait(a_empty + astage, aphase ^ 1, a.err)) {
          ok = false;
          break;
        }
        const float* stg = reinterpret_cast<const float*>(sR + rstage * PJ_R_BYTES);
        uint8_t* ah = sA + astage * AS;
        const int64_t row0 = rs + (int64_t)s * PJ_ROWS;
        const int lo = (int)(b0 > row0 ? b0 - row0 : 0);
        const int hi = (int)(bend - row0 < PJ_ROWS ? bend - row0 : PJ_ROWS);
        // r.r per 32-row step in FP32, across steps in FP64
        const float ss = (lo == 0 && hi == PJ_ROWS) ? pj_build<false>(stg, ah, ah + PJ_A_BYTES, t, 0, PJ_ROWS)
                                                    : pj_build<true>(stg, ah, ah + PJ_A_BYTES, t, lo, hi);
        rr += (double)ss;
        umma::fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) {
          mbar_arrive(r_empty + rstage);
          mbar_arrive(a_full + astage);
        }
        if (++rstage == PJ_RSTAGES) {
          rstage = 0;
          rphase ^= 1;
        }
        if (++astage == PJ_ASTAGES) {
          astage = 0;
          aphase ^= 1;
        }
      }
      if (!ok) break;
      if (!mbar_wait(acc_full + acc, acc_phase, a.err)) break;
      tc_fence_after();
      float cv[KP];
      const uint32_t taddr = tmem_base + (uint32_t)acc * ACC_COLS + ((uint32_t)(quarter * 32) << 16);
#pragma unroll
      for (int cb = 0; cb < KP / 16; ++cb) {
        uint32_t r[16];
        umma::tmem_ld16(taddr + cb * 16, r);
        umma::tmem_ld_wait();
#pragma unroll
        for (int q = 0; q < 16; ++q) cv[cb * 16 + q] = __uint_as_float(r[q]);
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(acc_empty + acc);
      if (++acc == 2) {
        acc = 0;
        acc_phase ^= 1;
      }
      const int j = ct * PJ_COLS + t;
      const float* gb = a.gain + (int64_t)b * a.k;
      float* ch = a.Ch + ((int64_t)b * a.c128 + j) * KP;
      float* cl = a.Cl + ((int64_t)b * a.c128 + j) * KP;
      float gcc = 0.f;  // sum_i g_i C_ij^2: 64 non-negative terms, FP32 is plenty
#pragma unroll
      for (int q = 0; q < KP / 4; ++q) {
        float h[4], l[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int i = 4 * q + e;
          const float x = (i < a.k ? gb[i] : 0.f) * cv[i];
          gcc = fmaf(x, cv[i], gcc);
          h[e] = tf32_round(x);
          l[e] = tf32_round(x - h[e]);
        }
        *reinterpret_cast<float4*>(ch + 4 * q) = make_float4(h[0], h[1], h[2], h[3]);
        *reinterpret_cast<float4*>(cl + 4 * q) = make_float4(l[0], l[1], l[2], l[3]);
      }
      if (a.rz && j < a.c) a.rz[(int64_t)b * a.c + j] = rr * a.inv1l + (double)gcc;
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 2) {
    tc_fence_after();
    umma::tmem_dealloc(tmem_base, TMEM_COLS);
  }
}

// ---------------------------------------------------------------------------
// Expansion.  Work unit = one 128-row tile of a block (rows past the block's end are
// computed from the next block's factors and discarded); per unit the Q_b rows (hi/lo,
// 128 x KP) stay in shared memory while the column steps of 64 stream through:
//   warp 0 (one lane): TMA of Q rows once per unit, then per step the C_b^T rows hi/lo
//          (64 x KP) into a ring of operand stages;
//   warp 3 (one lane): TMA of the R tile (128 x 64, two 128-byte-swizzled boxes) into a
//          deeper ring of R stages (the DRAM stream);
//   warp 1 (one lane): KP/8 K-substeps x 3 MMAs  D[r, j] += Q[r, :] C[:, j];
//   warps 4-7 (lane = row): z = R/(1+lam) + D written over the staged R, then stored to
//          Z by whole rows (two rows of 64 columns per warp instruction).
struct ExArgs {
  const int32_t* exp_block;
  const int32_t* exp_tile;
  int nexp;
  const int64_t* v0;
  const int32_t* rows;
  float* Z;
  int64_t ldz;
  int c, ncs;
  int64_t c128;
  float inv1l;
  const int32_t* run_flag;
  int* err;
};

constexpr int EX_RSTAGES = 3;
constexpr int EX_BSTAGES = 2;
constexpr uint32_t EX_RBOX = EX_ROWS * 128;                  // 16 KB (32 columns)
constexpr uint32_t EX_R_BYTES = (EX_COLS / 32) * EX_RBOX;    // 32 KB per R stage

template <int KP>
__host__ __device__ constexpr uint32_t ex_a_bytes() {
  return 2 * (KP / 32) * EX_ROWS * 128;
}
template <int KP>
__host__ __device__ constexpr uint32_t ex_b_bytes() {
  return 2 * (KP / 32) * EX_COLS * 128;
}
template <int KP>
__host__ __device__ constexpr uint32_t ex_smem_bytes() {
  return 1024 + ex_a_bytes<KP>() + EX_BSTAGES * ex_b_bytes<KP>() + EX_RSTAGES * EX_R_BYTES + 256;
}

template <int KP>
__global__ void __launch_bounds__(TC_THREADS, 1)
k_pc_expand_tc(const __grid_constant__ CUtensorMap mapR, const __grid_constant__ CUtensorMap mapQh,
               const __grid_constant__ CUtensorMap mapQl, const __grid_constant__ CUtensorMap mapCh,
               const __grid_constant__ CUtensorMap mapCl, ExArgs a) {
  if (a.run_flag && *a.run_flag == 0) return;
  constexpr int KB = KP / 32;                     // 128-byte K boxes
  constexpr uint32_t QBOX = EX_ROWS * 128;        // 16 KB
  constexpr uint32_t A_BYTES = ex_a_bytes<KP>();  // Qh then Ql
  constexpr uint32_t CBOX = EX_COLS * 128;        // 8 KB
  constexpr uint32_t B_BYTES = ex_b_bytes<KP>();  // Ch then Cl
  constexpr uint32_t ACC_COLS = EX_COLS;
  constexpr uint32_t TMEM_COLS = 2 * EX_COLS;
  constexpr uint32_t IDESC = umma::idesc_tf32_f32(EX_ROWS, EX_COLS);
  static_assert(A_BYTES % 1024 == 0 && B_BYTES % 1024 == 0, "tiles must keep 1024-byte alignment");

  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* sA = smem;
  uint8_t* sB = smem + A_BYTES;
  uint8_t* sR = sB + EX_BSTAGES * B_BYTES;
  uint64_t* a_full = reinterpret_cast<uint64_t*>(sR + EX_RSTAGES * EX_R_BYTES);
  uint64_t* a_empty = a_full + 1;
  uint64_t* b_full = a_empty + 1;
  uint64_t* b_empty = b_full + EX_BSTAGES;
  uint64_t* r_full = b_empty + EX_BSTAGES;
  uint64_t* r_empty = r_full + EX_RSTAGES;
  uint64_t* acc_full = r_empty + EX_RSTAGES;  // 2
  uint64_t* acc_empty = acc_full + 2;         // 2
  uint64_t* mma_drain = acc_empty + 2;        // 1: the issuer's MMAs, after an error
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(mma_drain + 1);

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    mbar_init(a_full, 1);
    mbar_init(a_empty, 1);
    for (int s = 0; s < EX_BSTAGES; ++s) {
      mbar_init(b_full + s, 1);
      mbar_init(b_empty + s, 1);
    }
    for (int s = 0; s < EX_RSTAGES; ++s) {
      mbar_init(r_full + s, 1);
      mbar_init(r_empty + s, 4);  // one arrival per epilogue warp
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(acc_full + b, 1);
      mbar_init(acc_empty + b, 4);
    }
    mbar_init(mma_drain, 1);
    umma::fence_barrier_init();
  }
  if (warp == 2) umma::tmem_alloc(tmem_slot, TMEM_COLS);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  if (warp == 0) {
    // ---------------- TMA producer: Q rows and C^T rows ----------------
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0, aphase = 0;
      bool ok = true;
      umma::ArmedPhases<EX_BSTAGES> armed;
      umma::ArmedPhases<1> a_armed;
      for (int u = blockIdx.x; u < a.nexp && ok; u += gridDim.x) {
        const int b = a.exp_block[u];
        const int row0 = (int)(a.v0[b] + (int64_t)a.exp_tile[u] * EX_ROWS);
        if (!mbar_wait(a_empty, aphase ^ 1, a.err)) break;
        a_armed.p[0] = (uint8_t)aphase;  // the phase of a_full this load completes
        aphase ^= 1;
        mbar_arrive_expect_tx(a_full, A_BYTES);
#pragma unroll
        for (int q = 0; q < KB; ++q) {
          tma_load_2d(sA + q * QBOX, &mapQh, a_full, 32 * q, row0);
          tma_load_2d(sA + (KB + q) * QBOX, &mapQl, a_full, 32 * q, row0);
        }
        const int crow = (int)((int64_t)b * a.c128);
        for (int cs = 0; cs < a.ncs; ++cs) {
          if (!mbar_wait(b_empty + stage, phase ^ 1, a.err)) {
            ok = false;
            break;
          }
          armed.p[stage] = (uint8_t)phase;
          uint8_t* sb = sB + stage * B_BYTES;
          mbar_arrive_expect_tx(b_full + stage, B_BYTES);
#pragma unroll
          for (int q = 0; q < KB; ++q) {
            tma_load_2d(sb + q * CBOX, &mapCh, b_full + stage, 32 * q, crow + cs * EX_COLS);
            tma_load_2d(sb + (KB + q) * CBOX, &mapCl, b_full + stage, 32 * q, crow + cs * EX_COLS);
          }
          if (++stage == EX_BSTAGES) {
            stage = 0;
            phase ^= 1;
          }
        }
      }
      if (*(volatile int*)a.err != 0) {
        armed.drain(b_full);
        a_armed.drain(a_full);
      }
    }
  } else if (warp == 3) {
    // ---------------- TMA producer: R tiles ----------------
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      bool ok = true;
      umma::ArmedPhases<EX_RSTAGES> armed;
      for (int u = blockIdx.x; u < a.nexp && ok; u += gridDim.x) {
        const int b = a.exp_block[u];
        const int row0 = (int)(a.v0[b] + (int64_t)a.exp_tile[u] * EX_ROWS);
        for (int cs = 0; cs < a.ncs; ++cs) {
          if (!mbar_wait(r_empty + stage, phase ^ 1, a.err)) {
            ok = false;
            break;
          }
          armed.p[stage] = (uint8_t)phase;
          uint8_t* sr = sR + stage * EX_R_BYTES;
          mbar_arrive_expect_tx(r_full + stage, EX_R_BYTES);
#pragma unroll
          for (int h = 0; h < EX_COLS / 32; ++h)
            tma_load_2d(sr + h * EX_RBOX, &mapR, r_full + stage, cs * EX_COLS + 32 * h, row0);
          if (++stage == EX_RSTAGES) {
            stage = 0;
            phase ^= 1;
          }
        }
      }
      if (*(volatile int*)a.err != 0) armed.drain(r_full);
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0, aphase = 0;
      int acc = 0;
      uint32_t acc_phase = 0;
      bool ok = true;
      const uint32_t a0 = smem_u32(sA);
      for (int u = blockIdx.x; u < a.nexp && ok; u += gridDim.x) {
        if (!mbar_wait(a_full, aphase, a.err)) break;
        aphase ^= 1;
        for (int cs = 0; cs < a.ncs; ++cs) {
          if (!mbar_wait(b_full + stage, phase, a.err) || !mbar_wait(acc_empty + acc, acc_phase ^ 1, a.err)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t d_tmem = tmem_base + (uint32_t)acc * ACC_COLS;
          const uint32_t b0 = smem_u32(sB + stage * B_BYTES);
#pragma unroll
          for (int kk = 0; kk < KP / 8; ++kk) {
            const int q = kk >> 2;
            const uint64_t off = (uint64_t)(((kk & 3) * 32) >> 4);
            const uint64_t ah = smem_desc_sw128(a0 + q * QBOX) + off;
            const uint64_t al = smem_desc_sw128(a0 + (KB + q) * QBOX) + off;
            const uint64_t bh = smem_desc_sw128(b0 + q * CBOX) + off;
            const uint64_t bl = smem_desc_sw128(b0 + (KB + q) * CBOX) + off;
            umma::mma_tf32(d_tmem, ah, bh, IDESC, kk > 0 ? 1u : 0u);
            umma::mma_tf32(d_tmem, ah, bl, IDESC, 1u);
            umma::mma_tf32(d_tmem, al, bh, IDESC, 1u);
          }
          umma::mma_commit(b_empty + stage);
          umma::mma_commit(acc_full + acc);
          if (++stage == EX_BSTAGES) {
            stage = 0;
            phase ^= 1;
          }
          if (++acc == 2) {
            acc = 0;
            acc_phase ^= 1;
          }
        }
        umma::mma_commit(a_empty);  // the Q tile is free once this unit's MMAs are done
      }
      if (*(volatile int*)a.err != 0) {
        umma::mma_commit(mma_drain);
        umma::mbar_drain(mma_drain, 0);
      }
    }
  } else if (warp >= 4) {
    // ---------------- epilogue ----------------
    const int quarter = warp & 3;
    const int t = quarter * 32 + lane;  // tile row (TMEM lane)
    int stage = 0;
    uint32_t phase = 0;
    int acc = 0;
    uint32_t acc_phase = 0;
    bool ok = true;
    for (int u = blockIdx.x; u < a.nexp && ok; u += gridDim.x) {
      const int b = a.exp_block[u];
      const int64_t row0 = a.v0[b] + (int64_t)a.exp_tile[u] * EX_ROWS;
      const int64_t bend = a.v0[b] + a.rows[b];
      for (int cs = 0; cs < a.ncs; ++cs) {
        if (!mbar_wait(acc_full + acc, acc_phase, a.err) || !mbar_wait(r_full + stage, phase, a.err)) {
          ok = false;
          break;
        }
        tc_fence_after();
        float d[EX_COLS];
        const uint32_t taddr = tmem_base + (uint32_t)acc * ACC_COLS + ((uint32_t)(quarter * 32) << 16);
#pragma unroll
        for (int cb = 0; cb < EX_COLS / 16; ++cb) {
          uint32_t r[16];
          umma::tmem_ld16(taddr + cb * 16, r);
          umma::tmem_ld_wait();
#pragma unroll
          for (int q = 0; q < 16; ++q) d[cb * 16 + q] = __uint_as_float(r[q]);
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(acc_empty + acc);
        if (++acc == 2) {
          acc = 0;
          acc_phase ^= 1;
        }
        // z = R/(1+lam) + D over this thread's row of the staged R tile
        uint8_t* rst = sR + stage * EX_R_BYTES;
#pragma unroll
        for (int h = 0; h < EX_COLS / 32; ++h)
#pragma unroll
          for (int g = 0; g < 8; ++g) {
            float4* p = reinterpret_cast<float4*>(rst + h * EX_RBOX + sw128_offset_f32(t, 4 * g));
            const float4 r = *p;
            const int j = 32 * h + 4 * g;
            *p = make_float4(fmaf(a.inv1l, r.x, d[j]), fmaf(a.inv1l, r.y, d[j + 1]), fmaf(a.inv1l, r.z, d[j + 2]),
                             fmaf(a.inv1l, r.w, d[j + 3]));
          }
        __syncwarp();
        // this warp's 32 rows to Z, two rows per instruction (16 lanes x 16 bytes each)
        const int ch = lane & 15, h = ch >> 3, g = ch & 7;
        const int col = cs * EX_COLS + 4 * ch;
#pragma unroll 4
        for (int it = 0; it < 16; ++it) {
          const int rr = quarter * 32 + 2 * it + (lane >> 4);
          const int64_t grow = row0 + rr;
          if (grow >= bend) continue;
          const float4 z = *reinterpret_cast<const float4*>(rst + h * EX_RBOX + sw128_offset_f32(rr, 4 * g));
          float* zp = a.Z + grow * a.ldz + col;
          if (col + 3 < a.c) {
            *reinterpret_cast<float4*>(zp) = z;
          } else {
            if (col < a.c) zp[0] = z.x;
            if (col + 1 < a.c) zp[1] = z.y;
            if (col + 2 < a.c) zp[2] = z.z;
          }
        }
        // the staged tile was also written through the generic proxy: order that
        // before the TMA that refills the stage
        umma::fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) mbar_arrive(r_empty + stage);
        if (++stage == EX_RSTAGES) {
          stage = 0;
          phase ^= 1;
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 2) {
    tc_fence_after();
    umma::tmem_dealloc(tmem_base, TMEM_COLS);
  }
}

}  // namespace

hgl_status precond_tc_maps(hgl_precond* P) {
  const uint64_t kp = (uint64_t)P->kp;
  const auto f32 = CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
  const auto sw = CU_TENSOR_MAP_SWIZZLE_128B;
  HGL_TRY(encode_map_2d(&P->mQh, f32, P->Qh, kp, (uint64_t)P->n, kp * 4, 32, EX_ROWS, sw));
  HGL_TRY(encode_map_2d(&P->mQl, f32, P->Ql, kp, (uint64_t)P->n, kp * 4, 32, EX_ROWS, sw));
  HGL_TRY(encode_map_2d(&P->mQTh, f32, P->QTh, (uint64_t)P->n4, kp, (uint64_t)P->n4 * 4, 32, (uint32_t)kp, sw));
  HGL_TRY(encode_map_2d(&P->mQTl, f32, P->QTl, (uint64_t)P->n4, kp, (uint64_t)P->n4 * 4, 32, (uint32_t)kp, sw));
  return HGL_OK;
}

namespace {

template <class F>
hgl_status tc_smem_attr(F* fn, size_t bytes) {
  HGL_CHECK_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
  return HGL_OK;
}

template <int KP>
hgl_status tc_apply(hgl_precond* P, const float* R, int64_t ldr, float* Z, int64_t ldz, int c, double* rz,
                    cudaStream_t st, const int32_t* run_flag) {
  const int64_t c128 = rup(c, PJ_COLS);
  hgl_status s = HGL_OK;
  float* Ch = static_cast<float*>(buffer_get(P->cbuf, sizeof(float) * 2 * (size_t)P->nb * c128 * KP, &s));
  if (!Ch) return s;
  float* Cl = Ch + (size_t)P->nb * c128 * KP;
  const auto f32 = CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
  CUtensorMap mRp, mRe, mCh, mCl;
  HGL_TRY(encode_map_2d(&mRp, f32, R, (uint64_t)c, (uint64_t)P->n, (uint64_t)ldr * 4, PJ_COLS, PJ_ROWS,
                        CU_TENSOR_MAP_SWIZZLE_NONE));
  HGL_TRY(encode_map_2d(&mRe, f32, R, (uint64_t)c, (uint64_t)P->n, (uint64_t)ldr * 4, 32, EX_ROWS,
                        CU_TENSOR_MAP_SWIZZLE_128B));
  HGL_TRY(encode_map_2d(&mCh, f32, Ch, KP, (uint64_t)P->nb * c128, KP * 4, 32, EX_COLS, CU_TENSOR_MAP_SWIZZLE_128B));
  HGL_TRY(encode_map_2d(&mCl, f32, Cl, KP, (uint64_t)P->nb * c128, KP * 4, 32, EX_COLS, CU_TENSOR_MAP_SWIZZLE_128B));
  const size_t smem_pj = pj_smem_bytes<KP>();
  const size_t smem_ex = ex_smem_bytes<KP>();
  // per call (a host-side attribute, also valid while a stream is being captured): the
  // setting is per device, and a process may apply on several
  HGL_TRY(tc_smem_attr(k_pc_proj_tc<KP>, smem_pj));
  HGL_TRY(tc_smem_attr(k_pc_expand_tc<KP>, smem_ex));
  const int sms = device_sm_count();
  PjArgs pa{P->blk_order, P->d_v0, P->d_rows, P->nb, (int)(c128 / PJ_COLS), c, P->k, P->gain32,
            1.0 / (1.0 + P->lam), Ch, Cl, c128, rz, run_flag, P->d_err};
  ExArgs ea{P->exp_block, P->exp_tile, P->nexp, P->d_v0, P->d_rows, Z, ldz, c, (c + EX_COLS - 1) / EX_COLS,
            c128, (float)(1.0 / (1.0 + P->lam)), run_flag, P->d_err};
  hgl::count_launch(2);
  k_pc_proj_tc<KP><<<std::min(P->nb * pa.nct, sms), TC_THREADS, smem_pj, st>>>(mRp, P->mQTh, P->mQTl, pa);
  k_pc_expand_tc<KP><<<std::min(P->nexp, sms), TC_THREADS, smem_ex, st>>>(mRe, P->mQh, P->mQl, mCh, mCl, ea);
  HGL_CHECK_CUDA(cudaGetLastError());
  return HGL_OK;
}

}  // namespace

bool precond_tc_usable(const hgl_precond* P, const void* R, int64_t ldr, const void* Z, int64_t ldz) {
  return P && P->tc && P->tc_on && ldr % 4 == 0 && ldz % 4 == 0 && (reinterpret_cast<uintptr_t>(R) & 15) == 0 &&
         (reinterpret_cast<uintptr_t>(Z) & 15) == 0 && P->n < ((int64_t)1 << 31);
}

hgl_status precond_tc_apply(hgl_precond* P, const float* R, int64_t ldr, float* Z, int64_t ldz, int c, double* rz,
                            cudaStream_t st, const int32_t* run_flag) {
  ProfScope prof(HGL_PROF_PRECOND, st);
  return P->kp == 32 ? tc_apply<32>(P, R, ldr, Z, ldz, c, rz, st, run_flag)
                     : tc_apply<64>(P, R, ldr, Z, ldz, c, rz, st, run_flag);
}

}  // namespace hgl

extern "C" hgl_status hgl_precond_tensor_cores(hgl_precond* P, int32_t on, int32_t* active) {
  if (!P) return hgl::record_error(HGL_ERR_INVALID_ARG, "preconditioner is NULL");
  P->tc_on = on != 0;
  if (active) *active = P->tc ? 1 : 0;
  return HGL_OK;
}

namespace hgl {

hgl_status precond_tc_status(hgl_precond* P, cudaStream_t st) {
  if (!P || !P->tc) return HGL_OK;
  int32_t e = 0;
  HGL_CHECK_CUDA(cudaMemcpyAsync(&e, P->d_err, sizeof(e), cudaMemcpyDeviceToHost, st));
  HGL_CHECK_CUDA(cudaStreamSynchronize(st));
  if (e == 0) return HGL_OK;
  HGL_CHECK_CUDA(cudaMemsetAsync(P->d_err, 0, sizeof(int32_t), st));
  return record_error(HGL_ERR_TIMEOUT, "a tensor-core preconditioner kernel hit its wait limit");
}

hgl_status precond_tc_prepare(hgl_precond* P, cudaStream_t st) {
  const int grid = (int)std::min<int64_t>((P->n4 + 31) / 32, (int64_t)device_sm_count() * 8);
  hgl::count_launch();
  if (P->kp == 32)
    k_tc_split<32><<<grid, 256, 0, st>>>(P->n, P->n4, P->k, static_cast<const float*>(P->Q), P->Qh, P->Ql, P->QTh,
                                         P->QTl);
  else
    k_tc_split<64><<<grid, 256, 0, st>>>(P->n, P->n4, P->k, static_cast<const float*>(P->Q), P->Qh, P->Ql, P->QTh,
                                         P->QTl);
  HGL_CHECK_CUDA(cudaGetLastError());
  return HGL_OK;
}

}  // namespace hgl
