// umma.cuh -- Blackwell (sm_103a) tensor-core primitives written as inline PTX:
// mbarriers with bounded waits, TMA tile loads, TMEM allocation, tcgen05.mma with
// BF16 inputs and FP32 accumulation in TMEM, and tcgen05.ld for the epilogue; plus
// the grouped GEMM of the block randomized SVD built from them.
//
// Grouped GEMM (one launch for all tessellation blocks):
//   D_b[r, :] = sum_k A_b[r, k] * B_b[:, k]     (D_b = Theta_bb * S_b, S_b^T stored as B_b)
// A: every block's Theta_bb, rows stacked (each block padded to a multiple of 128 rows),
//    row stride ldA, BF16, K-major.  B: the l_pad x (sum of padded block widths) matrix
//    holding S_b^T side by side, BF16, K-major.  D: FP32, rows as in A, l_pad columns.
// Work unit = (block, 128-row tile); persistent CTAs stride over units ordered by
// decreasing K.  Warp roles: warp 0 issues TMA loads into a ring of smem stages, warp 1
// issues tcgen05.mma (one elected lane) into a double-buffered TMEM accumulator, warp 2
// owns the TMEM allocation, warps 4-7 drain TMEM (one lane quarter each) and store D.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>

namespace hgl {
namespace umma {

constexpr int BLOCK_M = 128;   // rows per tile (TMEM lanes)
constexpr int BLOCK_K = 64;    // BF16 elements per 128-byte swizzle row
constexpr int UMMA_K = 16;     // K per tcgen05.mma for 16-bit inputs
constexpr int STAGES = 6;
constexpr int THREADS = 256;
constexpr unsigned long long SPIN_CYCLES = 4000000000ull;  // ~2 s at 2 GHz

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_barrier_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n"
      " .reg .pred p;\n"
      " mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n"
      "}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Wait for phase `parity` of a barrier.  Gives up after ~2 s, or soon after another
// role has flagged an error; on give-up records code 1 in *err and returns false so
// the caller can leave its loop.  The error word and the clock are read only every 64
// polls (each poll is a try_wait, which itself suspends for a while): a global read on
// every poll would delay the waiter's wake-up by a memory latency.
__device__ __forceinline__ bool mbar_wait_limit(uint64_t* bar, uint32_t parity, int* err,
                                                unsigned long long limit_cycles) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = clock64();
  for (uint32_t it = 1;; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((it & 63u) == 0) {
      if (*(volatile int*)err != 0) return false;
      if (clock64() - t0 > limit_cycles) {
        atomicExch(err, 1);
        return false;
      }
    }
  }
}

__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int* err) {
  return mbar_wait_limit(bar, parity, err, SPIN_CYCLES);
}

// After a role gave up: wait, again with a limit and whatever the error word says,
// for phase `parity` of `bar` -- the landing of a copy this thread issued, or (with a
// commit barrier) the completion of its MMAs -- so that nothing still writes shared
// memory or reads TMEM when the CTA frees them and exits.
constexpr unsigned long long DRAIN_CYCLES = 200000000ull;  // ~0.1 s
__device__ __forceinline__ void mbar_drain(uint64_t* bar, uint32_t parity) {
  const unsigned long long t0 = clock64();
  while (!mbar_try_wait(bar, parity))
    if (clock64() - t0 > DRAIN_CYCLES) return;
}

// Per-stage record of the phase a producer last armed (2 = never), for the drain.
template <int N>
struct ArmedPhases {
  uint8_t p[N];
  __device__ __forceinline__ ArmedPhases() {
#pragma unroll
    for (int i = 0; i < N; ++i) p[i] = 2;
  }
  __device__ __forceinline__ void drain(uint64_t* full) const {
#pragma unroll
    for (int i = 0; i < N; ++i)
      if (p[i] != 2) mbar_drain(full + i, p[i]);
  }
};

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::"r"(
          smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(x), "r"(y)
      : "memory");
}

__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)), "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// D[tmem] (+)= A[smem] * B[smem]^T, kind::f16 (BF16 in, FP32 accumulate), one CTA.
__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n"
      " .reg .pred p;\n"
      " setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n"
      "}\n" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

// D[tmem] (+)= A[smem] * B[smem]^T, kind::tf32 (FP32 storage read as TF32, FP32
// accumulate), one CTA.
__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n"
      " .reg .pred p;\n"
      " setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n"
      "}\n" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

// Make this thread's generic-proxy shared-memory writes visible to the async proxy
// (tcgen05.mma operands written by threads instead of TMA).
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Barrier among `count` threads (a multiple of 32) on hardware barrier `id` (1-15).
__device__ __forceinline__ void named_barrier(int id, int count) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}

// x rounded to TF32 (10 explicit mantissa bits), to nearest, ties away from zero.
__device__ __forceinline__ float tf32_round(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// Arrive on `bar` once all previously issued tcgen05.mma of this thread complete.
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

// 32 lanes x 16 consecutive 32-bit TMEM columns -> 16 registers per thread.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t* r) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}

__device__ __forceinline__ void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Shared-memory matrix descriptor for a K-major tile stored by TMA with 128-byte
// swizzling: rows of 128 bytes, 8-row (1024-byte) swizzle atoms stacked along M/N.
// Fields: start address >> 4 (bits 0-13), leading byte offset >> 4 (16-29, unused for
// this layout, set to 1), stride byte offset >> 4 (32-45, 1024 bytes between 8-row
// groups), descriptor version 1 (bits 46-47), layout SWIZZLE_128B = 2 (bits 61-63).
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}

// Instruction descriptor, kind::f16: D FP32 (bits 4-5 = 1), A and B BF16 (bits 7-9 and
// 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 in bits 17-22, M >> 4 in bits 24-28.
__host__ __device__ constexpr uint32_t idesc_bf16_f32(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// Instruction descriptor, kind::tf32: D FP32 (bits 4-5 = 1), A and B TF32 (bits 7-9
// and 10-12 = 2), both K-major, N >> 3 in bits 17-22, M >> 4 in bits 24-28.
__host__ __device__ constexpr uint32_t idesc_tf32_f32(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// Byte offset of element (row, k) of a K-major tile of 32-bit elements stored with
// 128-byte swizzling (the layout a TMA load with SWIZZLE_128B writes): 128-byte rows,
// the 16-byte chunk index XORed with row % 8.
__host__ __device__ constexpr uint32_t sw128_offset_f32(int row, int k) {
  return (uint32_t)row * 128u + ((((uint32_t)k >> 2) ^ ((uint32_t)row & 7u)) << 4) + (((uint32_t)k & 3u) << 2);
}

struct GemmUnits {
  const int32_t* unit_block;  // block of each work unit
  const int32_t* unit_tile;   // 128-row tile index inside the block
  const int32_t* blk_rows;    // rows (= K) of each block
  const int64_t* blk_arow;    // first row of the block in A and D
  const int64_t* blk_koff;    // first column of the block in B
  int nunits;
};

// Shared memory: STAGES x (A tile 16 KB + B tile l_pad*128 B) + barriers.
inline size_t gemm_smem_bytes(int l_pad) {
  return 1024 + (size_t)STAGES * (BLOCK_M * 128 + (size_t)l_pad * 128) + 256;
}

template <int LPAD>
__global__ void __launch_bounds__(THREADS, 1)
k_block_gemm(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB, GemmUnits U,
             float* __restrict__ D, int64_t ldd, int* __restrict__ err) {
  constexpr uint32_t A_BYTES = BLOCK_M * 128;
  constexpr uint32_t B_BYTES = LPAD * 128;
  constexpr uint32_t STAGE_BYTES = A_BYTES + B_BYTES;
  constexpr uint32_t ACC_COLS = LPAD <= 128 ? 128 : 256;  // one accumulator buffer
  constexpr uint32_t TMEM_COLS = 2 * ACC_COLS;              // double-buffered
  static_assert(TMEM_COLS <= 512, "accumulator does not fit TMEM");
  constexpr uint32_t IDESC = idesc_bf16_f32(BLOCK_M, LPAD);

  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + STAGES * STAGE_BYTES);
  uint64_t* empty = full + STAGES;
  uint64_t* acc_full = empty + STAGES;   // 2
  uint64_t* acc_empty = acc_full + 2;    // 2
  uint64_t* mma_drain = acc_empty + 2;   // 1: the issuer's MMAs, after an error
  uint32_t* tmem_base_slot = reinterpret_cast<uint32_t*>(mma_drain + 1);

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(full + s, 1);
      mbar_init(empty + s, 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(acc_full + b, 1);
      mbar_init(acc_empty + b, 4);  // one arrival per epilogue warp
    }
    mbar_init(mma_drain, 1);
    fence_barrier_init();
  }
  if (warp == 2) tmem_alloc(tmem_base_slot, TMEM_COLS);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_base_slot;

  if (warp == 0) {
    // ---------------- TMA producer ----------------
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      bool ok = true;
      ArmedPhases<STAGES> armed;
      for (int u = blockIdx.x; u < U.nunits && ok; u += gridDim.x) {
        const int b = U.unit_block[u];
        const int tile = U.unit_tile[u];
        const int K = U.blk_rows[b];
        const int ktiles = (K + BLOCK_K - 1) / BLOCK_K;
        const int ay = (int)(U.blk_arow[b] + (int64_t)tile * BLOCK_M);
        const int bx0 = (int)U.blk_koff[b];
        for (int kt = 0; kt < ktiles; ++kt) {
          if (!mbar_wait(empty + stage, phase ^ 1, err)) {
            ok = false;
            break;
          }
          uint8_t* sa = smem + stage * STAGE_BYTES;
          mbar_arrive_expect_tx(full + stage, STAGE_BYTES);
          tma_load_2d(sa, &mapA, full + stage, kt * BLOCK_K, ay);
          tma_load_2d(sa + A_BYTES, &mapB, full + stage, bx0 + kt * BLOCK_K, 0);
          armed.p[stage] = (uint8_t)phase;
          if (++stage == STAGES) {
            stage = 0;
            phase ^= 1;
          }
        }
      }
      if (*(volatile int*)err != 0) armed.drain(full);
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      int acc = 0;
      uint32_t acc_phase = 0;
      bool ok = true;
      for (int u = blockIdx.x; u < U.nunits && ok; u += gridDim.x) {
        const int b = U.unit_block[u];
        const int K = U.blk_rows[b];
        const int ktiles = (K + BLOCK_K - 1) / BLOCK_K;
        if (!mbar_wait(acc_empty + acc, acc_phase ^ 1, err)) break;
        tc_fence_after();
        const uint32_t d_tmem = tmem_base + (uint32_t)acc * ACC_COLS;
        for (int kt = 0; kt < ktiles; ++kt) {
          if (!mbar_wait(full + stage, phase, err)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t sa = smem_u32(smem + stage * STAGE_BYTES);
          const uint64_t adesc = smem_desc_sw128(sa);
          const uint64_t bdesc = smem_desc_sw128(sa + A_BYTES);
#pragma unroll
          for (int kk = 0; kk < BLOCK_K / UMMA_K; ++kk) {
            // advance 16 elements (32 bytes) along K inside the 128-byte swizzled row
            const uint64_t off = (uint64_t)((kk * UMMA_K * 2) >> 4);
            mma_bf16(d_tmem, adesc + off, bdesc + off, IDESC, (kt > 0 || kk > 0) ? 1u : 0u);
          }
          mma_commit(empty + stage);
          if (++stage == STAGES) {
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
      if (*(volatile int*)err != 0) {
        mma_commit(mma_drain);
        mbar_drain(mma_drain, 0);
      }
    }
  } else if (warp >= 4) {
    // ---------------- epilogue: TMEM -> registers -> D ----------------
    const int quarter = warp & 3;
    int acc = 0;
    uint32_t acc_phase = 0;
    for (int u = blockIdx.x; u < U.nunits; u += gridDim.x) {
      const int b = U.unit_block[u];
      const int tile = U.unit_tile[u];
      const int rows = U.blk_rows[b];
      if (!mbar_wait(acc_full + acc, acc_phase, err)) break;
      tc_fence_after();
      const int r_in_block = tile * BLOCK_M + quarter * 32 + lane;
      float* drow = D + (U.blk_arow[b] + (int64_t)tile * BLOCK_M + quarter * 32 + lane) * ldd;
      const uint32_t taddr = tmem_base + (uint32_t)acc * ACC_COLS + ((uint32_t)(quarter * 32) << 16);
#pragma unroll
      for (int cb = 0; cb < LPAD / 16; ++cb) {
        uint32_t r[16];
        tmem_ld16(taddr + cb * 16, r);
        tmem_ld_wait();
        if (r_in_block < rows) {
          float4* dst = reinterpret_cast<float4*>(drow + cb * 16);
#pragma unroll
          for (int q = 0; q < 4; ++q)
            dst[q] = make_float4(__uint_as_float(r[4 * q]), __uint_as_float(r[4 * q + 1]),
                                 __uint_as_float(r[4 * q + 2]), __uint_as_float(r[4 * q + 3]));
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
    tmem_dealloc(tmem_base, TMEM_COLS);
  }
}

}  // namespace umma
}  // namespace hgl
