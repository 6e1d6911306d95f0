// rsvd_kernels.cuh -- CUDA-core kernels of the block randomized SVD (Section 3,
// Algorithm 1) and of the block preconditioner built from it.
#pragma once

#include <cuda_bf16.h>

#include <cstdint>

#include "hgl_internal.cuh"
#include "panel.cuh"

namespace hgl {
namespace rsvd {

constexpr uint32_t OMEGA_STREAM = 0x4F6D6567u;

// Per-block layout shared by the kernels.
struct Blocks {
  int nb;            // number of blocks
  int l, lpad;       // subspace width and its padded width (multiple of 16)
  int k;             // target rank
  int64_t ldA;       // row stride of the dense block storage (elements)
  int64_t Ktot;      // columns of the transposed-basis storage
  const int64_t* v0;     // first vertex of block b
  const int32_t* rows;   // size of block b
  const int64_t* arow;   // first storage row of block b (blocks padded to 128 rows)
  const int64_t* koff;   // first basis column of block b (blocks padded to 64 columns)
  const int32_t* lb;     // min(l, size)
  const int32_t* kb;     // min(k, size)
};

__device__ __forceinline__ int find_block(const int64_t* starts, int nb, int64_t x) {
  int lo = 0, hi = nb - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (starts[mid] <= x)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

template <class T> __device__ __forceinline__ float to_float(T x);
template <> __device__ __forceinline__ float to_float<float>(float x) { return x; }
template <> __device__ __forceinline__ float to_float<double>(double x) { return (float)x; }
template <> __device__ __forceinline__ float to_float<__nv_bfloat16>(__nv_bfloat16 x) { return __bfloat162float(x); }

template <class T> __device__ __forceinline__ T from_double(double x);
template <> __device__ __forceinline__ double from_double<double>(double x) { return x; }
template <> __device__ __forceinline__ float from_double<float>(double x) { return (float)x; }
template <> __device__ __forceinline__ __nv_bfloat16 from_double<__nv_bfloat16>(double x) {
  return __float2bfloat16_rn((float)x);
}

template <class T> __device__ __forceinline__ double to_double(T x) { return (double)to_float<T>(x); }
template <> __device__ __forceinline__ double to_double<double>(double x) { return x; }

// storage <-> accumulation type of the block assembly (no FP64 step for FP32 sums)
template <class TA> __device__ __forceinline__ TA from_acc(double x) { return from_double<TA>(x); }
// An FP32 or FP64 basis entry into the transposed basis' type (FP32 -> BF16 directly: the
// same rounding as through FP64, without two conversions on the slow FP64 pipe).
template <class TB, class T> __device__ __forceinline__ TB basis_from(T x) { return from_double<TB>((double)x); }
template <> __device__ __forceinline__ __nv_bfloat16 basis_from<__nv_bfloat16, float>(float x) {
  return __float2bfloat16_rn(x);
}
template <class TA> __device__ __forceinline__ TA from_acc(float x);
template <> __device__ __forceinline__ __nv_bfloat16 from_acc<__nv_bfloat16>(float x) {
  return __float2bfloat16_rn(x);
}
template <class TA, class S> __device__ __forceinline__ S to_acc(TA x) { return (S)to_float<TA>(x); }
template <> __device__ __forceinline__ double to_acc<double, double>(double x) { return x; }

// ---------------------------------------------------------------------------
// Dense diagonal blocks Theta_bb[i, j] = s_u s_v sum_{e containing u and v} t_e,
// u = v0 + i, v = v0 + j.  One warp per storage row: the row (padded width) is zeroed,
// the diagonal is summed over the vertex's hyperedges, and the off-diagonal terms are
// added hyperedge by hyperedge from the members that fall inside the block (found by
// binary search in the sorted member list).  Padding rows stay zero.  The sums run in
// the scalings' type S: FP64 for FP64 blocks; FP32 (the graph's FP32 copies of s and t)
// for BF16 blocks, whose 8-bit mantissa FP32 sums of ~20 terms carry exactly -- FP64
// arithmetic and conversions kept the slow FP64 pipe 73% busy.
// ---------------------------------------------------------------------------
template <class TA, class S>
__global__ void k_assemble(Blocks B, int64_t rows_tot, const int64_t* __restrict__ csr_ptr,
                           const int32_t* __restrict__ csr_idx, const int64_t* __restrict__ csc_ptr,
                           const int32_t* __restrict__ csc_idx, const S* __restrict__ s,
                           const S* __restrict__ t, TA* __restrict__ A) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t r = warp; r < rows_tot; r += nwarps) {
    const int b = find_block(B.arow, B.nb, r);
    const int64_t i = r - B.arow[b];
    const int bs = B.rows[b];
    const int64_t width = ((int64_t)bs + 63) / 64 * 64;
    TA* row = A + r * B.ldA;
    // zero the used width with 16-byte stores (rows start on 128-byte boundaries and
    // the width is a multiple of 64 elements)
    {
      constexpr int PER = 16 / (int)sizeof(TA);
      uint4* row4 = reinterpret_cast<uint4*>(row);
      for (int64_t j = lane; j < width / PER; j += 32) row4[j] = make_uint4(0u, 0u, 0u, 0u);
    }
    if (i >= bs) continue;
    __syncwarp();
    const int64_t v0 = B.v0[b];
    const int64_t u = v0 + i;
    const S su = s[u];
    const int64_t beg = csr_ptr[u], end = csr_ptr[u + 1];
    S d = S(0);
    for (int64_t q = beg + lane; q < end; q += 32) d += t[csr_idx[q]];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
    if (lane == 0) row[i] = from_acc<TA>(su * su * d);
    __syncwarp();
    // off-diagonal terms: the lanes take 32 of u's hyperedges at a time and each finds
    // the members of its hyperedge inside [v0, v0 + bs) by two binary searches over
    // the sorted member list (independent searches, so their latencies overlap); the
    // warp then adds the hyperedges that hold another block member, in CSR order.
    for (int64_t q0 = beg; q0 < end; q0 += 32) {
      const int64_t q = q0 + lane;
      int64_t lo = 0, hi = 0;
      int32_t e = 0;
      if (q < end) {
        e = csr_idx[q];
        int64_t a = csc_ptr[e], z = csc_ptr[e + 1];
        const int64_t me = z;
        while (a < z) {
          const int64_t mid = (a + z) >> 1;
          if (csc_idx[mid] < v0) a = mid + 1; else z = mid;
        }
        lo = a;
        z = me;
        while (a < z) {
          const int64_t mid = (a + z) >> 1;
          if (csc_idx[mid] < v0 + bs) a = mid + 1; else z = mid;
        }
        hi = a;
      }
      unsigned todo = __ballot_sync(0xffffffffu, hi - lo > 1);
      while (todo) {
        const int src = __ffs(todo) - 1;
        todo &= todo - 1;
        const int64_t l2 = __shfl_sync(0xffffffffu, lo, src);
        const int64_t h2 = __shfl_sync(0xffffffffu, hi, src);
        const int32_t e2 = __shfl_sync(0xffffffffu, e, src);
        const S f = su * t[e2];
        for (int64_t p = l2 + lane; p < h2; p += 32) {
          const int32_t v = csc_idx[p];
          if (v != u) {
            const int64_t j = v - v0;
            row[j] = from_acc<TA>(to_acc<TA, S>(row[j]) + f * s[v]);
          }
        }
        __syncwarp();
      }
    }
  }
}

// ---------------------------------------------------------------------------
// The same blocks from a kept pattern.  Which members of which hyperedge fall inside a
// block depends on the incidence and the block layout, not on w, so a plan finds them
// once: per storage row, the segments (e, lo, hi) of the row vertex's hyperedges with
// another member in the block, [lo, hi) the block's part of e's sorted member list.  A
// build then clears only those entries (the rest of the storage is zero since the plan
// was created) and adds the terms in the same order as k_assemble, so the blocks come
// out identical, without zeroing the padded rows or searching the member lists.
// ---------------------------------------------------------------------------
struct Segment {
  int32_t e, lo, hi;
};

// Segments of storage row r (CSR order of the row vertex's hyperedges), counted
// (out == nullptr) or written to out; one warp per row.
__device__ __forceinline__ unsigned row_segments(const Blocks& B, int64_t r, const int64_t* __restrict__ csr_ptr,
                                                 const int32_t* __restrict__ csr_idx,
                                                 const int64_t* __restrict__ csc_ptr,
                                                 const int32_t* __restrict__ csc_idx, Segment* out) {
  const int lane = threadIdx.x & 31;
  const int b = find_block(B.arow, B.nb, r);
  const int64_t i = r - B.arow[b];
  const int bs = B.rows[b];
  if (i >= bs) return 0;
  const int64_t v0 = B.v0[b], u = v0 + i;
  const int64_t beg = csr_ptr[u], end = csr_ptr[u + 1];
  unsigned n = 0;
  for (int64_t q0 = beg; q0 < end; q0 += 32) {
    const int64_t q = q0 + lane;
    int64_t lo = 0, hi = 0;
    int32_t e = 0;
    if (q < end) {
      e = csr_idx[q];
      int64_t a = csc_ptr[e], z = csc_ptr[e + 1];
      const int64_t me = z;
      while (a < z) {
        const int64_t mid = (a + z) >> 1;
        if (csc_idx[mid] < v0) a = mid + 1; else z = mid;
      }
      lo = a;
      z = me;
      while (a < z) {
        const int64_t mid = (a + z) >> 1;
        if (csc_idx[mid] < v0 + bs) a = mid + 1; else z = mid;
      }
      hi = a;
    }
    const bool keep = hi - lo > 1;
    const unsigned mask = __ballot_sync(0xffffffffu, keep);
    if (out && keep) {
      const unsigned pos = n + __popc(mask & ((1u << lane) - 1u));
      out[pos] = Segment{e, (int32_t)lo, (int32_t)hi};
    }
    n += __popc(mask);
  }
  return n;
}

static __global__ void k_segment_count(Blocks B, int64_t rows_tot, const int64_t* __restrict__ csr_ptr,
                                const int32_t* __restrict__ csr_idx, const int64_t* __restrict__ csc_ptr,
                                const int32_t* __restrict__ csc_idx, unsigned* __restrict__ count) {
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t r = warp; r < rows_tot; r += nwarps) {
    const unsigned n = row_segments(B, r, csr_ptr, csr_idx, csc_ptr, csc_idx, nullptr);
    if ((threadIdx.x & 31) == 0) count[r] = n;
  }
}

static __global__ void k_segment_fill(Blocks B, int64_t rows_tot, const int64_t* __restrict__ csr_ptr,
                               const int32_t* __restrict__ csr_idx, const int64_t* __restrict__ csc_ptr,
                               const int32_t* __restrict__ csc_idx, const int64_t* __restrict__ seg_ptr,
                               Segment* __restrict__ seg) {
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t r = warp; r < rows_tot; r += nwarps)
    row_segments(B, r, csr_ptr, csr_idx, csc_ptr, csc_idx, seg + seg_ptr[r]);
}

template <class TA, class S>
__global__ void k_assemble_kept(Blocks B, int64_t rows_tot, const int64_t* __restrict__ csr_ptr,
                                const int32_t* __restrict__ csr_idx, const int32_t* __restrict__ csc_idx,
                                const int64_t* __restrict__ seg_ptr, const Segment* __restrict__ seg,
                                const S* __restrict__ s, const S* __restrict__ t, TA* __restrict__ A) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t r = warp; r < rows_tot; r += nwarps) {
    const int b = find_block(B.arow, B.nb, r);
    const int64_t i = r - B.arow[b];
    if (i >= B.rows[b]) continue;
    TA* row = A + r * B.ldA;
    const int64_t v0 = B.v0[b];
    const int64_t u = v0 + i;
    const int64_t k0 = seg_ptr[r], k1 = seg_ptr[r + 1];
    // clear the previous build's off-diagonal entries
    for (int64_t k = k0; k < k1; ++k) {
      const Segment sg = seg[k];
      for (int64_t p = sg.lo + lane; p < sg.hi; p += 32) {
        const int32_t v = csc_idx[p];
        if (v != u) row[v - v0] = from_acc<TA>(S(0));
      }
    }
    const S su = s[u];
    S d = S(0);
    for (int64_t q = csr_ptr[u] + lane, end = csr_ptr[u + 1]; q < end; q += 32) d += t[csr_idx[q]];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
    __syncwarp();
    if (lane == 0) row[i] = from_acc<TA>(su * su * d);
    __syncwarp();
    for (int64_t k = k0; k < k1; ++k) {
      const Segment sg = seg[k];
      const S f = su * t[sg.e];
      for (int64_t p = sg.lo + lane; p < sg.hi; p += 32) {
        const int32_t v = csc_idx[p];
        if (v != u) {
          const int64_t j = v - v0;
          row[j] = from_acc<TA>(to_acc<TA, S>(row[j]) + f * s[v]);
        }
      }
      __syncwarp();
    }
  }
}

// ---------------------------------------------------------------------------
// Sparse route for blocks that hold few of Theta's entries: Theta_bb S straight from
// the incidence lists, without dense blocks.
//   Theta_bb[u, u] = s_u^2 sum_{e ni u} t_e
//   Theta_bb[u, v] = s_u s_v sum_{e ni u, v} t_e      (u != v, both in block b)
// The members of a hyperedge that fall in block b form one run of its sorted member
// list, found by two binary searches (as in the assembly above).
// ---------------------------------------------------------------------------

// Run [lo, hi) of hyperedge e's sorted members inside [v0, v1).
__device__ __forceinline__ void member_run(const int64_t* __restrict__ csc_ptr, const int32_t* __restrict__ csc_idx,
                                           int32_t e, int64_t v0, int64_t v1, int64_t* lo, int64_t* hi) {
  int64_t a = csc_ptr[e], z = csc_ptr[e + 1];
  const int64_t me = z;
  while (a < z) {
    const int64_t mid = (a + z) >> 1;
    if (csc_idx[mid] < v0) a = mid + 1; else z = mid;
  }
  *lo = a;
  z = me;
  while (a < z) {
    const int64_t mid = (a + z) >> 1;
    if (csc_idx[mid] < v1) a = mid + 1; else z = mid;
  }
  *hi = a;
}

// Entries of all diagonal blocks (with one per hyperedge for repeated pairs), summed
// into *count: for every vertex u, the length of its block's run in each of its
// hyperedges.  bp: the nb + 1 block boundaries.
static __global__ void k_block_nnz(int64_t n, int nb, const int64_t* __restrict__ bp, const int64_t* __restrict__ csr_ptr,
                            const int32_t* __restrict__ csr_idx, const int64_t* __restrict__ csc_ptr,
                            const int32_t* __restrict__ csc_idx, unsigned long long* __restrict__ count) {
  unsigned long long local = 0;
  for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < n; u += (int64_t)gridDim.x * blockDim.x) {
    const int b = find_block(bp, nb, u);
    for (int64_t q = csr_ptr[u]; q < csr_ptr[u + 1]; ++q) {
      int64_t lo, hi;
      member_run(csc_ptr, csc_idx, csr_idx[q], bp[b], bp[b + 1], &lo, &hi);
      local += (unsigned long long)(hi - lo);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) local += __shfl_xor_sync(0xffffffffu, local, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(count, local);
}

// D = Theta_bb S for every block; S and D in the dense route's row layout (block b's
// row i at arow[b] + i, padding rows zero), LP FP32 columns.  One warp per row:
// lanes split the row's columns; for the off-diagonal terms the lanes take 32 of u's
// hyperedges at a time, search their runs, and the warp adds the rows of the runs
// longer than one, hyperedge by hyperedge in CSR order (a fixed summation order).
template <int LP>
__global__ void __launch_bounds__(256)
k_block_spmm(Blocks B, int64_t rows_tot, const int64_t* __restrict__ csr_ptr, const int32_t* __restrict__ csr_idx,
             const int64_t* __restrict__ csc_ptr, const int32_t* __restrict__ csc_idx, const double* __restrict__ s,
             const double* __restrict__ t, const float* __restrict__ S, float* __restrict__ D) {
  constexpr int PL = (LP + 31) / 32;
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t r = warp; r < rows_tot; r += nwarps) {
    const int b = find_block(B.arow, B.nb, r);
    const int64_t i = r - B.arow[b];
    float* drow = D + r * LP;
    if (i >= B.rows[b]) {
#pragma unroll
      for (int p = 0; p < PL; ++p)
        if (lane + 32 * p < LP) drow[lane + 32 * p] = 0.f;
      continue;
    }
    const int64_t v0 = B.v0[b], v1 = v0 + B.rows[b];
    const int64_t u = v0 + i;
    const double su = s[u];
    const int64_t beg = csr_ptr[u], end = csr_ptr[u + 1];
    double d = 0.0;
    for (int64_t q = beg + lane; q < end; q += 32) d += t[csr_idx[q]];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
    const float fd = (float)(su * su * d);
    const float* srow = S + r * LP;
    float acc[PL];
#pragma unroll
    for (int p = 0; p < PL; ++p) acc[p] = lane + 32 * p < LP ? fd * srow[lane + 32 * p] : 0.f;
    for (int64_t q0 = beg; q0 < end; q0 += 32) {
      const int64_t q = q0 + lane;
      int64_t lo = 0, hi = 0;
      int32_t e = 0;
      if (q < end) {
        e = csr_idx[q];
        member_run(csc_ptr, csc_idx, e, v0, v1, &lo, &hi);
      }
      unsigned todo = __ballot_sync(0xffffffffu, hi - lo > 1);
      while (todo) {
        const int src = __ffs(todo) - 1;
        todo &= todo - 1;
        const int64_t l2 = __shfl_sync(0xffffffffu, lo, src);
        const int64_t h2 = __shfl_sync(0xffffffffu, hi, src);
        const int32_t e2 = __shfl_sync(0xffffffffu, e, src);
        const double f = su * t[e2];
        for (int64_t p2 = l2; p2 < h2; ++p2) {
          const int32_t v = csc_idx[p2];
          if (v == u) continue;
          const float fv = (float)(f * s[v]);
          const float* vrow = S + (B.arow[b] + (v - v0)) * LP;
#pragma unroll
          for (int p = 0; p < PL; ++p)
            if (lane + 32 * p < LP) acc[p] = fmaf(fv, vrow[lane + 32 * p], acc[p]);
        }
      }
    }
#pragma unroll
    for (int p = 0; p < PL; ++p)
      if (lane + 32 * p < LP) drow[lane + 32 * p] = acc[p];
  }
}

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon et al., SC 2011) and the Gaussian test matrix Omega.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void philox4x32_10(uint32_t (&c)[4], uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const uint32_t lo0 = 0xD2511F53u * c[0], hi0 = __umulhi(0xD2511F53u, c[0]);
    const uint32_t lo1 = 0xCD9E8D57u * c[2], hi1 = __umulhi(0xCD9E8D57u, c[2]);
    const uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0;
    c[1] = lo1;
    c[2] = n2;
    c[3] = lo0;
  }
}

__device__ __forceinline__ double unit53(uint32_t a, uint32_t b) {
  return ((double)(a >> 5) * 67108864.0 + (double)(b >> 6) + 0.5) * 0x1p-53;
}

// Omega[g, 2p] and Omega[g, 2p+1] for global row g from one Philox draw (Box-Muller).
// FP64 storage evaluates the transform in FP64; BF16 storage in FP32 (the result is
// rounded to BF16 anyway).
template <class TB>
__device__ __forceinline__ void omega_pair(int64_t g, int p, uint64_t seed, double* z0, double* z1) {
  uint32_t c[4] = {(uint32_t)g, (uint32_t)p, OMEGA_STREAM, 0u};
  philox4x32_10(c, (uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32));
  if constexpr (sizeof(TB) == 8) {
    const double u1 = unit53(c[0], c[1]);
    const double u2 = unit53(c[2], c[3]);
    const double r = sqrt(-2.0 * log(u1));
    double sn, cs;
    sincos(2.0 * 3.14159265358979323846 * u2, &sn, &cs);
    *z0 = r * cs;
    *z1 = r * sn;
  } else {
    const float u1 = (float)unit53(c[0], c[1]);
    const float u2 = (float)unit53(c[2], c[3]);
    const float r = sqrtf(-2.0f * logf(u1));
    float sn, cs;
    sincospif(2.0f * u2, &sn, &cs);
    *z0 = (double)(r * cs);
    *z1 = (double)(r * sn);
  }
}

// Transposed basis St (lpad x Ktot): St[j, koff_b + i] = Omega[v0_b + i, j] for j < lb_b,
// i < rows_b; every other entry (columns j >= lb, padding i) is zero.  One thread per
// (column pair, basis column).
template <class TB>
__global__ void k_omega(Blocks B, uint64_t seed_arg, const uint64_t* __restrict__ seed_dev, TB* __restrict__ St) {
  const uint64_t seed = seed_dev ? *seed_dev : seed_arg;
  const int64_t total = (int64_t)(B.lpad / 2) * B.Ktot;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
    const int p = (int)(q / B.Ktot);
    const int64_t col = q % B.Ktot;
    const int b = find_block(B.koff, B.nb, col);
    const int64_t i = col - B.koff[b];
    double z0 = 0.0, z1 = 0.0;
    if (i < B.rows[b] && 2 * p < B.lb[b]) omega_pair<TB>(B.v0[b] + i, p, seed, &z0, &z1);
    St[(int64_t)(2 * p) * B.Ktot + col] = from_double<TB>(z0);
    St[(int64_t)(2 * p + 1) * B.Ktot + col] = from_double<TB>(2 * p + 1 < B.lb[b] ? z1 : 0.0);
  }
}

// Omega in the row layout of the sparse route: S[arow_b + i, c] (FP32, LP columns) for
// the same Gaussian numbers as k_omega (zero beyond l_b and on padding rows).
template <int LP>
__global__ void k_omega_rows(Blocks B, int64_t rows_tot, uint64_t seed_arg, const uint64_t* __restrict__ seed_dev,
                             float* __restrict__ S) {
  const uint64_t seed = seed_dev ? *seed_dev : seed_arg;
  const int64_t total = rows_tot * (LP / 2);
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = q / (LP / 2);
    const int p = (int)(q % (LP / 2));
    const int b = find_block(B.arow, B.nb, r);
    const int64_t i = r - B.arow[b];
    double z0 = 0.0, z1 = 0.0;
    if (i < B.rows[b] && 2 * p < B.lb[b]) omega_pair<float>(B.v0[b] + i, p, seed, &z0, &z1);
    S[r * LP + 2 * p] = (float)z0;
    S[r * LP + 2 * p + 1] = 2 * p + 1 < B.lb[b] ? (float)z1 : 0.f;
  }
}

// ---------------------------------------------------------------------------
// FP64 grouped GEMM on CUDA cores (checking path): D[r, :] = A[r, 0:K] St[:, koff:koff+K]^T
// ---------------------------------------------------------------------------
template <int LPAD>
__global__ void __launch_bounds__(256)
k_block_gemm_f64(Blocks B, const int32_t* __restrict__ unit_block, const int32_t* __restrict__ unit_tile,
                 int nunits, const double* __restrict__ A, const double* __restrict__ St, double* __restrict__ D) {
  constexpr int TM = 128, TK = 16, CPT = LPAD / 16;
  __shared__ double sa[TM][TK + 1];
  __shared__ double sb[LPAD][TK + 1];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;  // 16 x 16 threads; thread: 8 rows x CPT cols
  for (int u = blockIdx.x; u < nunits; u += gridDim.x) {
    const int b = unit_block[u];
    const int K = B.rows[b];
    const int64_t r0 = B.arow[b] + (int64_t)unit_tile[u] * TM;
    const int64_t k0 = B.koff[b];
    double acc[8][CPT];
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
      for (int c = 0; c < CPT; ++c) acc[a][c] = 0.0;
    for (int kt = 0; kt < K; kt += TK) {
      for (int q = threadIdx.x; q < TM * TK; q += blockDim.x) {
        const int rr = q / TK, kk = q % TK;
        sa[rr][kk] = (kt + kk < K) ? A[(r0 + rr) * B.ldA + kt + kk] : 0.0;
      }
      for (int q = threadIdx.x; q < LPAD * TK; q += blockDim.x) {
        const int jj = q / TK, kk = q % TK;
        sb[jj][kk] = (kt + kk < K) ? St[(int64_t)jj * B.Ktot + k0 + kt + kk] : 0.0;
      }
      __syncthreads();
#pragma unroll 4
      for (int kk = 0; kk < TK; ++kk) {
        double bv[CPT];
#pragma unroll
        for (int c = 0; c < CPT; ++c) bv[c] = sb[tx + 16 * c][kk];
#pragma unroll
        for (int a = 0; a < 8; ++a) {
          const double av = sa[ty + 16 * a][kk];
#pragma unroll
          for (int c = 0; c < CPT; ++c) acc[a][c] = fma(av, bv[c], acc[a][c]);
        }
      }
      __syncthreads();
    }
    const int rows = B.rows[b];
#pragma unroll
    for (int a = 0; a < 8; ++a) {
      const int rr = ty + 16 * a;
      if ((int64_t)unit_tile[u] * TM + rr < rows)
#pragma unroll
        for (int c = 0; c < CPT; ++c) D[(r0 + rr) * LPAD + tx + 16 * c] = acc[a][c];
    }
  }
}

// ---------------------------------------------------------------------------
// Per-block cross Gram G_b = X_b^T Y_b (lpad x lpad, FP64) of two row panels with
// row stride lpad.  Each CTA takes one block and one range of GRAM_SPLIT rows and
// writes a partial Gram; k_gram_reduce adds a block's partials in range order.  A
// thread owns a TxT tile of the Gram (T = lpad/16): per row it reads T values of each
// panel from shared memory and does T*T FMAs in the panel type; tile sums over 64 rows
// are added into accumulators of ~FP64 accuracy: FP64 for FP64 panels, an unevaluated
// FP32 pair (TwoSum, Knuth) for FP32 panels -- FP64 adds and conversions would keep
// the slow FP64 pipe the bound.
// ---------------------------------------------------------------------------
constexpr int GRAM_SPLIT = 1024;

template <class T> struct GramAcc {
  double s = 0.0;
  __device__ __forceinline__ void add(T x) { s += (double)x; }
  __device__ __forceinline__ double value() const { return s; }
};
template <> struct GramAcc<float> {
  float hi = 0.f, lo = 0.f;
  __device__ __forceinline__ void add(float x) {
    const float s = __fadd_rn(hi, x);
    const float bb = __fsub_rn(s, hi);
    const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(x, bb));
    hi = s;
    lo = __fadd_rn(lo, e);
  }
  __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

// SYM (X == Y): only the 16 x 16 tiles on and above the diagonal are formed (15 of 25 for
// LPAD = 80); k_gram_reduce mirrors the others.  Products commute, so the mirrored
// entries are the ones a full pass would form.
template <class T, int LPAD, bool SYM>
__global__ void __launch_bounds__(256) k_gram_part(Blocks B, int max_splits, const T* __restrict__ X,
                                                    const T* __restrict__ Y, double* __restrict__ Gpart) {
  constexpr int TR = sizeof(T) == 8 ? 32 : 64;
  constexpr int TT = LPAD / 16;
  __shared__ T sx[TR][LPAD];
  __shared__ T sy[TR][LPAD];
  const int b = blockIdx.x / max_splits, split = blockIdx.x % max_splits;
  const int rows = B.rows[b];
  const int r_begin = split * GRAM_SPLIT;
  double* out = Gpart + (int64_t)blockIdx.x * LPAD * LPAD;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  if (r_begin >= rows) return;
  const int r_end = rows < r_begin + GRAM_SPLIT ? rows : r_begin + GRAM_SPLIT;
  const int64_t r0 = B.arow[b];
  GramAcc<T> acc[TT][TT];
  for (int t0 = r_begin; t0 < r_end; t0 += TR) {
    const int nr = r_end - t0 < TR ? r_end - t0 : TR;
    for (int q = threadIdx.x; q < TR * LPAD; q += blockDim.x) {
      const int rr = q / LPAD, jj = q % LPAD;
      sx[rr][jj] = rr < nr ? X[(r0 + t0 + rr) * LPAD + jj] : T(0);
      sy[rr][jj] = rr < nr ? Y[(r0 + t0 + rr) * LPAD + jj] : T(0);
    }
    __syncthreads();
    T part[TT][TT];
#pragma unroll
    for (int a = 0; a < TT; ++a)
#pragma unroll
      for (int c = 0; c < TT; ++c) part[a][c] = T(0);
#pragma unroll 4
    for (int rr = 0; rr < TR; ++rr) {
      T xv[TT], yv[TT];
#pragma unroll
      for (int a = 0; a < TT; ++a) xv[a] = sx[rr][ty + 16 * a];
#pragma unroll
      for (int c = 0; c < TT; ++c) yv[c] = sy[rr][tx + 16 * c];
#pragma unroll
      for (int a = 0; a < TT; ++a)
#pragma unroll
        for (int c = 0; c < TT; ++c)
          if (!SYM || a <= c) part[a][c] = fma(xv[a], yv[c], part[a][c]);
    }
#pragma unroll
    for (int a = 0; a < TT; ++a)
#pragma unroll
      for (int c = 0; c < TT; ++c)
        if (!SYM || a <= c) acc[a][c].add(part[a][c]);
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < TT; ++a)
#pragma unroll
    for (int c = 0; c < TT; ++c)
      if (!SYM || a <= c) out[(ty + 16 * a) * LPAD + tx + 16 * c] = acc[a][c].value();
}

// G[b] = sum of the block's partial Grams in range order (sym: the entries below the
// diagonal's 16 x 16 tiles from their mirror images)
template <int LPAD>
__global__ void k_gram_reduce(Blocks B, int max_splits, const double* __restrict__ Gpart, double* __restrict__ G,
                              bool sym) {
  const int b = blockIdx.x;
  const int nsplit = (B.rows[b] + GRAM_SPLIT - 1) / GRAM_SPLIT;
  for (int q = threadIdx.x; q < LPAD * LPAD; q += blockDim.x) {
    const int i = q / LPAD, j = q % LPAD;
    const int src = sym && (i >> 4) > (j >> 4) ? j * LPAD + i : q;
    double s = 0.0;
    for (int sp = 0; sp < nsplit; ++sp) s += Gpart[((int64_t)b * max_splits + sp) * LPAD * LPAD + src];
    G[(int64_t)b * LPAD * LPAD + q] = s;
  }
}

// ---------------------------------------------------------------------------
// Per-block Cholesky G = L L^T of the leading lb x lb Gram (symmetrised, with a
// relative diagonal shift `shift` * trace / lb), then Rinv = L^-T (upper triangular,
// so Q = Y Rinv has orthonormal columns).  The factorisation is rank revealing: a
// pivot below `drop` * max diag(G) marks a direction Y does not span (a rank-deficient
// block, e.g. one whose vertices lost all hyperedge weight); its row and column of
// Rinv are zero, so the matching basis column is zero and contributes nothing later.
// A block whose Gram trace is 0 or not finite gets Rinv = 0.  One CTA per block.
// ---------------------------------------------------------------------------
template <int LPAD>
__global__ void __launch_bounds__(256) k_chol_inv(Blocks B, const double* __restrict__ G, double shift, double drop,
                                                   double* __restrict__ Rinv, int32_t* __restrict__ fail) {
  // row stride LS = LPAD + 1 (odd): a warp walking down a column of doubles touches
  // distinct banks
  constexpr int LS = LPAD + 1;
  extern __shared__ double sm[];
  double* L = sm;                 // LPAD x LS
  double* X = sm + LPAD * LS;     // LPAD x LS
  __shared__ double s_trace, s_dmax;
  __shared__ int dead[LPAD];
  __shared__ int s_ndead;
  const int b = blockIdx.x;
  const int lb = B.lb[b];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr int NW = 256 / 32;
  const double* Gb = G + (int64_t)b * LPAD * LPAD;
  for (int i = warp; i < LPAD; i += NW)
    for (int j = lane; j < LPAD; j += 32) {
      L[i * LS + j] = (i < lb && j < lb) ? 0.5 * (Gb[i * LPAD + j] + Gb[j * LPAD + i]) : 0.0;
      X[i * LS + j] = 0.0;
    }
  for (int j = threadIdx.x; j < LPAD; j += blockDim.x) dead[j] = 0;
  __syncthreads();
  if (threadIdx.x == 0) {
    double tr = 0.0, dm = 0.0;
    for (int i = 0; i < lb; ++i) {
      tr += L[i * LS + i];
      dm = fmax(dm, L[i * LS + i]);
    }
    s_trace = tr;
    s_dmax = dm;
    s_ndead = 0;
  }
  __syncthreads();
  const double tr = s_trace;
  double* Rb = Rinv + (int64_t)b * LPAD * LPAD;
  if (!(tr > 0.0) || !isfinite(tr)) {
    for (int q = threadIdx.x; q < LPAD * LPAD; q += blockDim.x) Rb[q] = 0.0;
    return;
  }
  const double sigma = shift * tr / lb;
  const double floor_pivot = drop * s_dmax;
  for (int i = threadIdx.x; i < lb; i += blockDim.x) L[i * LS + i] += sigma;
  __syncthreads();
  // right-looking Cholesky with dropped pivots
  for (int j = 0; j < lb; ++j) {
    if (threadIdx.x == 0) {
      const double d = L[j * LS + j];
      if (!(d > floor_pivot) || !isfinite(d)) {
        dead[j] = 1;
        s_ndead += 1;
        L[j * LS + j] = 1.0;
      } else {
        L[j * LS + j] = sqrt(d);
      }
    }
    __syncthreads();
    const double dj = L[j * LS + j];
    const bool dj_dead = dead[j] != 0;
    for (int i = j + 1 + threadIdx.x; i < lb; i += blockDim.x)
      L[i * LS + j] = dj_dead ? 0.0 : L[i * LS + j] / dj;
    __syncthreads();
    // trailing update of the lower triangle: a warp per row, lanes along it
    for (int i = j + 1 + warp; i < lb; i += NW) {
      const double lij = L[i * LS + j];
      for (int k = j + 1 + lane; k <= i; k += 32) L[i * LS + k] -= lij * L[k * LS + j];
    }
    __syncthreads();
  }
  // X = L^-1 (lower), one column per thread: forward substitution
  for (int c = threadIdx.x; c < lb; c += blockDim.x) {
    X[c * LS + c] = 1.0 / L[c * LS + c];
    for (int i = c + 1; i < lb; ++i) {
      double sacc = 0.0;
      for (int k = c; k < i; ++k) sacc += L[i * LS + k] * X[k * LS + c];
      X[i * LS + c] = -sacc / L[i * LS + i];
    }
  }
  __syncthreads();
  // Rinv = X^T (upper); dead directions get a zero row and column
  for (int i = warp; i < LPAD; i += NW)
    for (int j = lane; j < LPAD; j += 32)
      Rb[i * LPAD + j] = (i < lb && j < lb && !dead[i] && !dead[j]) ? X[j * LS + i] : 0.0;
  if (threadIdx.x == 0 && s_ndead) atomicAdd(fail, 1);
}

// Q = Y Rinv on one 128-row tile of a block per CTA iteration.  A thread owns 8 rows x
// LPAD/16 columns of the tile (rows tr + 16a, columns tc + 16c) and accumulates over
// the block's lb basis columns from shared memory; Rinv is upper triangular (its
// lower part is stored as zeros), so the sum over all i equals the sum over i <= j in
// the same order.  The tile is staged with a row stride of LPAD + 1 words, which keeps
// both the row products and the transposed St write free of bank conflicts.  Writes
// the row panel Qf (row stride lpad; in place is fine, each tile reads its rows
// before writing them) and, if St is given, the transposed basis St[j, koff + i].
template <class T, class TB, int LPAD>
__global__ void __launch_bounds__(256) k_apply_rinv(Blocks B, const int32_t* __restrict__ unit_block,
                                                     const int32_t* __restrict__ unit_tile, int nunits,
                                                     const T* Y, const double* __restrict__ Rinv, T* Qf,
                                                     TB* __restrict__ St) {
  constexpr int TR = 128, LS = LPAD + 1, CT = LPAD / 16, RT = TR / 16;
  extern __shared__ __align__(16) uint8_t smraw[];
  T* sr = reinterpret_cast<T*>(smraw);  // LPAD x LPAD
  T* sy = sr + LPAD * LPAD;              // TR x LS
  const int tc = threadIdx.x & 15, tr = threadIdx.x >> 4;
  for (int u = blockIdx.x; u < nunits; u += gridDim.x) {
    const int b = unit_block[u];
    const int rows = B.rows[b];
    const int lb = B.lb[b];
    const int i0 = unit_tile[u] * TR;
    const int nr = rows - i0 < TR ? rows - i0 : TR;
    const int64_t r0 = B.arow[b] + i0;
    for (int q = threadIdx.x; q < LPAD * LPAD; q += blockDim.x) sr[q] = (T)Rinv[(int64_t)b * LPAD * LPAD + q];
    for (int q = threadIdx.x; q < TR * LPAD; q += blockDim.x) {
      const int rr = q / LPAD, jj = q % LPAD;
      sy[rr * LS + jj] = rr < nr ? Y[(r0 + rr) * LPAD + jj] : T(0);
    }
    __syncthreads();
    T acc[RT][CT];
#pragma unroll
    for (int a = 0; a < RT; ++a)
#pragma unroll
      for (int c = 0; c < CT; ++c) acc[a][c] = T(0);
#pragma unroll 2
    for (int i = 0; i < lb; ++i) {
      T yv[RT], rv[CT];
#pragma unroll
      for (int a = 0; a < RT; ++a) yv[a] = sy[(tr + 16 * a) * LS + i];
#pragma unroll
      for (int c = 0; c < CT; ++c) rv[c] = sr[i * LPAD + tc + 16 * c];
#pragma unroll
      for (int a = 0; a < RT; ++a)
#pragma unroll
        for (int c = 0; c < CT; ++c) acc[a][c] = fma(yv[a], rv[c], acc[a][c]);
    }
    __syncthreads();  // every read of the input tile is done
#pragma unroll
    for (int a = 0; a < RT; ++a) {
      const int row = tr + 16 * a;
#pragma unroll
      for (int c = 0; c < CT; ++c) {
        const int col = tc + 16 * c;
        sy[row * LS + col] = acc[a][c];
        if (row < nr) Qf[(r0 + row) * LPAD + col] = acc[a][c];
      }
    }
    __syncthreads();
    if (St) {
      const int64_t kb0 = B.koff[b] + i0;
      for (int q = threadIdx.x; q < LPAD * TR; q += blockDim.x) {
        const int j = q / TR, rr = q % TR;
        if (rr < nr) St[(int64_t)j * B.Ktot + kb0 + rr] = basis_from<TB, T>(sy[rr * LS + j]);
      }
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Symmetric eigendecomposition of T_b (lb x lb) by cyclic Jacobi with a round-robin
// (tournament) ordering of disjoint pairs, in arithmetic type TJ (FP64 for the FP64
// route; FP32 for the BF16 route, whose products are BF16-accurate anyway).  Sweeps
// stop once the off-diagonal mass is below tol2 times the total.  Writes the
// eigenvalues in descending order and the matching eigenvectors (columns of V,
// LPAD x LPAD, FP64).
// ---------------------------------------------------------------------------
template <class TJ, int LPAD>
__global__ void __launch_bounds__(256) k_jacobi(Blocks B, const double* __restrict__ Tm, double* __restrict__ V,
                                                 double* __restrict__ evals, int max_sweeps, double tol2) {
  // row stride LS = LPAD + 1 (odd): a warp walking down a column touches 32 banks
  constexpr int LS = LPAD + 1;
  extern __shared__ __align__(16) uint8_t jsm_raw[];
  TJ* A = reinterpret_cast<TJ*>(jsm_raw);   // LPAD x LS
  TJ* W = A + LPAD * LS;                     // eigenvectors, LPAD x LS
  __shared__ TJ cs[LPAD / 2], sn[LPAD / 2];
  __shared__ int pp[LPAD / 2], qq[LPAD / 2];
  __shared__ double off_s, tot_s;
  __shared__ int order[LPAD];
  const int b = blockIdx.x;
  const int lb = B.lb[b];
  const int n = (lb + 1) & ~1;  // even, a dummy index when lb is odd
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr int NW = 256 / 32;
  const double* Tb = Tm + (int64_t)b * LPAD * LPAD;
  for (int i = warp; i < LPAD; i += NW)
    for (int j = lane; j < LPAD; j += 32) {
      A[i * LS + j] = (i < lb && j < lb) ? (TJ)(0.5 * (Tb[i * LPAD + j] + Tb[j * LPAD + i])) : TJ(0);
      W[i * LS + j] = (i == j) ? TJ(1) : TJ(0);
    }
  __syncthreads();
  __shared__ double red_off[NW], red_tot[NW];
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    {
      double off = 0.0, tot = 0.0;
      for (int i = warp; i < lb; i += NW)
        for (int j = lane; j < lb; j += 32) {
          const double a = (double)A[i * LS + j];
          tot += a * a;
          if (i != j) off += a * a;
        }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        off += __shfl_xor_sync(0xffffffffu, off, o);
        tot += __shfl_xor_sync(0xffffffffu, tot, o);
      }
      if (lane == 0) {
        red_off[warp] = off;
        red_tot[warp] = tot;
      }
      __syncthreads();
      if (threadIdx.x == 0) {
        double a = 0.0, t = 0.0;
        for (int w = 0; w < NW; ++w) {
          a += red_off[w];
          t += red_tot[w];
        }
        off_s = a;
        tot_s = t;
      }
    }
    __syncthreads();
    if (!(off_s > tol2 * tot_s) || lb < 2) break;
    for (int round = 0; round < n - 1; ++round) {
      // tournament pairs: position 0 fixed, others rotate
      for (int p = threadIdx.x; p < n / 2; p += blockDim.x) {
        int a = p == 0 ? 0 : 1 + (p - 1 + round) % (n - 1);
        int z = 1 + (n - 2 - p + round) % (n - 1);
        if (a > z) {
          const int tmp = a;
          a = z;
          z = tmp;
        }
        pp[p] = a;
        qq[p] = z;
        TJ c = TJ(1), s = TJ(0);
        if (z < lb) {
          const TJ apq = A[a * LS + z];
          if (apq != TJ(0)) {
            const TJ app = A[a * LS + a], aqq = A[z * LS + z];
            const TJ theta = (aqq - app) / (TJ(2) * apq);
            const TJ tt = (theta >= TJ(0) ? TJ(1) : TJ(-1)) / (fabs(theta) + sqrt(theta * theta + TJ(1)));
            c = TJ(1) / sqrt(tt * tt + TJ(1));
            s = tt * c;
          }
        }
        cs[p] = c;
        sn[p] = s;
      }
      __syncthreads();
      // rows: A <- J^T A (a warp per pair, lanes along the row)
      for (int p = warp; p < n / 2; p += NW) {
        const int a = pp[p], z = qq[p];
        if (z >= lb) continue;
        const TJ c = cs[p], s = sn[p];
        for (int col = lane; col < lb; col += 32) {
          const TJ x = A[a * LS + col], y = A[z * LS + col];
          A[a * LS + col] = c * x - s * y;
          A[z * LS + col] = s * x + c * y;
        }
      }
      __syncthreads();
      // columns: A <- A J, V <- V J (a warp per pair, lanes down the column)
      for (int p = warp; p < n / 2; p += NW) {
        const int a = pp[p], z = qq[p];
        if (z >= lb) continue;
        const TJ c = cs[p], s = sn[p];
        for (int row = lane; row < lb; row += 32) {
          const TJ x = A[row * LS + a], y = A[row * LS + z];
          A[row * LS + a] = c * x - s * y;
          A[row * LS + z] = s * x + c * y;
          const TJ vx = W[row * LS + a], vy = W[row * LS + z];
          W[row * LS + a] = c * vx - s * vy;
          W[row * LS + z] = s * vx + c * vy;
        }
      }
      __syncthreads();
    }
  }
  // sort eigenvalues descending (selection by rank; ties broken by index)
  for (int i = threadIdx.x; i < lb; i += blockDim.x) {
    const TJ di = A[i * LS + i];
    int rank = 0;
    for (int j = 0; j < lb; ++j) {
      const TJ dj = A[j * LS + j];
      if (dj > di || (dj == di && j < i)) ++rank;
    }
    order[rank] = i;
  }
  __syncthreads();
  double* Vb = V + (int64_t)b * LPAD * LPAD;
  for (int q = threadIdx.x; q < LPAD * LPAD; q += blockDim.x) {
    const int i = q / LPAD, r = q % LPAD;  // Vb[i, r] = W[i, order[r]]
    Vb[q] = (r < lb && i < lb) ? (double)W[i * LS + order[r]] : 0.0;
  }
  for (int r = threadIdx.x; r < LPAD; r += blockDim.x)
    evals[(int64_t)b * LPAD + r] = r < lb ? (double)A[order[r] * LS + order[r]] : 0.0;
}

// Ritz vectors: Qout[v0 + i, r] = sum_j S[i, j] V[j, r] for r < kb (row panel S with
// stride lpad; output row stride k).  One 128-row tile per CTA iteration, register
// tiled as k_apply_rinv (V staged zero-padded to LPAD x LPAD).
template <class T, int LPAD>
__global__ void __launch_bounds__(256) k_ritz(Blocks B, const int32_t* __restrict__ unit_block,
                                               const int32_t* __restrict__ unit_tile, int nunits,
                                               const T* __restrict__ S, const double* __restrict__ V,
                                               T* __restrict__ Qout) {
  constexpr int TR = 128, LS = LPAD + 1, CT = LPAD / 16, RT = TR / 16;
  extern __shared__ __align__(16) uint8_t smraw[];
  T* sv = reinterpret_cast<T*>(smraw);  // LPAD x LPAD
  T* ss = sv + LPAD * LPAD;              // TR x LS
  const int k = B.k;
  const int tc = threadIdx.x & 15, tr = threadIdx.x >> 4;
  for (int u = blockIdx.x; u < nunits; u += gridDim.x) {
    const int b = unit_block[u];
    const int rows = B.rows[b];
    const int lb = B.lb[b], kb = B.kb[b];
    const int i0 = unit_tile[u] * TR;
    const int nr = rows - i0 < TR ? rows - i0 : TR;
    const int64_t r0 = B.arow[b] + i0;
    for (int q = threadIdx.x; q < LPAD * LPAD; q += blockDim.x) {
      const int j = q / LPAD, r = q % LPAD;
      sv[q] = (j < lb && r < kb) ? (T)V[(int64_t)b * LPAD * LPAD + q] : T(0);
    }
    for (int q = threadIdx.x; q < TR * LPAD; q += blockDim.x) {
      const int rr = q / LPAD, jj = q % LPAD;
      ss[rr * LS + jj] = rr < nr ? S[(r0 + rr) * LPAD + jj] : T(0);
    }
    __syncthreads();
    T acc[RT][CT];
#pragma unroll
    for (int a = 0; a < RT; ++a)
#pragma unroll
      for (int c = 0; c < CT; ++c) acc[a][c] = T(0);
#pragma unroll 2
    for (int j = 0; j < lb; ++j) {
      T sv_[CT], xv[RT];
#pragma unroll
      for (int a = 0; a < RT; ++a) xv[a] = ss[(tr + 16 * a) * LS + j];
#pragma unroll
      for (int c = 0; c < CT; ++c) sv_[c] = sv[j * LPAD + tc + 16 * c];
#pragma unroll
      for (int a = 0; a < RT; ++a)
#pragma unroll
        for (int c = 0; c < CT; ++c) acc[a][c] = fma(xv[a], sv_[c], acc[a][c]);
    }
#pragma unroll
    for (int a = 0; a < RT; ++a) {
      const int row = tr + 16 * a;
      if (row < nr)
#pragma unroll
        for (int c = 0; c < CT; ++c) {
          const int r = tc + 16 * c;
          if (r < k) Qout[(B.v0[b] + i0 + row) * k + r] = acc[a][c];
        }
    }
    __syncthreads();
  }
}

}  // namespace rsvd
}  // namespace hgl

namespace hgl {
namespace rsvd {

// ---------------------------------------------------------------------------
// Layout moves for hgl_block_product: a caller's row-major n x l panel S (FP32) into
// the transposed basis St (lpad x Ktot, zero beyond l and on padding columns) or into
// the block-row layout of the sparse route (rows_tot x LP, zero-padded), and the
// block-row product D back into the caller's n x l panel.
// ---------------------------------------------------------------------------
template <class TB>
__global__ void k_rows_to_st(Blocks B, const float* __restrict__ S, int64_t lds, int l, TB* __restrict__ St) {
  const int64_t total = (int64_t)B.lpad * B.Ktot;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(q / B.Ktot);
    const int64_t col = q % B.Ktot;
    const int b = find_block(B.koff, B.nb, col);
    const int64_t i = col - B.koff[b];
    const float x = (j < l && i < B.rows[b]) ? S[(B.v0[b] + i) * lds + j] : 0.f;
    St[(int64_t)j * B.Ktot + col] = from_double<TB>((double)x);
  }
}

template <int LP>
__global__ void k_rows_to_blockrows(Blocks B, int64_t rows_tot, const float* __restrict__ S, int64_t lds, int l,
                                    float* __restrict__ Qf) {
  const int64_t total = rows_tot * LP;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = q / LP;
    const int j = (int)(q % LP);
    const int b = find_block(B.arow, B.nb, r);
    const int64_t i = r - B.arow[b];
    Qf[q] = (j < l && i < B.rows[b]) ? S[(B.v0[b] + i) * lds + j] : 0.f;
  }
}

template <int LP>
__global__ void k_blockrows_to_rows(Blocks B, int64_t n, const float* __restrict__ Dw, int l, float* __restrict__ D,
                                    int64_t ldd) {
  const int64_t total = n * l;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t v = q / l;
    const int j = (int)(q % l);
    const int b = find_block(B.v0, B.nb, v);
    D[v * ldd + j] = Dw[(B.arow[b] + (v - B.v0[b])) * LP + j];
  }
}

}  // namespace rsvd
}  // namespace hgl

namespace hgl {
namespace rsvd {

// The symmetric part of a dense nb x nb matrix L into the block storage of a single
// block: A[i, j] = (L[i, j] + L[j, i]) / 2 for i, j < nb; zero elsewhere in the rows_tot
// x ldA storage (padding rows and columns).
static __global__ void k_sym_load(int64_t nb, int64_t rows_tot, int64_t ldA, const double* __restrict__ L, int64_t ldl,
                           double* __restrict__ A) {
  const int64_t total = rows_tot * ldA;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = q / ldA, j = q % ldA;
    A[q] = (i < nb && j < nb) ? 0.5 * (L[i * ldl + j] + L[j * ldl + i]) : 0.0;
  }
}

}  // namespace rsvd
}  // namespace hgl
