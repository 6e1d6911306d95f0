// theta_kernels.cuh -- the two gather passes that apply Theta (Eq. 1) matrix-free.
//
//   hyperedge pass:  T[q, :] = t_e * sum_{v in e} s_v X[v, :]  for the large hyperedges
//                    e = order[q] (more than SMALL_EDGE members)   (W De^-1 H^T Dv^-1/2 X)
//   vertex pass:     Z[u, :] = a X[u, :] + b s_u (sum_{large e ni u} T[slot(e), :]
//                              + sum_{small e ni u} t_e sum_{v in e} s_v X[v, :])   (+ gy Y[u, :])
//
// with s = dv^-1/2 and t = w / de.  A small hyperedge's terms are read straight from X
// by its members (the v = u term is the per-vertex diagonal s_u^2 sum t_e), which for
// d <= SMALL_EDGE members moves fewer bytes than an intermediate row written once and
// gathered d times.  Both passes are row gathers over the compressed
// layouts: one warp owns one output row at a time; the warp is split into G = 32/LG
// groups of LG lanes, each group reads one input row per step (16-byte vector loads,
// NV vectors per lane), and the groups are summed with a shuffle butterfly.  The
// right-hand-side columns are processed in chunks of LG*NV*E columns (E elements
// per 16 bytes) so that the gathered slice of X can stay in L2 across the pass.
#pragma once

#include "hgl_internal.cuh"
#include "panel.cuh"

namespace hgl {

constexpr int OP_THREADS = 256;
constexpr int OP_WARPS = OP_THREADS / 32;

// The small hyperedges' terms of the vertex pass (hgl_graph::scsr_*, scoef, sdiag).
template <class A>
struct SmallTerms {
  const int64_t* ptr;  // n+1
  const int32_t* nb;   // other member of a small hyperedge
  const A* coef;       // t_e s_nb
  const A* diag;       // n: s_u^2 sum_{small e ni u} t_e
};

// z + gy y of the residual epilogue: in FP64 for FP64 accumulators, in FP32 for FP32
// ones (an FP32 residual is an estimate: its rounding, a few units of 2^-24 of |lam Y|,
// is far above FP64's, and FP64 arithmetic would slow the pass several-fold).
__device__ __forceinline__ double resid_add(double z, double gy, double y) { return z + gy * y; }
__device__ __forceinline__ float resid_add(float z, double gy, double y) {
  return __fmaf_rn((float)gy, (float)y, z);
}

// Hyperedges are visited in decreasing size order (`order`).  The first `nheavy` of
// them (more than HEAVY_ROW members) get one thread block each: the block's warps
// split the member list and their partial sums are added in warp order through
// shared memory.  The remaining blocks walk the light rows one warp per row.
// One heavy hyperedge (order[blockIdx.x]) per thread block: the block's warps split
// the member list, groups of LG lanes read one member row each, and the warps' partial
// sums are added in warp order through shared memory.
template <class TX, class TT, int LG, int NV>
__device__ __forceinline__ void edge_heavy_block(const int64_t* __restrict__ csc_ptr,
                                                 const int32_t* __restrict__ csc_idx,
                                                 const int32_t* __restrict__ order, const typename AccOf<TX>::type* __restrict__ s,
                                                 const typename AccOf<TX>::type* __restrict__ t, const TX* __restrict__ X, int64_t ldx,
                                                 int c0, int cw, TT* __restrict__ Tp, int64_t ldt) {
  using A = typename AccOf<TX>::type;
  constexpr int E = 16 / (int)sizeof(TX);
  constexpr int G = 32 / LG;
  constexpr int TILE = LG * NV * E;
  const int lane = threadIdx.x & 31, grp = lane / LG, l = lane % LG, wid = threadIdx.x >> 5;
  const TX* Xc = X + c0;
  A acc[NV][E];
  __shared__ A red[OP_WARPS][TILE];
  const int32_t e = order[blockIdx.x];
  const int64_t beg = __ldg(csc_ptr + e), end = __ldg(csc_ptr + e + 1);
#pragma unroll
  for (int k = 0; k < NV; ++k)
#pragma unroll
    for (int j = 0; j < E; ++j) acc[k][j] = A(0);
  for (int64_t i = beg + wid * G + grp; i < end; i += OP_WARPS * G) {
    const int32_t v = __ldg(csc_idx + i);
    const A sv = (A)__ldg(s + v);
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      const int col = (k * LG + l) * E;
      if (col < cw) {
        A x[E];
        vload<A, TX, E>(Xc + (int64_t)v * ldx + col, x);
#pragma unroll
        for (int j = 0; j < E; ++j) acc[k][j] = fma(sv, x[j], acc[k][j]);
      }
    }
  }
#pragma unroll
  for (int off = LG; off < 32; off <<= 1)
#pragma unroll
    for (int k = 0; k < NV; ++k)
#pragma unroll
      for (int j = 0; j < E; ++j) acc[k][j] += __shfl_xor_sync(0xffffffffu, acc[k][j], off);
  if (grp == 0)
#pragma unroll
    for (int k = 0; k < NV; ++k)
#pragma unroll
      for (int j = 0; j < E; ++j) red[wid][(k * LG + l) * E + j] = acc[k][j];
  __syncthreads();
  if (wid == 0 && grp == 0) {
    const A te = (A)__ldg(t + e);
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      const int col = (k * LG + l) * E;
      if (col < cw) {
        A o[E];
#pragma unroll
        for (int j = 0; j < E; ++j) {
          A sum = A(0);
          for (int w = 0; w < OP_WARPS; ++w) sum += red[w][col + j];
          o[j] = te * sum;
        }
        vstore<TT, A, E>(Tp + (int64_t)blockIdx.x * ldt + col, o, E);
      }
    }
  }
}

// m: the number of large hyperedges (slots 0 .. m-1 of `order`); T row q is slot q.
template <class TX, class TT, int LG, int NV>
__global__ void __launch_bounds__(OP_THREADS)
k_edge_pass(int64_t m, const int64_t* __restrict__ csc_ptr, const int32_t* __restrict__ csc_idx,
            const int32_t* __restrict__ order, int64_t nheavy, const typename AccOf<TX>::type* __restrict__ s,
            const typename AccOf<TX>::type* __restrict__ t, const TX* __restrict__ X, int64_t ldx, int c0, int cw, TT* __restrict__ Tp,
            int64_t ldt, const int32_t* __restrict__ run_flag) {
  if (run_flag && *run_flag == 0) return;
  using A = typename AccOf<TX>::type;
  constexpr int E = 16 / (int)sizeof(TX);
  constexpr int G = 32 / LG;
  constexpr int U = 2;
  const int lane = threadIdx.x & 31, grp = lane / LG, l = lane % LG;
  const TX* Xc = X + c0;
  A acc[NV][E];
  if (blockIdx.x < nheavy) {
    edge_heavy_block<TX, TT, LG, NV>(csc_ptr, csc_idx, order, s, t, X, ldx, c0, cw, Tp, ldt);
    return;
  }
  const int64_t warp = (((int64_t)blockIdx.x - nheavy) * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = (((int64_t)gridDim.x - nheavy) * blockDim.x) >> 5;
  for (int64_t q = nheavy + warp; q < m; q += nwarps) {
    const int32_t e = order[q];
    const int64_t beg = __ldg(csc_ptr + e), end = __ldg(csc_ptr + e + 1);
#pragma unroll
    for (int k = 0; k < NV; ++k)
#pragma unroll
      for (int j = 0; j < E; ++j) acc[k][j] = A(0);
    int64_t i = beg + grp;
    for (; i + (U - 1) * G < end; i += U * G) {
      int32_t v[U];
      A sv[U];
#pragma unroll
      for (int u = 0; u < U; ++u) v[u] = __ldg(csc_idx + i + u * G);
#pragma unroll
      for (int u = 0; u < U; ++u) sv[u] = (A)__ldg(s + v[u]);
#pragma unroll
      for (int u = 0; u < U; ++u)
#pragma unroll
        for (int k = 0; k < NV; ++k) {
          const int col = (k * LG + l) * E;
          if (col < cw) {
            A x[E];
            vload<A, TX, E>(Xc + (int64_t)v[u] * ldx + col, x);
#pragma unroll
            for (int j = 0; j < E; ++j) acc[k][j] = fma(sv[u], x[j], acc[k][j]);
          }
        }
    }
    for (; i < end; i += G) {
      const int32_t v = __ldg(csc_idx + i);
      const A sv = (A)__ldg(s + v);
#pragma unroll
      for (int k = 0; k < NV; ++k) {
        const int col = (k * LG + l) * E;
        if (col < cw) {
          A x[E];
          vload<A, TX, E>(Xc + (int64_t)v * ldx + col, x);
#pragma unroll
          for (int j = 0; j < E; ++j) acc[k][j] = fma(sv, x[j], acc[k][j]);
        }
      }
    }
#pragma unroll
    for (int off = LG; off < 32; off <<= 1)
#pragma unroll
      for (int k = 0; k < NV; ++k)
#pragma unroll
        for (int j = 0; j < E; ++j) acc[k][j] += __shfl_xor_sync(0xffffffffu, acc[k][j], off);
    if (grp == 0) {
      const A te = (A)__ldg(t + e);
#pragma unroll
      for (int k = 0; k < NV; ++k) {
        const int col = (k * LG + l) * E;
        if (col < cw) {
          A o[E];
#pragma unroll
          for (int j = 0; j < E; ++j) o[j] = te * acc[k][j];
          vstore<TT, A, E>(Tp + q * ldt + col, o, E);
        }
      }
    }
  }
}

// The CG's variant with BF16 search directions and one vector per lane is bounded to
// five resident blocks per SM (48 registers instead of 64, 48 bytes spilled): its
// dependent intermediate-row gathers gain more from the extra warps than the spills cost
// (8.62 against 8.88 ms per apply at n = 1M, c = 512); the other variants keep the
// compiler's choice (wider tiles would spill hundreds of bytes).
template <class TX, class TT, class TZ, int LG, int NV, int EPI>
__global__ void __launch_bounds__(OP_THREADS, (sizeof(TX) == 2 && EPI == EPI_DOT_XZ && NV == 1) ? 5 : 1)
k_vertex_pass(int64_t n, const int64_t* __restrict__ csr_ptr, const int32_t* __restrict__ csr_idx,
              const SmallTerms<typename AccOf<TX>::type> sm,
              const typename AccOf<TX>::type* __restrict__ s, const TT* __restrict__ Tp, int64_t ldt, const TX* __restrict__ X,
              int64_t ldx, TZ* __restrict__ Z, int64_t ldz, int c0, int cw, int c, double a, double b,
              const double* __restrict__ Y, int64_t ldy, double gy, double* __restrict__ partials,
              const int32_t* __restrict__ run_flag) {
  if (run_flag && *run_flag == 0) return;
  using A = typename AccOf<TX>::type;
  constexpr int E = 16 / (int)sizeof(TX);
  constexpr int G = 32 / LG;
  constexpr int U = 2;
  constexpr int TILE = LG * NV * E;
  const int lane = threadIdx.x & 31, grp = lane / LG, l = lane % LG;
  const int wid = threadIdx.x >> 5;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const A aa = (A)a, bb = (A)b;
  DotAcc<A> dot[NV][E];
  for (int64_t v = warp; v < n; v += nwarps) {
    const int64_t beg = __ldg(csr_ptr + v), end = __ldg(csr_ptr + v + 1);
    A acc[NV][E];
#pragma unroll
    for (int k = 0; k < NV; ++k)
#pragma unroll
      for (int j = 0; j < E; ++j) acc[k][j] = A(0);
    int64_t i = beg + grp;
    for (; i + (U - 1) * G < end; i += U * G) {
      int32_t e[U];
#pragma unroll
      for (int u = 0; u < U; ++u) e[u] = __ldg(csr_idx + i + u * G);
#pragma unroll
      for (int u = 0; u < U; ++u)
#pragma unroll
        for (int k = 0; k < NV; ++k) {
          const int col = (k * LG + l) * E;
          if (col < cw) {
            A x[E];
            vload<A, TT, E>(Tp + (int64_t)e[u] * ldt + col, x);
#pragma unroll
            for (int j = 0; j < E; ++j) acc[k][j] += x[j];
          }
        }
    }
    for (; i < end; i += G) {
      const int32_t e = __ldg(csr_idx + i);
#pragma unroll
      for (int k = 0; k < NV; ++k) {
        const int col = (k * LG + l) * E;
        if (col < cw) {
          A x[E];
          vload<A, TT, E>(Tp + (int64_t)e * ldt + col, x);
#pragma unroll
          for (int j = 0; j < E; ++j) acc[k][j] += x[j];
        }
      }
    }
    // small hyperedges: the other members' rows of X, weighted by t_e s_nb
    for (int64_t k2 = __ldg(sm.ptr + v) + grp, kend = __ldg(sm.ptr + v + 1); k2 < kend; k2 += G) {
      const int32_t u = __ldg(sm.nb + k2);
      const A cf = __ldg(sm.coef + k2);
#pragma unroll
      for (int k = 0; k < NV; ++k) {
        const int col = (k * LG + l) * E;
        if (col < cw) {
          A x[E];
          vload<A, TX, E>(X + (int64_t)u * ldx + c0 + col, x);
#pragma unroll
          for (int j = 0; j < E; ++j) acc[k][j] = fma(cf, x[j], acc[k][j]);
        }
      }
    }
#pragma unroll
    for (int off = LG; off < 32; off <<= 1)
#pragma unroll
      for (int k = 0; k < NV; ++k)
#pragma unroll
        for (int j = 0; j < E; ++j) acc[k][j] += __shfl_xor_sync(0xffffffffu, acc[k][j], off);
    if (grp == 0) {
      const A sb = bb * (A)__ldg(s + v);
      const A ad = aa + bb * __ldg(sm.diag + v);
#pragma unroll
      for (int k = 0; k < NV; ++k) {
        const int col = (k * LG + l) * E;
        if (col < cw) {
          A x[E], z[E];
          vload<A, TX, E>(X + v * ldx + c0 + col, x);
#pragma unroll
          for (int j = 0; j < E; ++j) z[j] = fma(ad, x[j], sb * acc[k][j]);
          if constexpr (EPI == EPI_RESID) {
            double y[E];
            const int nv = cw - col < E ? cw - col : E;
            for (int j = 0; j < E; ++j) y[j] = j < nv ? Y[v * ldy + c0 + col + j] : 0.0;
#pragma unroll
            for (int j = 0; j < E; ++j) z[j] = resid_add(z[j], gy, y[j]);
          }
          const int nvalid = cw - col;
          vstore<TZ, A, E>(Z + v * ldz + c0 + col, z, nvalid);
          if constexpr (EPI == EPI_DOT_XZ) {
#pragma unroll
            for (int j = 0; j < E; ++j) dot[k][j].add(x[j], z[j]);
          } else if constexpr (EPI == EPI_RESID) {
#pragma unroll
            for (int j = 0; j < E; ++j) dot[k][j].add(z[j], z[j]);
          }
        }
      }
    }
  }
  if constexpr (EPI != EPI_PLAIN) {
    // deterministic block reduction: warps add their column partials in turn
    __shared__ double red[TILE];
    for (int q = threadIdx.x; q < TILE; q += blockDim.x) red[q] = 0.0;
    __syncthreads();
    for (int w = 0; w < OP_WARPS; ++w) {
      if (wid == w && grp == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k)
#pragma unroll
          for (int j = 0; j < E; ++j) red[(k * LG + l) * E + j] += dot[k][j].value();
      }
      __syncthreads();
    }
    for (int q = threadIdx.x; q < cw && q < TILE; q += blockDim.x) partials[(int64_t)blockIdx.x * c + c0 + q] = red[q];
  }
}

// ---------------------------------------------------------------------------
// Narrow column chunks (LG * E columns, LG <= 8): one group of LG lanes owns one output
// row, so a warp keeps 32 / LG rows in flight and every group walks its own row's
// members with RU gathers outstanding; no reduction across groups is needed.  The
// per-row chain of dependent loads (order, row pointers, member ids, gathered rows)
// is thereby overlapped 32 / LG ways, and a chunk narrow enough for its slice of X
// (or of the intermediate) to stay in L2 is served mostly from L2.  Members are
// summed in list order, as in the wide kernels.  Heavy hyperedges keep one thread
// block each.
// ---------------------------------------------------------------------------
constexpr int RU = 4;

template <class TX, class TT, int LG>
__global__ void __launch_bounds__(OP_THREADS)
k_edge_rows(int64_t m, const int64_t* __restrict__ csc_ptr, const int32_t* __restrict__ csc_idx,
            const int32_t* __restrict__ order, int64_t nheavy, const typename AccOf<TX>::type* __restrict__ s,
            const typename AccOf<TX>::type* __restrict__ t, const TX* __restrict__ X, int64_t ldx, int c0, int cw, TT* __restrict__ Tp,
            int64_t ldt, const int32_t* __restrict__ run_flag) {
  if (run_flag && *run_flag == 0) return;
  using A = typename AccOf<TX>::type;
  constexpr int E = 16 / (int)sizeof(TX);
  if (blockIdx.x < nheavy) {
    edge_heavy_block<TX, TT, LG, 1>(csc_ptr, csc_idx, order, s, t, X, ldx, c0, cw, Tp, ldt);
    return;
  }
  const int col = ((threadIdx.x & 31) % LG) * E;
  const bool active = col < cw;
  const TX* Xc = X + c0 + col;
  const int64_t grp = (((int64_t)blockIdx.x - nheavy) * blockDim.x + threadIdx.x) / LG;
  const int64_t ngrp = (((int64_t)gridDim.x - nheavy) * blockDim.x) / LG;
  for (int64_t q = nheavy + grp; q < m; q += ngrp) {
    const int32_t e = __ldg(order + q);
    const int64_t beg = __ldg(csc_ptr + e), end = __ldg(csc_ptr + e + 1);
    A acc[E];
#pragma unroll
    for (int j = 0; j < E; ++j) acc[j] = A(0);
    int64_t i = beg;
    for (; i + RU <= end; i += RU) {
      int32_t v[RU];
      A sv[RU];
      A x[RU][E];
#pragma unroll
      for (int u = 0; u < RU; ++u) v[u] = __ldg(csc_idx + i + u);
      if (active) {
#pragma unroll
        for (int u = 0; u < RU; ++u) {
          sv[u] = (A)__ldg(s + v[u]);
          vload<A, TX, E>(Xc + (int64_t)v[u] * ldx, x[u]);
        }
#pragma unroll
        for (int u = 0; u < RU; ++u)
#pragma unroll
          for (int j = 0; j < E; ++j) acc[j] = fma(sv[u], x[u][j], acc[j]);
      }
    }
    for (; i < end; ++i) {
      const int32_t v = __ldg(csc_idx + i);
      if (active) {
        const A sv = (A)__ldg(s + v);
        A x[E];
        vload<A, TX, E>(Xc + (int64_t)v * ldx, x);
#pragma unroll
        for (int j = 0; j < E; ++j) acc[j] = fma(sv, x[j], acc[j]);
      }
    }
    if (active) {
      const A te = (A)__ldg(t + e);
      A o[E];
#pragma unroll
      for (int j = 0; j < E; ++j) o[j] = te * acc[j];
      vstore<TT, A, E>(Tp + q * ldt + col, o, E);
    }
  }
}

template <class TX, class TT, class TZ, int LG, int EPI>
__global__ void __launch_bounds__(OP_THREADS)
k_vertex_rows(int64_t n, const int64_t* __restrict__ csr_ptr, const int32_t* __restrict__ csr_idx,
              const SmallTerms<typename AccOf<TX>::type> sm,
              const typename AccOf<TX>::type* __restrict__ s, const TT* __restrict__ Tp, int64_t ldt, const TX* __restrict__ X,
              int64_t ldx, TZ* __restrict__ Z, int64_t ldz, int c0, int cw, int c, double a, double b,
              const double* __restrict__ Y, int64_t ldy, double gy, double* __restrict__ partials,
              const int32_t* __restrict__ run_flag) {
  if (run_flag && *run_flag == 0) return;
  using A = typename AccOf<TX>::type;
  constexpr int E = 16 / (int)sizeof(TX);
  constexpr int TILE = LG * E;
  const int lane = threadIdx.x & 31, l = lane % LG, wid = threadIdx.x >> 5;
  const int col = l * E;
  const bool active = col < cw;
  const TT* Tc = Tp + col;
  const int64_t grp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / LG;
  const int64_t ngrp = ((int64_t)gridDim.x * blockDim.x) / LG;
  const A aa = (A)a, bb = (A)b;
  DotAcc<A> dot[E];
  for (int64_t v = grp; v < n; v += ngrp) {
    const int64_t beg = __ldg(csr_ptr + v), end = __ldg(csr_ptr + v + 1);
    A acc[E];
#pragma unroll
    for (int j = 0; j < E; ++j) acc[j] = A(0);
    int64_t i = beg;
    for (; i + RU <= end; i += RU) {
      int32_t e[RU];
      A x[RU][E];
#pragma unroll
      for (int u = 0; u < RU; ++u) e[u] = __ldg(csr_idx + i + u);
      if (active) {
#pragma unroll
        for (int u = 0; u < RU; ++u) vload<A, TT, E>(Tc + (int64_t)e[u] * ldt, x[u]);
#pragma unroll
        for (int u = 0; u < RU; ++u)
#pragma unroll
          for (int j = 0; j < E; ++j) acc[j] += x[u][j];
      }
    }
    for (; i < end; ++i) {
      const int32_t e = __ldg(csr_idx + i);
      if (active) {
        A x[E];
        vload<A, TT, E>(Tc + (int64_t)e * ldt, x);
#pragma unroll
        for (int j = 0; j < E; ++j) acc[j] += x[j];
      }
    }
    // small hyperedges: the other members' rows of X, weighted by t_e s_nb
    for (int64_t k2 = __ldg(sm.ptr + v), kend = __ldg(sm.ptr + v + 1); k2 < kend; ++k2) {
      const int32_t u = __ldg(sm.nb + k2);
      const A cf = __ldg(sm.coef + k2);
      if (active) {
        A x[E];
        vload<A, TX, E>(X + (int64_t)u * ldx + c0 + col, x);
#pragma unroll
        for (int j = 0; j < E; ++j) acc[j] = fma(cf, x[j], acc[j]);
      }
    }
    if (active) {
      const A sb = bb * (A)__ldg(s + v);
      const A ad = aa + bb * __ldg(sm.diag + v);
      A x[E], z[E];
      vload<A, TX, E>(X + v * ldx + c0 + col, x);
#pragma unroll
      for (int j = 0; j < E; ++j) z[j] = fma(ad, x[j], sb * acc[j]);
      if constexpr (EPI == EPI_RESID) {
        double y[E];
        const int nv = cw - col < E ? cw - col : E;
        for (int j = 0; j < E; ++j) y[j] = j < nv ? Y[v * ldy + c0 + col + j] : 0.0;
#pragma unroll
        for (int j = 0; j < E; ++j) z[j] = resid_add(z[j], gy, y[j]);
      }
      vstore<TZ, A, E>(Z + v * ldz + c0 + col, z, cw - col);
      if constexpr (EPI == EPI_DOT_XZ) {
#pragma unroll
        for (int j = 0; j < E; ++j) dot[j].add(x[j], z[j]);
      } else if constexpr (EPI == EPI_RESID) {
#pragma unroll
        for (int j = 0; j < E; ++j) dot[j].add(z[j], z[j]);
      }
    }
  }
  if constexpr (EPI != EPI_PLAIN) {
    // deterministic reduction: the groups of a warp by a butterfly, then warps in order
    double dv[E];
#pragma unroll
    for (int j = 0; j < E; ++j) dv[j] = dot[j].value();
#pragma unroll
    for (int off = LG; off < 32; off <<= 1)
#pragma unroll
      for (int j = 0; j < E; ++j) dv[j] += __shfl_xor_sync(0xffffffffu, dv[j], off);
    __shared__ double red[OP_WARPS][TILE];
    if (lane < LG)
#pragma unroll
      for (int j = 0; j < E; ++j) red[wid][col + j] = dv[j];
    __syncthreads();
    for (int q = threadIdx.x; q < cw && q < TILE; q += blockDim.x) {
      double sum = 0.0;
      for (int w = 0; w < OP_WARPS; ++w) sum += red[w][q];
      partials[(int64_t)blockIdx.x * c + c0 + q] = sum;
    }
  }
}

// (LG, NV) configurations compiled for every kernel family.
#define HGL_FOR_EACH_TILE(X) X(1, 1) X(2, 1) X(4, 1) X(8, 1) X(16, 1) X(32, 1) X(32, 2) X(32, 4)
// The operator takes the row-per-group kernels for LG <= 8 and the wide ones above.
#define HGL_FOR_EACH_ROW_LG(X) X(1) X(2) X(4) X(8)
#define HGL_FOR_EACH_WIDE_TILE(X) X(16, 1) X(32, 1) X(32, 2) X(32, 4)

// Pick (LG, NV) for a chunk of `vecs` 16-byte vectors per row (vecs >= 1):
// LG = min(32, next power of two), NV = ceil(vecs / 32) rounded up to 1, 2 or 4.
inline void pick_tile(int vecs, int* lg, int* nv) {
  if (vecs <= 32) {
    int p = 1;
    while (p < vecs) p <<= 1;
    *lg = p;
    *nv = 1;
  } else {
    *lg = 32;
    *nv = vecs <= 64 ? 2 : 4;
  }
}

}  // namespace hgl
