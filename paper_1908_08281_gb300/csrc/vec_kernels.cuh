// vec_kernels.cuh -- row-parallel panel kernels of the CG recurrences (Eqs. 16-20)
// and the per-column reductions behind alpha and beta.
//
// Lane layout: a warp is split into G = 32/LG groups of LG lanes; a group owns one
// row at a time and each lane one 16-byte vector of E columns; blockIdx.y selects the
// column tile of LG*E columns.  Per-column partial sums leave every block as one row
// of a [gridDim.x x c] FP64 array, reduced in a fixed order by k_cg_reduce.
#pragma once

#include "hgl_internal.cuh"
#include "panel.cuh"

namespace hgl {

constexpr int VEC_THREADS = 256;

struct CgState {
  int c;
  double* b2;      // ||lam y_j||^2
  double* rr;      // r^T r
  double* rz;      // r^T z (= rr without preconditioner)
  double* alpha;
  double* beta;
  double* target;  // stop once rr_j <= target_j
  double* relres;  // final relative residual
  int32_t* active;
  int32_t* iters;
  int32_t* bad;    // non-finite or breakdown seen in column j
  int32_t* run_flag;
  unsigned* done;  // last-block counter of k_cg_reduce
  int32_t* need;   // captured solves: 1 while a refinement sweep is needed (k_inner_targets)
  const int32_t* guard = nullptr;  // RED_RESID: skip the reduction when *guard == 0
};

enum ReduceMode : int {
  RED_B2 = 0,      // b2 = sum a
  RED_INIT = 1,    // rr = sum a, rz = sum b (or rr); active = rr > target
  RED_ALPHA = 2,   // alpha = rz / sum a
  RED_BETA = 3,    // rr' = sum a, rz' = sum b; beta = rz'/rz; active &= rr' > target
  RED_RESID = 4,   // relres = sqrt(sum a / b2)
};

template <class T, int LG>
struct VecLayout {
  static constexpr int E = 16 / (int)sizeof(T);
  static constexpr int G = 32 / LG;
  static constexpr int TILE = LG * E;
};

// Sum this thread's E column partials into partials[blockIdx.x * c + col] in a fixed order.
template <int E, int LG>
__device__ __forceinline__ void block_col_partials(const double (&v)[E], int col0, int c, double* partials) {
  __shared__ double red[VEC_THREADS * E];
#pragma unroll
  for (int j = 0; j < E; ++j) red[threadIdx.x * E + j] = v[j];
  __syncthreads();
  constexpr int TILE = LG * E;
  constexpr int G = 32 / LG;
  for (int q = threadIdx.x; q < TILE; q += blockDim.x) {
    const int l = q / E, j = q % E;
    double acc = 0.0;
    for (int w = 0; w < VEC_THREADS / 32; ++w)
      for (int g = 0; g < G; ++g) acc += red[(w * 32 + g * LG + l) * E + j];
    if (col0 + q < c) partials[(int64_t)blockIdx.x * c + col0 + q] = acc;
  }
  __syncthreads();
}

// partials <- per-column sums of scale * A[:, j] * B[:, j]  (B may alias A)
template <class TA, class TB, int LG>
__global__ void __launch_bounds__(VEC_THREADS)
k_panel_dot(int64_t n, int c, const TA* __restrict__ A, int64_t lda, const TB* __restrict__ B, int64_t ldb,
            double scale, double* __restrict__ partials, const int32_t* __restrict__ run_flag) {
  if (run_flag && *run_flag == 0) return;
  using L = VecLayout<TA, LG>;
  constexpr int E = L::E;
  using Acc = typename AccOf<TA>::type;
  const int lane = threadIdx.x & 31, grp = lane / LG, l = lane % LG, wid = threadIdx.x >> 5;
  const int col0 = blockIdx.y * L::TILE;
  const int col = col0 + l * E;
  DotAcc<Acc> d[E];
  if (col < c) {
    const int64_t rstep = (int64_t)gridDim.x * (VEC_THREADS / 32) * L::G;
    for (int64_t r = ((int64_t)blockIdx.x * (VEC_THREADS / 32) + wid) * L::G + grp; r < n; r += rstep) {
      Acc a[E], b[E];
      vload<Acc, TA, E>(A + r * lda + col, a);
      vload<Acc, TB, E>(B + r * ldb + col, b);
#pragma unroll
      for (int j = 0; j < E; ++j) d[j].add(a[j], b[j]);
    }
  }
  double v[E];
#pragma unroll
  for (int j = 0; j < E; ++j) v[j] = scale * d[j].value();
  block_col_partials<E, LG>(v, col0, c, partials);
}

// Z <- scale * X (type conversion allowed); optional partial sums of Z.Z
template <class TX, class TZ, int LG, bool DOT>
__global__ void __launch_bounds__(VEC_THREADS)
k_panel_scale(int64_t n, int c, const TX* __restrict__ X, int64_t ldx, double scale, TZ* __restrict__ Z,
              int64_t ldz, double* __restrict__ partials, const int32_t* __restrict__ run_flag) {
  if (run_flag && *run_flag == 0) return;
  using L = VecLayout<TZ, LG>;
  constexpr int E = L::E;
  using Acc = typename AccOf<TX>::type;
  const int lane = threadIdx.x & 31, grp = lane / LG, l = lane % LG, wid = threadIdx.x >> 5;
  const int col0 = blockIdx.y * L::TILE;
  const int col = col0 + l * E;
  DotAcc<Acc> d[E];
  // a unit scale is a plain copy (no FP64 conversions on FP32 panels)
  const bool unit = scale == 1.0;
  if (col < c) {
    const int64_t rstep = (int64_t)gridDim.x * (VEC_THREADS / 32) * L::G;
    for (int64_t r = ((int64_t)blockIdx.x * (VEC_THREADS / 32) + wid) * L::G + grp; r < n; r += rstep) {
      Acc x[E];
      vload<Acc, TX, E>(X + r * ldx + col, x);
      if (!unit)
#pragma unroll
        for (int j = 0; j < E; ++j) x[j] = (Acc)(scale * (double)x[j]);
      vstore<TZ, Acc, E>(Z + r * ldz + col, x, c - col);
      if (DOT) {
#pragma unroll
        for (int j = 0; j < E; ++j) d[j].add(x[j], x[j]);
      }
    }
  }
  if (DOT) {
    double v[E];
#pragma unroll
    for (int j = 0; j < E; ++j) v[j] = d[j].value();
    block_col_partials<E, LG>(v, col0, c, partials);
  }
}

// x += alpha p;  r -= alpha q;  partials <- r.r   (TP: type of p, TV: type of x, r, q)
template <class TP, class TV, int LG>
__global__ void __launch_bounds__(VEC_THREADS)
k_cg_update_xr(int64_t n, int c, const TP* __restrict__ P, int64_t ldp, const TV* __restrict__ Q, int64_t ldq,
               TV* __restrict__ X, int64_t ldx, TV* __restrict__ R, int64_t ldr, const double* __restrict__ alpha,
               double* __restrict__ partials, const int32_t* __restrict__ run_flag) {
  if (*run_flag == 0) return;
  using L = VecLayout<TV, LG>;
  constexpr int E = L::E;
  using Acc = typename AccOf<TV>::type;
  const int lane = threadIdx.x & 31, grp = lane / LG, l = lane % LG, wid = threadIdx.x >> 5;
  const int col0 = blockIdx.y * L::TILE;
  const int col = col0 + l * E;
  DotAcc<Acc> d[E];
  if (col < c) {
    Acc al[E];
#pragma unroll
    for (int j = 0; j < E; ++j) al[j] = col + j < c ? (Acc)alpha[col + j] : Acc(0);
    const int64_t rstep = (int64_t)gridDim.x * (VEC_THREADS / 32) * L::G;
    for (int64_t r = ((int64_t)blockIdx.x * (VEC_THREADS / 32) + wid) * L::G + grp; r < n; r += rstep) {
      Acc p[E], q[E], x[E], rv[E];
      vload<Acc, TP, E, false>(P + r * ldp + col, p);
      vload<Acc, TV, E, false>(Q + r * ldq + col, q);
      vload<Acc, TV, E, false>(X + r * ldx + col, x);
      vload<Acc, TV, E, false>(R + r * ldr + col, rv);
#pragma unroll
      for (int j = 0; j < E; ++j) {
        x[j] = fma(al[j], p[j], x[j]);
        rv[j] = fma(-al[j], q[j], rv[j]);
        d[j].add(rv[j], rv[j]);
      }
      vstore<TV, Acc, E>(X + r * ldx + col, x, c - col);
      vstore<TV, Acc, E>(R + r * ldr + col, rv, c - col);
    }
  }
  double v[E];
#pragma unroll
  for (int j = 0; j < E; ++j) v[j] = d[j].value();
  block_col_partials<E, LG>(v, col0, c, partials);
}

// p <- z + beta p   (z = r without preconditioner)
template <class TP, class TV, int LG>
__global__ void __launch_bounds__(VEC_THREADS)
k_cg_update_p(int64_t n, int c, const TV* __restrict__ Zr, int64_t ldz, TP* __restrict__ P, int64_t ldp,
              const double* __restrict__ beta, const int32_t* __restrict__ run_flag) {
  if (*run_flag == 0) return;
  using L = VecLayout<TV, LG>;
  constexpr int E = L::E;
  using Acc = typename AccOf<TV>::type;
  const int lane = threadIdx.x & 31, grp = lane / LG, l = lane % LG, wid = threadIdx.x >> 5;
  const int col0 = blockIdx.y * L::TILE;
  const int col = col0 + l * E;
  if (col >= c) return;
  Acc be[E];
#pragma unroll
  for (int j = 0; j < E; ++j) be[j] = col + j < c ? (Acc)beta[col + j] : Acc(0);
  const int64_t rstep = (int64_t)gridDim.x * (VEC_THREADS / 32) * L::G;
  for (int64_t r = ((int64_t)blockIdx.x * (VEC_THREADS / 32) + wid) * L::G + grp; r < n; r += rstep) {
    Acc z[E], p[E];
    vload<Acc, TV, E, false>(Zr + r * ldz + col, z);
    vload<Acc, TP, E, false>(P + r * ldp + col, p);
#pragma unroll
    for (int j = 0; j < E; ++j) p[j] = fma(be[j], p[j], z[j]);
    vstore<TP, Acc, E>(P + r * ldp + col, p, c - col);
  }
}

// F (FP64) += D (TD)
template <class TD, int LG>
__global__ void __launch_bounds__(VEC_THREADS)
k_add_correction(int64_t n, int c, const TD* __restrict__ D, int64_t ldd, double* __restrict__ F, int64_t ldf) {
  using L = VecLayout<double, LG>;
  constexpr int E = L::E;
  const int lane = threadIdx.x & 31, grp = lane / LG, l = lane % LG, wid = threadIdx.x >> 5;
  const int col = blockIdx.y * L::TILE + l * E;
  if (col >= c) return;
  const int64_t rstep = (int64_t)gridDim.x * (VEC_THREADS / 32) * L::G;
  for (int64_t r = ((int64_t)blockIdx.x * (VEC_THREADS / 32) + wid) * L::G + grp; r < n; r += rstep) {
    double f[E], d[E];
    vload<double, double, E, false>(F + r * ldf + col, f);
    vload<double, TD, E, false>(D + r * ldd + col, d);
#pragma unroll
    for (int j = 0; j < E; ++j) f[j] += d[j];
    vstore<double, double, E>(F + r * ldf + col, f, c - col);
  }
}

// Z[r, 0 : round4(c)] = 0 for FP32 panels with ldz a multiple of 4 (internal panels:
// their padding columns are zeroed too); returns at once when *run_flag == 0.
static __global__ void k_zero_panel(int64_t n, int c, float* __restrict__ Z, int64_t ldz,
                             const int32_t* __restrict__ run_flag) {
  if (run_flag && *run_flag == 0) return;
  const int vecs = (c + 3) / 4;
  const int64_t total = n * vecs;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x)
    *reinterpret_cast<float4*>(Z + (q / vecs) * ldz + (q % vecs) * 4) = make_float4(0.f, 0.f, 0.f, 0.f);
}

// Per-column reduction of [rows x c] partials and the scalar CG logic of column j.
// One warp per column (lanes over rows, fixed butterfly), the last block to finish
// sets run_flag = (number of active columns > 0).
template <int MODE>
__global__ void __launch_bounds__(256)
k_cg_reduce(const double* __restrict__ pa, const double* __restrict__ pb, int rows, CgState S) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int c = S.c;
  const int j = blockIdx.x * 8 + wid;
  if (MODE != RED_B2 && MODE != RED_INIT && MODE != RED_RESID && *S.run_flag == 0) return;
  if (MODE == RED_RESID && S.guard && *S.guard == 0) return;
  if (j < c) {
    double a = 0.0, b = 0.0;
    for (int r = lane; r < rows; r += 32) {
      a += pa[(int64_t)r * c + j];
      if (pb) b += pb[(int64_t)r * c + j];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      a += __shfl_xor_sync(0xffffffffu, a, o);
      b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    if (lane == 0) {
      if (MODE == RED_B2) {
        S.b2[j] = a;
      } else if (MODE == RED_INIT) {
        const double rz = pb ? b : a;
        S.rr[j] = a;
        S.rz[j] = rz;
        const bool finite = isfinite(a) && isfinite(rz);
        if (!finite) S.bad[j] = 1;
        S.active[j] = (finite && S.b2[j] > 0.0 && a > S.target[j]) ? 1 : 0;
        S.alpha[j] = 0.0;
        S.beta[j] = 0.0;
      } else if (MODE == RED_ALPHA) {
        double al = 0.0;
        if (S.active[j]) {
          if (a > 0.0 && isfinite(a)) {
            al = S.rz[j] / a;
          } else {
            S.bad[j] = 1;
            S.active[j] = 0;
          }
        }
        S.alpha[j] = al;
      } else if (MODE == RED_BETA) {
        if (S.active[j]) {
          const double rz = pb ? b : a;
          S.iters[j] += 1;
          if (!isfinite(a) || !isfinite(rz)) {
            S.bad[j] = 1;
            S.active[j] = 0;
            S.beta[j] = 0.0;
          } else {
            S.beta[j] = S.rz[j] > 0.0 ? rz / S.rz[j] : 0.0;
            S.rr[j] = a;
            S.rz[j] = rz;
            if (!(a > S.target[j])) S.active[j] = 0;
          }
        } else {
          S.beta[j] = 0.0;
        }
      } else if (MODE == RED_RESID) {
        S.rr[j] = a;
        const double b2 = S.b2[j];
        if (!isfinite(a) || !isfinite(b2)) {
          // a non-finite right-hand side or residual: relres NaN, so the column is
          // reported non-finite instead of passing as relres 0
          S.bad[j] = 1;
          S.relres[j] = __longlong_as_double(0x7ff8000000000000LL);
        } else {
          S.relres[j] = b2 > 0.0 ? sqrt(a / b2) : 0.0;
        }
      }
    }
  }
  if (MODE == RED_INIT || MODE == RED_BETA || MODE == RED_ALPHA) {
    __shared__ bool last;
    __shared__ int cnt[8];
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(S.done, 1u) == gridDim.x - 1;
    __syncthreads();
    if (last) {
      __threadfence();
      int a = 0;
      for (int q = threadIdx.x; q < c; q += blockDim.x) a += ((volatile int32_t*)S.active)[q];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
      if (lane == 0) cnt[wid] = a;
      __syncthreads();
      if (threadIdx.x == 0) {
        int tot = 0;
        for (int w = 0; w < 8; ++w) tot += cnt[w];
        *S.run_flag = tot > 0 ? 1 : 0;
        *S.done = 0u;
      }
    }
  }
}

}  // namespace hgl
