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

// ---------------------------------------------------------------------------
// Dense diagonal blocks Theta_bb[i, j] = s_u s_v sum_{e containing u and v} t_e,
// u = v0 + i, v = v0 + j.  One warp per storage row: the row (padded width) is zeroed,
// the diagonal is summed over the vertex's hyperedges, and the off-diagonal terms are
// added hyperedge by hyperedge from the members that fall inside the block (found by
// binary search in the sorted member list).  Padding rows stay zero.
// ---------------------------------------------------------------------------
template <class TA>
__global__ void k_assemble(Blocks B, int64_t rows_tot, const int64_t* __restrict__ csr_ptr,
                           const int32_t* __restrict__ csr_idx, const int64_t* __restrict__ csc_ptr,
                           const int32_t* __restrict__ csc_idx, const double* __restrict__ s,
                           const double* __restrict__ t, TA* __restrict__ A) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t r = warp; r < rows_tot; r += nwarps) {
    const int b = find_block(B.arow, B.nb, r);
    const int64_t i = r - B.arow[b];
    const int bs = B.rows[b];
    const int64_t width = ((int64_t)bs + 63) / 64 * 64;
    TA* row = A + r * B.ldA;
    for (int64_t j = lane; j < width; j += 32) row[j] = from_double<TA>(0.0);
    if (i >= bs) continue;
    __syncwarp();
    const int64_t v0 = B.v0[b];
    const int64_t u = v0 + i;
    const double su = s[u];
    const int64_t beg = csr_ptr[u], end = csr_ptr[u + 1];
    double d = 0.0;
    for (int64_t q = beg + lane; q < end; q += 32) d += t[csr_idx[q]];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
    if (lane == 0) row[i] = from_double<TA>(su * su * d);
    __syncwarp();
    for (int64_t q = beg; q < end; ++q) {
      const int32_t e = csr_idx[q];
      const int64_t mb = csc_ptr[e], me = csc_ptr[e + 1];
      // members of e inside [v0, v0 + bs): lower bounds by binary search (lane 0)
      int64_t lo = 0, hi = 0;
      if (lane == 0) {
        int64_t a = mb, z = me;
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
      lo = __shfl_sync(0xffffffffu, lo, 0);
      hi = __shfl_sync(0xffffffffu, hi, 0);
      if (hi - lo > 1) {
        const double f = su * t[e];
        for (int64_t p = lo + lane; p < hi; p += 32) {
          const int32_t v = csc_idx[p];
          if (v != u) {
            const int64_t j = v - v0;
            row[j] = from_double<TA>(to_double<TA>(row[j]) + f * s[v]);
          }
        }
      }
      __syncwarp();
    }
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

// Omega[g, j] for global row g and column j (Box-Muller on one Philox draw per pair).
__device__ __forceinline__ double omega_entry(int64_t g, int j, uint64_t seed) {
  uint32_t c[4] = {(uint32_t)g, (uint32_t)(j >> 1), OMEGA_STREAM, 0u};
  philox4x32_10(c, (uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32));
  const double u1 = unit53(c[0], c[1]);
  const double u2 = unit53(c[2], c[3]);
  const double r = sqrt(-2.0 * log(u1));
  double sn, cs;
  sincos(2.0 * 3.14159265358979323846 * u2, &sn, &cs);
  return (j & 1) ? r * sn : r * cs;
}

// Transposed basis St (lpad x Ktot): St[j, koff_b + i] = Omega[v0_b + i, j] for j < lb_b,
// i < rows_b; every other entry (columns j >= lb, padding i) is zero.
template <class TB>
__global__ void k_omega(Blocks B, uint64_t seed, TB* __restrict__ St) {
  const int64_t total = (int64_t)B.lpad * B.Ktot;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(q / B.Ktot);
    const int64_t col = q % B.Ktot;
    const int b = find_block(B.koff, B.nb, col);
    const int64_t i = col - B.koff[b];
    double v = 0.0;
    if (i < B.rows[b] && j < B.lb[b]) v = omega_entry(B.v0[b] + i, j, seed);
    St[q] = from_double<TB>(v);
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
// row stride lpad: one CTA per block, rows in tiles of 64; products in the panel type,
// tile partial sums added into FP64 accumulators.
// ---------------------------------------------------------------------------
template <class T, int LPAD>
__global__ void __launch_bounds__(256) k_gram(Blocks B, const T* __restrict__ X, const T* __restrict__ Y,
                                               double* __restrict__ G) {
  constexpr int TR = 64;
  constexpr int NE = (LPAD * LPAD + 255) / 256;
  __shared__ T sx[TR][LPAD];
  __shared__ T sy[TR][LPAD];
  const int b = blockIdx.x;
  const int rows = B.rows[b];
  const int64_t r0 = B.arow[b];
  double acc[NE];
#pragma unroll
  for (int e = 0; e < NE; ++e) acc[e] = 0.0;
  for (int t0 = 0; t0 < rows; t0 += TR) {
    const int nr = rows - t0 < TR ? rows - t0 : TR;
    for (int q = threadIdx.x; q < TR * LPAD; q += blockDim.x) {
      const int rr = q / LPAD, jj = q % LPAD;
      sx[rr][jj] = rr < nr ? X[(r0 + t0 + rr) * LPAD + jj] : T(0);
      sy[rr][jj] = rr < nr ? Y[(r0 + t0 + rr) * LPAD + jj] : T(0);
    }
    __syncthreads();
#pragma unroll
    for (int e = 0; e < NE; ++e) {
      const int q = threadIdx.x + e * 256;
      if (q < LPAD * LPAD) {
        const int i = q / LPAD, j = q % LPAD;
        T a = T(0);
        for (int rr = 0; rr < TR; ++rr) a = fma(sx[rr][i], sy[rr][j], a);
        acc[e] += (double)a;
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int e = 0; e < NE; ++e) {
    const int q = threadIdx.x + e * 256;
    if (q < LPAD * LPAD) G[(int64_t)b * LPAD * LPAD + q] = acc[e];
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
  extern __shared__ double sm[];
  double* L = sm;                   // LPAD x LPAD
  double* X = sm + LPAD * LPAD;     // LPAD x LPAD
  __shared__ double s_trace, s_dmax;
  __shared__ int dead[LPAD];
  __shared__ int s_ndead;
  const int b = blockIdx.x;
  const int lb = B.lb[b];
  const double* Gb = G + (int64_t)b * LPAD * LPAD;
  for (int q = threadIdx.x; q < LPAD * LPAD; q += blockDim.x) {
    const int i = q / LPAD, j = q % LPAD;
    L[q] = (i < lb && j < lb) ? 0.5 * (Gb[i * LPAD + j] + Gb[j * LPAD + i]) : 0.0;
    X[q] = 0.0;
  }
  for (int j = threadIdx.x; j < LPAD; j += blockDim.x) dead[j] = 0;
  __syncthreads();
  if (threadIdx.x == 0) {
    double tr = 0.0, dm = 0.0;
    for (int i = 0; i < lb; ++i) {
      tr += L[i * LPAD + i];
      dm = fmax(dm, L[i * LPAD + i]);
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
  for (int i = threadIdx.x; i < lb; i += blockDim.x) L[i * LPAD + i] += sigma;
  __syncthreads();
  // right-looking Cholesky with dropped pivots
  for (int j = 0; j < lb; ++j) {
    if (threadIdx.x == 0) {
      const double d = L[j * LPAD + j];
      if (!(d > floor_pivot) || !isfinite(d)) {
        dead[j] = 1;
        s_ndead += 1;
        L[j * LPAD + j] = 1.0;
      } else {
        L[j * LPAD + j] = sqrt(d);
      }
    }
    __syncthreads();
    const double dj = L[j * LPAD + j];
    const bool dj_dead = dead[j] != 0;
    for (int i = j + 1 + threadIdx.x; i < lb; i += blockDim.x)
      L[i * LPAD + j] = dj_dead ? 0.0 : L[i * LPAD + j] / dj;
    __syncthreads();
    const int m = lb - j - 1;
    for (int q = threadIdx.x; q < m * m; q += blockDim.x) {
      const int i = j + 1 + q / m, k = j + 1 + q % m;
      if (k <= i) L[i * LPAD + k] -= L[i * LPAD + j] * L[k * LPAD + j];
    }
    __syncthreads();
  }
  // X = L^-1 (lower), one column per thread: forward substitution
  for (int c = threadIdx.x; c < lb; c += blockDim.x) {
    X[c * LPAD + c] = 1.0 / L[c * LPAD + c];
    for (int i = c + 1; i < lb; ++i) {
      double sacc = 0.0;
      for (int k = c; k < i; ++k) sacc += L[i * LPAD + k] * X[k * LPAD + c];
      X[i * LPAD + c] = -sacc / L[i * LPAD + i];
    }
  }
  __syncthreads();
  // Rinv = X^T (upper); dead directions get a zero row and column
  for (int q = threadIdx.x; q < LPAD * LPAD; q += blockDim.x) {
    const int i = q / LPAD, j = q % LPAD;
    Rb[q] = (i < lb && j < lb && !dead[i] && !dead[j]) ? X[j * LPAD + i] : 0.0;
  }
  if (threadIdx.x == 0 && s_ndead) atomicAdd(fail, 1);
}

// Q = Y Rinv row by row (one CTA per 64-row tile of a block); writes the row panel Qf
// (row stride lpad) and, if St is given, the transposed basis St[j, koff + i] for the
// next product.  TY: panel type of Y/Qf; TR: type of Rinv used in the product.
template <class T, class TB, int LPAD>
__global__ void __launch_bounds__(256) k_apply_rinv(Blocks B, const int32_t* __restrict__ unit_block,
                                                     const int32_t* __restrict__ unit_tile, int nunits,
                                                     const T* __restrict__ Y, const double* __restrict__ Rinv,
                                                     T* __restrict__ Qf, TB* __restrict__ St) {
  constexpr int TR = 128;
  extern __shared__ uint8_t smraw[];
  T* sr = reinterpret_cast<T*>(smraw);             // LPAD x LPAD
  T* sy = sr + LPAD * LPAD;                         // 32 x LPAD staging
  for (int u = blockIdx.x; u < nunits; u += gridDim.x) {
    const int b = unit_block[u];
    const int rows = B.rows[b];
    const int lb = B.lb[b];
    const int64_t r0 = B.arow[b] + (int64_t)unit_tile[u] * TR;
    const int i0 = unit_tile[u] * TR;
    for (int q = threadIdx.x; q < LPAD * LPAD; q += blockDim.x)
      sr[q] = (T)Rinv[(int64_t)b * LPAD * LPAD + q];
    __syncthreads();
    // each thread: one row (of up to 128) per pass, LPAD/2 columns per half-warp pairing
    for (int sub = 0; sub < TR; sub += 32) {
      for (int q = threadIdx.x; q < 32 * LPAD; q += blockDim.x) {
        const int rr = q / LPAD, jj = q % LPAD;
        sy[q] = (i0 + sub + rr < rows) ? Y[(r0 + sub + rr) * LPAD + jj] : T(0);
      }
      __syncthreads();
      for (int q = threadIdx.x; q < 32 * LPAD; q += blockDim.x) {
        const int rr = q / LPAD, j = q % LPAD;
        T a = T(0);
        if (j < lb)
          for (int i = 0; i <= j; ++i) a = fma(sy[rr * LPAD + i], sr[i * LPAD + j], a);
        const int irow = i0 + sub + rr;
        if (irow < rows) {
          Qf[(r0 + sub + rr) * LPAD + j] = a;
          if (St) St[(int64_t)j * B.Ktot + B.koff[b] + irow] = from_double<TB>((double)a);
        }
      }
      __syncthreads();
    }
  }
}

// ---------------------------------------------------------------------------
// Symmetric eigendecomposition of T_b (lb x lb, FP64) by cyclic Jacobi with a
// round-robin (tournament) ordering of disjoint pairs.  Writes the eigenvalues in
// descending order and the matching eigenvectors (columns of V, LPAD x LPAD).
// ---------------------------------------------------------------------------
template <int LPAD>
__global__ void __launch_bounds__(256) k_jacobi(Blocks B, const double* __restrict__ Tm, double* __restrict__ V,
                                                 double* __restrict__ evals, int max_sweeps) {
  extern __shared__ double sm[];
  double* A = sm;                     // LPAD x LPAD
  double* W = sm + LPAD * LPAD;       // eigenvectors
  __shared__ double cs[LPAD / 2], sn[LPAD / 2];
  __shared__ int pp[LPAD / 2], qq[LPAD / 2];
  __shared__ double off_s, tot_s;
  __shared__ int order[LPAD];
  const int b = blockIdx.x;
  const int lb = B.lb[b];
  const int n = (lb + 1) & ~1;  // even, a dummy index when lb is odd
  const double* Tb = Tm + (int64_t)b * LPAD * LPAD;
  for (int q = threadIdx.x; q < LPAD * LPAD; q += blockDim.x) {
    const int i = q / LPAD, j = q % LPAD;
    A[q] = (i < lb && j < lb) ? 0.5 * (Tb[i * LPAD + j] + Tb[j * LPAD + i]) : 0.0;
    W[q] = (i == j) ? 1.0 : 0.0;
  }
  __syncthreads();
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    if (threadIdx.x == 0) {
      double off = 0.0, tot = 0.0;
      for (int i = 0; i < lb; ++i)
        for (int j = 0; j < lb; ++j) {
          const double a = A[i * LPAD + j];
          tot += a * a;
          if (i != j) off += a * a;
        }
      off_s = off;
      tot_s = tot;
    }
    __syncthreads();
    if (!(off_s > 1e-30 * tot_s) || lb < 2) break;
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
        double c = 1.0, s = 0.0;
        if (z < lb) {
          const double apq = A[a * LPAD + z];
          if (apq != 0.0) {
            const double app = A[a * LPAD + a], aqq = A[z * LPAD + z];
            const double theta = (aqq - app) / (2.0 * apq);
            const double tt = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
            c = 1.0 / sqrt(tt * tt + 1.0);
            s = tt * c;
          }
        }
        cs[p] = c;
        sn[p] = s;
      }
      __syncthreads();
      // rows: A <- J^T A
      for (int q = threadIdx.x; q < (n / 2) * lb; q += blockDim.x) {
        const int p = q / lb, col = q % lb;
        const int a = pp[p], z = qq[p];
        if (z < lb) {
          const double c = cs[p], s = sn[p];
          const double x = A[a * LPAD + col], y = A[z * LPAD + col];
          A[a * LPAD + col] = c * x - s * y;
          A[z * LPAD + col] = s * x + c * y;
        }
      }
      __syncthreads();
      // columns: A <- A J, V <- V J
      for (int q = threadIdx.x; q < (n / 2) * lb; q += blockDim.x) {
        const int p = q / lb, row = q % lb;
        const int a = pp[p], z = qq[p];
        if (z < lb) {
          const double c = cs[p], s = sn[p];
          const double x = A[row * LPAD + a], y = A[row * LPAD + z];
          A[row * LPAD + a] = c * x - s * y;
          A[row * LPAD + z] = s * x + c * y;
          const double vx = W[row * LPAD + a], vy = W[row * LPAD + z];
          W[row * LPAD + a] = c * vx - s * vy;
          W[row * LPAD + z] = s * vx + c * vy;
        }
      }
      __syncthreads();
    }
  }
  // sort eigenvalues descending (selection by rank; ties broken by index)
  for (int i = threadIdx.x; i < lb; i += blockDim.x) {
    const double di = A[i * LPAD + i];
    int rank = 0;
    for (int j = 0; j < lb; ++j) {
      const double dj = A[j * LPAD + j];
      if (dj > di || (dj == di && j < i)) ++rank;
    }
    order[rank] = i;
  }
  __syncthreads();
  double* Vb = V + (int64_t)b * LPAD * LPAD;
  for (int q = threadIdx.x; q < LPAD * LPAD; q += blockDim.x) {
    const int i = q / LPAD, r = q % LPAD;  // Vb[i, r] = W[i, order[r]]
    Vb[q] = (r < lb && i < lb) ? W[i * LPAD + order[r]] : 0.0;
  }
  for (int r = threadIdx.x; r < LPAD; r += blockDim.x)
    evals[(int64_t)b * LPAD + r] = r < lb ? A[order[r] * LPAD + order[r]] : 0.0;
}

// Ritz vectors: Qout[v0 + i, r] = sum_j S[i, j] V[j, r] for r < kb (row panel S with
// stride lpad; output row stride k).  One CTA per 128-row tile.
template <class T, int LPAD>
__global__ void __launch_bounds__(256) k_ritz(Blocks B, const int32_t* __restrict__ unit_block,
                                               const int32_t* __restrict__ unit_tile, int nunits,
                                               const T* __restrict__ S, const double* __restrict__ V,
                                               T* __restrict__ Qout) {
  extern __shared__ uint8_t smraw[];
  T* sv = reinterpret_cast<T*>(smraw);  // LPAD x k
  const int k = B.k;
  for (int u = blockIdx.x; u < nunits; u += gridDim.x) {
    const int b = unit_block[u];
    const int rows = B.rows[b];
    const int lb = B.lb[b], kb = B.kb[b];
    const int i0 = unit_tile[u] * 128;
    const int64_t r0 = B.arow[b] + i0;
    for (int q = threadIdx.x; q < LPAD * k; q += blockDim.x) {
      const int j = q / k, r = q % k;
      sv[q] = (j < lb && r < kb) ? (T)V[(int64_t)b * LPAD * LPAD + j * LPAD + r] : T(0);
    }
    __syncthreads();
    for (int q = threadIdx.x; q < 128 * k; q += blockDim.x) {
      const int rr = q / k, r = q % k;
      if (i0 + rr < rows) {
        T a = T(0);
        for (int j = 0; j < lb; ++j) a = fma(S[(r0 + rr) * LPAD + j], sv[j * k + r], a);
        Qout[(B.v0[b] + i0 + rr) * k + r] = a;
      }
    }
    __syncthreads();
  }
}

}  // namespace rsvd
}  // namespace hgl
