// bcg.cu -- hgl_block_cg_solve: block CG with a shared Krylov space (O'Leary, Linear
// Algebra Appl. 29, 1980) on M F = lam Y, the columns taken in groups of s, FP64.
// Each group runs the block recurrences with its search block kept orthonormal and
// rank revealed (the breakdown-free form of Ji and Li, 2017), so that columns that
// converge or become dependent leave the search space instead of making P^T M P
// singular:
//   R = B - M F,  P = orth(R)
//   repeat:  Q = M P;  a = (P^T Q)^+ P^T R;  F += P a;  R -= Q a
//            stop the group when ||r_j|| <= tol ||b_j|| for all its columns
//            b = -(P^T Q)^+ Q^T R;  P = orth(R + P b)
// orth is CholeskyQR2 with unit-normalised columns and dropped pivots; ^+ solves on the
// kept pivots of a Cholesky factorisation.  All groups advance in the same launches;
// finished groups skip their updates.  Small s x s work runs one CTA per group.
#include <algorithm>
#include <cmath>
#include <vector>

#include "hgl_internal.cuh"

namespace hgl {
namespace {

constexpr int BCG_MAXS = 32;
constexpr int BCG_THREADS = 256;
constexpr int GRAM_SLAB = 2048;   // rows per partial Gram
constexpr int GRAM_TILE = 64;     // rows staged in shared memory at a time
// Relative pivot of a unit-diagonal Gram below which a direction is dropped.  The Gram
// squares the singular values of the block, so this drops directions whose singular
// value is below 1e-6 of the column norms: the same rank decision as an SVD-based
// orthonormalisation with a relative singular-value threshold of 1e-6.
constexpr double PIVOT_DROP = 1e-12;

struct DevBuf {
  void* p = nullptr;
  ~DevBuf() {
    if (p) cudaFree(p);
  }
};

// part[(slab * G + g) * s * s + i * s + j] = sum over the slab's rows r of
// A[r, g s + i] * B[r, g s + j]
__global__ void __launch_bounds__(BCG_THREADS)
k_grp_gram_part(int64_t n, int s, int G, const double* __restrict__ A, int64_t lda, const double* __restrict__ B,
                int64_t ldb, double* __restrict__ part) {
  __shared__ double sa[GRAM_TILE][BCG_MAXS + 1];
  __shared__ double sb[GRAM_TILE][BCG_MAXS + 1];
  const int slab = blockIdx.x, g = blockIdx.y;
  const int64_t r0 = (int64_t)slab * GRAM_SLAB;
  const int64_t r1 = n < r0 + GRAM_SLAB ? n : r0 + GRAM_SLAB;
  const int nout = s * s;
  double acc[(BCG_MAXS * BCG_MAXS) / BCG_THREADS];
#pragma unroll
  for (int q = 0; q < (BCG_MAXS * BCG_MAXS) / BCG_THREADS; ++q) acc[q] = 0.0;
  for (int64_t t0 = r0; t0 < r1; t0 += GRAM_TILE) {
    const int nr = (int)(r1 - t0 < GRAM_TILE ? r1 - t0 : GRAM_TILE);
    for (int q = threadIdx.x; q < GRAM_TILE * s; q += blockDim.x) {
      const int rr = q / s, i = q % s;
      const int64_t col = (int64_t)g * s + i;
      sa[rr][i] = rr < nr ? A[(t0 + rr) * lda + col] : 0.0;
      sb[rr][i] = rr < nr ? B[(t0 + rr) * ldb + col] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < (BCG_MAXS * BCG_MAXS) / BCG_THREADS; ++q) {
      const int o = threadIdx.x + BCG_THREADS * q;
      if (o < nout) {
        const int i = o / s, j = o % s;
        double x = 0.0;
        for (int rr = 0; rr < nr; ++rr) x = fma(sa[rr][i], sb[rr][j], x);
        acc[q] += x;
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < (BCG_MAXS * BCG_MAXS) / BCG_THREADS; ++q) {
    const int o = threadIdx.x + BCG_THREADS * q;
    if (o < nout) part[((int64_t)slab * G + g) * nout + o] = acc[q];
  }
}

// out[g * s * s + o] = sum of the slabs' partials in slab order
__global__ void k_grp_gram_reduce(int nslabs, int G, int s, const double* __restrict__ part, double* __restrict__ out) {
  const int nout = s * s;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < G * nout; q += gridDim.x * blockDim.x) {
    const int g = q / nout, o = q % nout;
    double x = 0.0;
    for (int sl = 0; sl < nslabs; ++sl) x += part[((int64_t)sl * G + g) * nout + o];
    out[q] = x;
  }
}

// Cholesky L L^T of the symmetrised s x s matrix in L (lower triangle used) with
// dropped pivots: a pivot <= drop * (largest diagonal) marks a direction outside the
// kept subspace (dead[j] = 1; its row and column of L become the identity's).
// One thread.
__device__ void chol_drop(double (*L)[BCG_MAXS + 1], int s, double drop, int* dead) {
  double dmax = 0.0;
  for (int i = 0; i < s; ++i) dmax = fmax(dmax, L[i][i]);
  for (int j = 0; j < s; ++j) {
    double d = L[j][j];
    for (int k = 0; k < j; ++k) d -= L[j][k] * L[j][k];
    if (!(d > drop * dmax) || !isfinite(d)) {
      dead[j] = 1;
      L[j][j] = 1.0;
      for (int i = j + 1; i < s; ++i) L[i][j] = 0.0;
      for (int k = 0; k < j; ++k) L[j][k] = 0.0;
      continue;
    }
    dead[j] = 0;
    const double ljj = sqrt(d);
    L[j][j] = ljj;
    for (int i = j + 1; i < s; ++i) {
      double x = L[i][j];
      for (int k = 0; k < j; ++k) x -= L[i][k] * L[j][k];
      L[i][j] = x / ljj;
    }
  }
}

// out_g = sign * A_g^+ RHS_g for every active group (s x s each): A_g = P^T Q, solved by
// Cholesky with dropped pivots (zero rows of the result there).  Inactive groups get 0.
__global__ void __launch_bounds__(BCG_THREADS)
k_grp_solve(int s, const double* __restrict__ A, const double* __restrict__ rhs, double sign,
            const int32_t* __restrict__ active, double* __restrict__ out) {
  __shared__ double L[BCG_MAXS][BCG_MAXS + 1];
  __shared__ double X[BCG_MAXS][BCG_MAXS + 1];
  __shared__ int dead[BCG_MAXS];
  const int g = blockIdx.x;
  const int nout = s * s;
  const double* Ag = A + (int64_t)g * nout;
  const double* Rg = rhs + (int64_t)g * nout;
  double* Og = out + (int64_t)g * nout;
  if (!active[g]) {
    for (int o = threadIdx.x; o < nout; o += blockDim.x) Og[o] = 0.0;
    return;
  }
  for (int o = threadIdx.x; o < nout; o += blockDim.x) {
    const int i = o / s, j = o % s;
    L[i][j] = 0.5 * (Ag[i * s + j] + Ag[j * s + i]);
    X[i][j] = Rg[o];
  }
  __syncthreads();
  if (threadIdx.x == 0) chol_drop(L, s, PIVOT_DROP, dead);
  __syncthreads();
  // one right-hand-side column per thread: L y = rhs, then L^T x = y (dead entries 0)
  for (int cidx = threadIdx.x; cidx < s; cidx += blockDim.x) {
    for (int i = 0; i < s; ++i) {
      double y = X[i][cidx];
      for (int k = 0; k < i; ++k) y -= L[i][k] * X[k][cidx];
      X[i][cidx] = dead[i] ? 0.0 : y / L[i][i];
    }
    for (int i = s - 1; i >= 0; --i) {
      double x = X[i][cidx];
      for (int k = i + 1; k < s; ++k) x -= L[k][i] * X[k][cidx];
      X[i][cidx] = dead[i] ? 0.0 : x / L[i][i];
    }
  }
  __syncthreads();
  for (int o = threadIdx.x; o < nout; o += blockDim.x) {
    const int i = o / s, j = o % s;
    Og[o] = sign * X[i][j];
  }
}

// CholeskyQR step for every active group: from the Gram W^T W, coef = D L^-T with
// D = diag(1 / ||w_i||) (0 for a zero column) and L L^T = D W^T W D (dropped pivots give
// zero rows and columns), so that W coef has orthonormal (or zero) columns.
__global__ void __launch_bounds__(BCG_THREADS)
k_grp_orth_coef(int s, const double* __restrict__ gram, const int32_t* __restrict__ active,
                double* __restrict__ coef) {
  __shared__ double L[BCG_MAXS][BCG_MAXS + 1];
  __shared__ double Li[BCG_MAXS][BCG_MAXS + 1];
  __shared__ double sc[BCG_MAXS];
  __shared__ int dead[BCG_MAXS];
  const int g = blockIdx.x;
  const int nout = s * s;
  const double* Gg = gram + (int64_t)g * nout;
  double* Cg = coef + (int64_t)g * nout;
  if (!active[g]) {
    for (int o = threadIdx.x; o < nout; o += blockDim.x) Cg[o] = 0.0;
    return;
  }
  for (int i = threadIdx.x; i < s; i += blockDim.x) {
    const double d = Gg[i * s + i];
    sc[i] = (d > 0.0 && isfinite(d)) ? 1.0 / sqrt(d) : 0.0;
  }
  __syncthreads();
  for (int o = threadIdx.x; o < nout; o += blockDim.x) {
    const int i = o / s, j = o % s;
    L[i][j] = sc[i] * sc[j] * 0.5 * (Gg[i * s + j] + Gg[j * s + i]);
    Li[i][j] = 0.0;
  }
  __syncthreads();
  if (threadIdx.x == 0) chol_drop(L, s, PIVOT_DROP, dead);
  __syncthreads();
  // L^-1 column by column (lower triangular; dead rows and columns stay 0)
  for (int cidx = threadIdx.x; cidx < s; cidx += blockDim.x) {
    if (dead[cidx]) continue;
    for (int i = cidx; i < s; ++i) {
      if (dead[i]) continue;
      double x = i == cidx ? 1.0 : 0.0;
      for (int k = cidx; k < i; ++k) x -= L[i][k] * Li[k][cidx];
      Li[i][cidx] = x / L[i][i];
    }
  }
  __syncthreads();
  // coef[i][j] = sc[i] * (L^-T)[i][j] = sc[i] * Li[j][i]
  for (int o = threadIdx.x; o < nout; o += blockDim.x) {
    const int i = o / s, j = o % s;
    Cg[o] = sc[i] * Li[j][i];
  }
}

// Out[r, g s + j] = (Y ? Y[r, g s + j] : 0) + sign * sum_i X[r, g s + i] coef_g[i][j]
// for the rows of this block and the active groups (grid: row blocks x groups; a thread
// per row; Out may be Y, each thread reading its segment before writing it).
__global__ void __launch_bounds__(BCG_THREADS)
k_grp_update(int64_t n, int s, const double* __restrict__ X, int64_t ldx, const double* __restrict__ coef,
             const double* Y, int64_t ldy, double sign, const int32_t* __restrict__ active, double* Out, int64_t ldo) {
  __shared__ double C[BCG_MAXS][BCG_MAXS + 1];
  const int g = blockIdx.y;
  if (!active[g]) return;
  const int nout = s * s;
  for (int o = threadIdx.x; o < nout; o += blockDim.x) C[o / s][o % s] = coef[(int64_t)g * nout + o];
  __syncthreads();
  const int64_t c0 = (int64_t)g * s;
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
    double x[BCG_MAXS];
    for (int i = 0; i < s; ++i) x[i] = X[r * ldx + c0 + i];
    for (int j = 0; j < s; ++j) {
      double acc = Y ? Y[r * ldy + c0 + j] : 0.0;
      double t = 0.0;
      for (int i = 0; i < s; ++i) t = fma(x[i], C[i][j], t);
      Out[r * ldo + c0 + j] = fma(sign, t, acc);
    }
  }
}

// part[block * cp + j] = sum over this block's rows of A[r, j]^2 (columns j < cp)
__global__ void __launch_bounds__(BCG_THREADS)
k_col_sumsq_part(int64_t n, int cp, const double* __restrict__ A, int64_t lda, double* __restrict__ part) {
  for (int j = threadIdx.x; j < cp; j += blockDim.x) {
    double x = 0.0;
    for (int64_t r = blockIdx.x; r < n; r += gridDim.x) {
      const double a = A[r * lda + j];
      x = fma(a, a, x);
    }
    part[(int64_t)blockIdx.x * cp + j] = x;
  }
}

__global__ void k_col_sumsq_reduce(int nblocks, int cp, const double* __restrict__ part, double* __restrict__ out) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < cp; j += gridDim.x * blockDim.x) {
    double x = 0.0;
    for (int b = 0; b < nblocks; ++b) x += part[(int64_t)b * cp + j];
    out[j] = x;
  }
}

// B = lam Y on the first c columns, 0 on the padding; F0 likewise from F (or 0)
__global__ void k_bcg_load(int64_t n, int c, int cp, const double* __restrict__ Y, int64_t ldy, double lam,
                           const double* __restrict__ F, int64_t ldf, double* __restrict__ Bp,
                           double* __restrict__ Fp, int64_t ldp) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n * cp; q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = q / cp;
    const int j = (int)(q % cp);
    Bp[r * ldp + j] = j < c ? lam * Y[r * ldy + j] : 0.0;
    Fp[r * ldp + j] = (j < c && F) ? F[r * ldf + j] : 0.0;
  }
}

// R = B - MF (MF given), or F[:, :c] = Fp[:, :c]
__global__ void k_bcg_sub(int64_t n, int cp, const double* __restrict__ Bp, const double* __restrict__ MF,
                          double* __restrict__ R, int64_t ldp) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n * cp; q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = q / cp;
    const int j = (int)(q % cp);
    R[r * ldp + j] = Bp[r * ldp + j] - MF[r * ldp + j];
  }
}

__global__ void k_bcg_store(int64_t n, int c, const double* __restrict__ Fp, int64_t ldp, double* __restrict__ F,
                            int64_t ldf) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n * c; q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = q / c;
    const int j = (int)(q % c);
    F[r * ldf + j] = Fp[r * ldp + j];
  }
}

}  // namespace
}  // namespace hgl

extern "C" hgl_status hgl_block_cg_solve(const hgl_graph* gc, const double* w, double lam, const double* Y,
                                         int64_t ldy, double* F, int64_t ldf, int32_t c, int32_t s, double tol,
                                         int32_t max_iter, int32_t flags, double* relres, int32_t* iters,
                                         void* stream) {
  using namespace hgl;
  if (!gc || !w) return record_error(HGL_ERR_INVALID_ARG, "graph or w is NULL");
  if (c < 1) return record_error(HGL_ERR_INVALID_ARG, "c must be >= 1");
  if (s < 1 || s > BCG_MAXS) return record_error(HGL_ERR_INVALID_ARG, "s must be in [1, %d]", BCG_MAXS);
  if (!(lam > 0.0)) return record_error(HGL_ERR_INVALID_ARG, "lam must be positive");
  if (!(tol > 0.0)) return record_error(HGL_ERR_INVALID_ARG, "tol must be positive");
  if (max_iter < 1) return record_error(HGL_ERR_INVALID_ARG, "max_iter must be >= 1");
  HGL_TRY(check_panel(Y, ldy, c, 8, "Y"));
  HGL_TRY(check_panel(F, ldf, c, 8, "F"));
  hgl_graph* g = const_cast<hgl_graph*>(gc);
  cudaStream_t st = as_stream(stream);
  const int64_t n = g->n;
  const int G = (c + s - 1) / s;
  const int cp = G * s;
  const int64_t ldp = (cp + 1) / 2 * 2;  // even: 16-byte rows for the operator's vector loads
  HGL_TRY(degrees_launch(g, w, st));

  // work: B, F, R, P, Q, W, T panels (n x ldp FP64), Gram partials and small matrices
  const int nslabs = (int)std::max<int64_t>(1, (n + GRAM_SLAB - 1) / GRAM_SLAB);
  const int nsq = g->num_sms * 4;
  const size_t panel = (size_t)n * ldp;
  const size_t small = (size_t)G * s * s;
  DevBuf buf;
  const size_t bytes = sizeof(double) * (7 * panel + (size_t)nslabs * small + 6 * small + (size_t)nsq * cp + cp) +
                       sizeof(int32_t) * G;
  HGL_CHECK_CUDA(cudaMalloc(&buf.p, bytes));
  double* Bp = static_cast<double*>(buf.p);
  double* Fp = Bp + panel;
  double* R = Fp + panel;
  double* P = R + panel;
  double* Q = P + panel;
  double* W = Q + panel;
  double* T = W + panel;
  double* gpart = T + panel;
  double* PQ = gpart + (size_t)nslabs * small;
  double* PR = PQ + small;
  double* QZ = PR + small;
  double* coefA = QZ + small;
  double* coefB = coefA + small;
  double* gram = coefB + small;
  double* sqpart = gram + small;
  double* colsq = sqpart + (size_t)nsq * cp;
  int32_t* d_active = reinterpret_cast<int32_t*>(colsq + cp);
  // all seven panels start at zero, padding columns (j >= cp) included: a group that
  // never becomes active keeps zero columns in the search, product and scratch panels,
  // and the operator's 16-byte loads read defined values in the padding
  HGL_CHECK_CUDA(cudaMemsetAsync(Bp, 0, sizeof(double) * 7 * panel, st));

  const int vec_blocks = g->num_sms * 8;
  auto gram_of = [&](const double* A, const double* Bm, double* out) -> hgl_status {
    count_launch(2);
    k_grp_gram_part<<<dim3(nslabs, G), BCG_THREADS, 0, st>>>(n, s, G, A, ldp, Bm, ldp, gpart);
    k_grp_gram_reduce<<<(int)std::min<size_t>((small + 255) / 256, 1024), 256, 0, st>>>(nslabs, G, s, gpart, out);
    HGL_CHECK_CUDA(cudaGetLastError());
    return HGL_OK;
  };
  const int upd_rows = (int)std::max<int64_t>(1, std::min<int64_t>((n + BCG_THREADS - 1) / BCG_THREADS, 4096));
  auto update = [&](const double* X, const double* coef, const double* Yin, double sign, double* Out) -> hgl_status {
    count_launch();
    k_grp_update<<<dim3(upd_rows, G), BCG_THREADS, 0, st>>>(n, s, X, ldp, coef, Yin, ldp, sign, d_active, Out, ldp);
    HGL_CHECK_CUDA(cudaGetLastError());
    return HGL_OK;
  };
  auto apply_m = [&](const double* X, double* Z) -> hgl_status {  // Z = M X = (1+lam) X - Theta X
    OpCall cl{};
    cl.g = g;
    cl.xdt = HGL_FP64;
    cl.zdt = HGL_FP64;
    cl.X = X;
    cl.ldx = ldp;
    cl.Z = Z;
    cl.ldz = ldp;
    cl.c = cp;
    cl.a = 1.0 + lam;
    cl.b = -1.0;
    cl.epi = EPI_PLAIN;
    cl.chunk_cols = g->chunk_cols;
    return op_launch(cl, st, nullptr);
  };
  std::vector<double> hsq(cp), bnorm(cp);
  auto col_norms = [&](const double* A, std::vector<double>& out) -> hgl_status {
    count_launch(2);
    k_col_sumsq_part<<<nsq, BCG_THREADS, 0, st>>>(n, cp, A, ldp, sqpart);
    k_col_sumsq_reduce<<<(cp + 255) / 256, 256, 0, st>>>(nsq, cp, sqpart, colsq);
    HGL_CHECK_CUDA(cudaGetLastError());
    HGL_CHECK_CUDA(cudaMemcpyAsync(out.data(), colsq, sizeof(double) * cp, cudaMemcpyDeviceToHost, st));
    HGL_CHECK_CUDA(cudaStreamSynchronize(st));
    for (int j = 0; j < cp; ++j) out[j] = std::sqrt(out[j]);
    return HGL_OK;
  };
  std::vector<int32_t> active(G, 0), its(G, 0);
  // per group: active while some column with ||b_j|| > 0 has ||r_j|| > tol ||b_j||
  auto set_active = [&](const std::vector<double>& rn, bool only_active) -> bool {
    bool any = false;
    for (int gi = 0; gi < G; ++gi) {
      if (only_active && !active[gi]) continue;
      int a = 0;
      for (int j = gi * s; j < gi * s + s && j < c; ++j)
        if (bnorm[j] > 0.0 && !(rn[j] <= tol * bnorm[j])) a = 1;
      active[gi] = a;
      any = any || a;
    }
    return any;
  };
  auto push_active = [&]() -> hgl_status {
    HGL_CHECK_CUDA(cudaMemcpyAsync(d_active, active.data(), sizeof(int32_t) * G, cudaMemcpyHostToDevice, st));
    HGL_CHECK_CUDA(cudaStreamSynchronize(st));  // the host vector is rewritten next
    return HGL_OK;
  };
  // orth(W) -> P for the active groups: two CholeskyQR steps through T
  auto orth = [&](const double* Win) -> hgl_status {
    HGL_TRY(gram_of(Win, Win, gram));
    count_launch();
    k_grp_orth_coef<<<G, BCG_THREADS, 0, st>>>(s, gram, d_active, coefA);
    HGL_TRY(update(Win, coefA, nullptr, 1.0, T));
    HGL_TRY(gram_of(T, T, gram));
    count_launch();
    k_grp_orth_coef<<<G, BCG_THREADS, 0, st>>>(s, gram, d_active, coefA);
    return update(T, coefA, nullptr, 1.0, P);
  };

  // R = B - M F0, P = orth(R)
  count_launch();
  k_bcg_load<<<vec_blocks, 256, 0, st>>>(n, c, cp, Y, ldy, lam, (flags & HGL_SOLVE_WARM_START) ? F : nullptr, ldf,
                                         Bp, Fp, ldp);
  HGL_CHECK_CUDA(cudaGetLastError());
  HGL_TRY(col_norms(Bp, bnorm));
  // a column with a zero right-hand side has the exact solution 0 (M is nonsingular):
  // a warm start there is discarded, so the column starts (and stays) converged
  if (flags & HGL_SOLVE_WARM_START)
    for (int j = 0; j < c; ++j)
      if (bnorm[j] == 0.0)
        HGL_CHECK_CUDA(cudaMemset2DAsync(Fp + j, sizeof(double) * ldp, 0, sizeof(double), n, st));
  HGL_TRY(apply_m(Fp, Q));
  count_launch();
  k_bcg_sub<<<vec_blocks, 256, 0, st>>>(n, cp, Bp, Q, R, ldp);
  HGL_CHECK_CUDA(cudaGetLastError());
  HGL_TRY(col_norms(R, hsq));
  bool any = set_active(hsq, false);
  HGL_TRY(push_active());
  if (any) HGL_TRY(orth(R));
  for (int it = 0; it < max_iter && any; ++it) {
    HGL_TRY(apply_m(P, Q));
    HGL_TRY(gram_of(P, Q, PQ));
    HGL_TRY(gram_of(P, R, PR));
    count_launch();
    k_grp_solve<<<G, BCG_THREADS, 0, st>>>(s, PQ, PR, 1.0, d_active, coefA);
    HGL_TRY(update(P, coefA, Fp, 1.0, Fp));   // F += P a
    HGL_TRY(update(Q, coefA, R, -1.0, R));    // R -= Q a
    for (int gi = 0; gi < G; ++gi) its[gi] += active[gi];
    HGL_TRY(col_norms(R, hsq));
    any = set_active(hsq, true);
    HGL_TRY(push_active());
    if (!any) break;
    HGL_TRY(gram_of(Q, R, QZ));
    count_launch();
    k_grp_solve<<<G, BCG_THREADS, 0, st>>>(s, PQ, QZ, -1.0, d_active, coefB);
    HGL_TRY(update(P, coefB, R, 1.0, W));     // W = R + P b
    HGL_TRY(orth(W));                         // P = orth(W)
  }
  // F out; the true relative residual lam Y - M F per column; iterations per group
  count_launch();
  k_bcg_store<<<vec_blocks, 256, 0, st>>>(n, c, Fp, ldp, F, ldf);
  HGL_CHECK_CUDA(cudaGetLastError());
  HGL_TRY(apply_m(Fp, Q));
  count_launch();
  k_bcg_sub<<<vec_blocks, 256, 0, st>>>(n, cp, Bp, Q, R, ldp);
  HGL_CHECK_CUDA(cudaGetLastError());
  HGL_TRY(col_norms(R, hsq));
  std::vector<double> rel(c);
  int missed = 0, nonfinite = 0;
  for (int j = 0; j < c; ++j) {
    // relative residual; for a zero right-hand side the absolute ||r_j|| (0 after the
    // column was zeroed, so such a column always meets the tolerance)
    rel[j] = bnorm[j] > 0.0 ? hsq[j] / bnorm[j] : hsq[j];
    if (!std::isfinite(rel[j]) || !std::isfinite(bnorm[j])) nonfinite++;
    else if (rel[j] > tol) missed++;
  }
  if (relres) HGL_CHECK_CUDA(cudaMemcpyAsync(relres, rel.data(), sizeof(double) * c, cudaMemcpyHostToDevice, st));
  if (iters) HGL_CHECK_CUDA(cudaMemcpyAsync(iters, its.data(), sizeof(int32_t) * G, cudaMemcpyHostToDevice, st));
  HGL_CHECK_CUDA(cudaStreamSynchronize(st));
  if (nonfinite) return record_error(HGL_ERR_NONFINITE, "non-finite value in %d column(s)", nonfinite);
  if (missed) return record_error(HGL_ERR_NOT_CONVERGED, "%d of %d columns missed the tolerance", missed, c);
  return HGL_OK;
}
