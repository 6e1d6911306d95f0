// precond.cu -- the block preconditioner built by hgl_block_rsvd (Section 3, Eq. 15):
//   z_b = r_b / (1+lam) + Q_b diag(g_b) Q_b^T r_b,   g = ev / ((1+lam)(1+lam-ev)),
// applied block by block to an n x c panel: C_b = diag(g_b) Q_b^T R_b (k x c, reduced
// over the block's rows by one CTA per block and column chunk), then
// Z_b = R_b/(1+lam) + Q_b C_b (one CTA per 32-row tile and column chunk).
#include <algorithm>
#include <cstring>
#include <vector>

#include "rsvd_kernels.cuh"
#include "precond.cuh"
#include "solver.cuh"

namespace hgl {
namespace {

constexpr int CW = 64;  // columns per CTA

__global__ void k_gains(int nb, int k, int lpad, const double* __restrict__ ev_in, const int32_t* __restrict__ kb,
                        double lam, double* __restrict__ ev_out, double* __restrict__ gain) {
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nb * k; q += gridDim.x * blockDim.x) {
    const int b = q / k, r = q % k;
    double e = r < kb[b] ? ev_in[(int64_t)b * lpad + r] : 0.0;
    e = e < 0.0 ? 0.0 : (e > 1.0 ? 1.0 : e);  // spec(Theta_bb) lies in [0, 1]
    ev_out[q] = e;
    gain[q] = r < kb[b] ? e / ((1.0 + lam) * (1.0 + lam - e)) : 0.0;
  }
}

template <class T> struct AccT { using type = float; };
template <> struct AccT<double> { using type = double; };

// Column chunk per CTA and rows per tile of the two kernels.  Threads form 8 rows of
// 32 lanes; a thread owns KP/8 (projection) or 8 (expansion) output rows and
// CW/32 columns, so every shared-memory load feeds several FMAs.
template <class TP> struct ApplyShape {
  static constexpr int CW = sizeof(TP) == 8 ? 64 : 128;
  static constexpr int RT = 32;   // rows per tile in the projection
  static constexpr int UR = 64;   // rows per expansion unit
  static constexpr int KC = 16;   // rank rows of C staged at a time
};

// C[b, r, col] = gain[b, r] * sum_i Q[v0+i, r] R[v0+i, col]   (grid: blocks x column chunks)
template <class TP, class TQ, int KP>
__global__ void __launch_bounds__(256)
k_precond_proj(int nb, const int64_t* __restrict__ v0, const int32_t* __restrict__ rows, const TQ* __restrict__ Q,
               int k, const TP* __restrict__ R, int64_t ldr, int c, const double* __restrict__ gain,
               typename AccT<TP>::type* __restrict__ C, const int32_t* __restrict__ run_flag) {
  if (run_flag && *run_flag == 0) return;
  using A = typename AccT<TP>::type;
  using S = ApplyShape<TP>;
  constexpr int CW = S::CW, RT = S::RT, NR = KP / 8, NC = CW / 32;
  extern __shared__ __align__(16) uint8_t smraw[];
  A* sq = reinterpret_cast<A*>(smraw);   // RT x KP
  A* sr = sq + RT * KP;                  // RT x CW
  const int b = blockIdx.x;
  const int c0 = blockIdx.y * CW;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int64_t base = v0[b];
  const int nrows = rows[b];
  A acc[NR][NC];
#pragma unroll
  for (int a = 0; a < NR; ++a)
#pragma unroll
    for (int cc = 0; cc < NC; ++cc) acc[a][cc] = A(0);
  for (int t0 = 0; t0 < nrows; t0 += RT) {
    for (int q = threadIdx.x; q < RT * KP; q += blockDim.x) {
      const int i = q / KP, r = q % KP;
      sq[q] = (t0 + i < nrows && r < k) ? (A)Q[(base + t0 + i) * k + r] : A(0);
    }
    for (int q = threadIdx.x; q < RT * CW; q += blockDim.x) {
      const int i = q / CW, j = q % CW;
      sr[q] = (t0 + i < nrows && c0 + j < c) ? (A)R[(base + t0 + i) * ldr + c0 + j] : A(0);
    }
    __syncthreads();
#pragma unroll 2
    for (int i = 0; i < RT; ++i) {
      A rv[NC], qv[NR];
#pragma unroll
      for (int cc = 0; cc < NC; ++cc) rv[cc] = sr[i * CW + tx + 32 * cc];
#pragma unroll
      for (int a = 0; a < NR; ++a) qv[a] = sq[i * KP + ty * NR + a];
#pragma unroll
      for (int a = 0; a < NR; ++a)
#pragma unroll
        for (int cc = 0; cc < NC; ++cc) acc[a][cc] = fma(qv[a], rv[cc], acc[a][cc]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < NR; ++a) {
    const int r = ty * NR + a;
    if (r < k) {
      const A gr = (A)gain[(int64_t)b * k + r];
#pragma unroll
      for (int cc = 0; cc < NC; ++cc) {
        const int col = c0 + tx + 32 * cc;
        if (col < c) C[((int64_t)b * k + r) * c + col] = gr * acc[a][cc];
      }
    }
  }
}

// Z = R / (1+lam) + Q C_b on one 64-row unit of a block and one column chunk
template <class TP, class TQ, int KP>
__global__ void __launch_bounds__(256)
k_precond_expand(const int32_t* __restrict__ unit_block, const int32_t* __restrict__ unit_tile, int nunits,
                 const int64_t* __restrict__ v0, const int32_t* __restrict__ rows, const TQ* __restrict__ Q, int k,
                 const TP* __restrict__ R, int64_t ldr, TP* __restrict__ Z, int64_t ldz, int c, double inv1l,
                 const typename AccT<TP>::type* __restrict__ C, const int32_t* __restrict__ run_flag) {
  if (run_flag && *run_flag == 0) return;
  using A = typename AccT<TP>::type;
  using S = ApplyShape<TP>;
  constexpr int CW = S::CW, UR = S::UR, KC = S::KC, NR = UR / 8, NC = CW / 32;
  static_assert(KP % KC == 0, "rank chunk must divide the padded rank");
  extern __shared__ __align__(16) uint8_t smraw[];
  A* sq = reinterpret_cast<A*>(smraw);   // UR x (KP + 1)
  A* sc = sq + UR * (KP + 1);             // KC x CW
  const int c0 = blockIdx.y * CW;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  for (int u = blockIdx.x; u < nunits; u += gridDim.x) {
    const int b = unit_block[u];
    const int i0 = unit_tile[u] * UR;
    const int nrows = rows[b];
    const int64_t base = v0[b] + i0;
    for (int q = threadIdx.x; q < UR * KP; q += blockDim.x) {
      const int i = q / KP, r = q % KP;
      sq[i * (KP + 1) + r] = (i0 + i < nrows && r < k) ? (A)Q[(base + i) * k + r] : A(0);
    }
    A acc[NR][NC];
#pragma unroll
    for (int a = 0; a < NR; ++a)
#pragma unroll
      for (int cc = 0; cc < NC; ++cc) {
        const int i = ty * NR + a, col = c0 + tx + 32 * cc;
        acc[a][cc] = (i0 + i < nrows && col < c) ? (A)R[(base + i) * ldr + col] * (A)inv1l : A(0);
      }
    for (int r0 = 0; r0 < KP; r0 += KC) {
      __syncthreads();
      for (int q = threadIdx.x; q < KC * CW; q += blockDim.x) {
        const int r = q / CW, j = q % CW;
        sc[q] = (r0 + r < k && c0 + j < c) ? C[((int64_t)b * k + r0 + r) * c + c0 + j] : A(0);
      }
      __syncthreads();
#pragma unroll 4
      for (int r = 0; r < KC; ++r) {
        A cv[NC];
#pragma unroll
        for (int cc = 0; cc < NC; ++cc) cv[cc] = sc[r * CW + tx + 32 * cc];
#pragma unroll
        for (int a = 0; a < NR; ++a) {
          const A qv = sq[(ty * NR + a) * (KP + 1) + r0 + r];
#pragma unroll
          for (int cc = 0; cc < NC; ++cc) acc[a][cc] = fma(qv, cv[cc], acc[a][cc]);
        }
      }
    }
#pragma unroll
    for (int a = 0; a < NR; ++a) {
      const int i = ty * NR + a;
      if (i0 + i < nrows)
#pragma unroll
        for (int cc = 0; cc < NC; ++cc) {
          const int col = c0 + tx + 32 * cc;
          if (col < c) Z[(base + i) * ldz + col] = (TP)acc[a][cc];
        }
    }
    __syncthreads();
  }
}

template <class TP, class TQ>
hgl_status apply_typed(hgl_precond* P, const TP* R, int64_t ldr, TP* Z, int64_t ldz, int c, cudaStream_t st,
                       const int32_t* run_flag) {
  using A = typename AccT<TP>::type;
  using S = ApplyShape<TP>;
  ProfScope prof(HGL_PROF_PRECOND, st);
  hgl_status s = HGL_OK;
  A* C = static_cast<A*>(buffer_get(P->cbuf, sizeof(A) * (size_t)P->nb * P->k * c, &s));
  if (!C) return s;
  const int kp = (int)((P->k + 15) / 16 * 16);
  const int sms = device_sm_count();
  dim3 g1(P->nb, (c + S::CW - 1) / S::CW);
  dim3 g2(std::min(P->nunits, sms * 8), (c + S::CW - 1) / S::CW);
  const TQ* Q = static_cast<const TQ*>(P->Q);
  const double inv1l = 1.0 / (1.0 + P->lam);
#define HGL_KP_CASE(KPV)                                                                                         \
  case KPV: {                                                                                                    \
    const size_t sm1 = sizeof(A) * (size_t)S::RT * (KPV + S::CW);                                                \
    const size_t sm2 = sizeof(A) * ((size_t)S::UR * (KPV + 1) + (size_t)S::KC * S::CW);                          \
    HGL_CHECK_CUDA(cudaFuncSetAttribute(k_precond_proj<TP, TQ, KPV>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                        (int)sm1));                                                              \
    HGL_CHECK_CUDA(cudaFuncSetAttribute(k_precond_expand<TP, TQ, KPV>,                                           \
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm2));                 \
    hgl::count_launch(2);                                                                                        \
    k_precond_proj<TP, TQ, KPV><<<g1, 256, sm1, st>>>(P->nb, P->d_v0, P->d_rows, Q, P->k, R, ldr, c, P->gain, C, \
                                                      run_flag);                                                 \
    k_precond_expand<TP, TQ, KPV><<<g2, 256, sm2, st>>>(P->unit_block, P->unit_tile, P->nunits, P->d_v0,        \
                                                        P->d_rows, Q, P->k, R, ldr, Z, ldz, c, inv1l, C,         \
                                                        run_flag);                                               \
  } break;
  switch (kp) {
    HGL_KP_CASE(16)
    HGL_KP_CASE(32)
    HGL_KP_CASE(48)
    HGL_KP_CASE(64)
    HGL_KP_CASE(80)
    default:
      HGL_KP_CASE(96)
  }
#undef HGL_KP_CASE
  HGL_CHECK_CUDA(cudaGetLastError());
  return HGL_OK;
}

template <class TO>
__global__ void k_export_q(const float* __restrict__ Qf, const double* __restrict__ Qd, int64_t first, int64_t rows,
                           int k, TO* __restrict__ out) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < rows * k; q += (int64_t)gridDim.x * blockDim.x)
    out[q] = Qf ? (TO)Qf[first * k + q] : (TO)Qd[first * k + q];
}

}  // namespace

hgl_status precond_gains_launch(hgl_precond* P, const double* ev_lpad, int lpad, cudaStream_t st) {
  hgl::count_launch(); k_gains<<<(P->nb * P->k + 255) / 256, 256, 0, st>>>(P->nb, P->k, lpad, ev_lpad, P->d_kb, P->lam, P->ev, P->gain);
  HGL_CHECK_CUDA(cudaGetLastError());
  return HGL_OK;
}

hgl_status precond_check(const hgl_precond* P, const hgl_graph* g, double lam) {
  if (!P) return record_error(HGL_ERR_INVALID_ARG, "preconditioner is NULL");
  if (P->n != g->n) return record_error(HGL_ERR_INVALID_ARG, "preconditioner was built for another graph size");
  if (P->lam != lam)
    return record_error(HGL_ERR_INVALID_ARG, "preconditioner was built for lam = %g, the solve uses %g", P->lam, lam);
  return HGL_OK;
}

hgl_status precond_apply_launch(const hgl_precond* Pc, const hgl_graph* g, const void* R, int64_t ldr, void* Z,
                                int64_t ldz, int c, int dt, double* partials_rz, cudaStream_t st, int* rows,
                                const int32_t* run_flag) {
  hgl_precond* P = const_cast<hgl_precond*>(Pc);
  const bool f32q = P->dtype == HGL_BF16;
  if (dt == HGL_FP64) {
    if (f32q)
      HGL_TRY((apply_typed<double, float>(P, (const double*)R, ldr, (double*)Z, ldz, c, st, run_flag)));
    else
      HGL_TRY((apply_typed<double, double>(P, (const double*)R, ldr, (double*)Z, ldz, c, st, run_flag)));
  } else if (dt == HGL_FP32) {
    if (f32q)
      HGL_TRY((apply_typed<float, float>(P, (const float*)R, ldr, (float*)Z, ldz, c, st, run_flag)));
    else
      HGL_TRY((apply_typed<float, double>(P, (const float*)R, ldr, (float*)Z, ldz, c, st, run_flag)));
  } else {
    return record_error(HGL_ERR_INVALID_ARG, "preconditioner panels must be FP64 or FP32");
  }
  if (partials_rz) HGL_TRY(panel_dot_launch(g, c, dt, R, ldr, Z, ldz, partials_rz, st, rows));
  return HGL_OK;
}

}  // namespace hgl

extern "C" hgl_status hgl_block_rsvd(const hgl_graph* g, const double* w, double lam, const int64_t* block_ptr,
                                     int32_t nblocks, int32_t k, int32_t p, int32_t q, uint64_t seed,
                                     hgl_dtype gemm_dtype, void* stream, hgl_precond** out) {
  if (!out) return hgl::record_error(HGL_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!g || !w) return hgl::record_error(HGL_ERR_INVALID_ARG, "graph or w is NULL");
  if (!(lam > 0.0)) return hgl::record_error(HGL_ERR_INVALID_ARG, "lam must be positive");
  return hgl::precond_build(g, w, lam, block_ptr, nblocks, k, p, q, seed, gemm_dtype, hgl::as_stream(stream), out,
                            false);
}

extern "C" void hgl_precond_destroy(hgl_precond* P) {
  if (!P) return;
  cudaFree(P->dev);
  hgl::buffer_free(P->cbuf);
  delete P;
}

extern "C" hgl_status hgl_precond_export(const hgl_precond* P, int32_t b, double* Q, double* ev, int32_t* kb,
                                         void* stream) {
  if (!P) return hgl::record_error(HGL_ERR_INVALID_ARG, "preconditioner is NULL");
  if (b < 0 || b >= P->nb) return hgl::record_error(HGL_ERR_INVALID_ARG, "block index out of range");
  cudaStream_t st = hgl::as_stream(stream);
  const int64_t first = P->bptr[b], rows = P->bptr[b + 1] - P->bptr[b];
  if (kb) *kb = P->kb[b];
  if (Q) {
    hgl::count_launch();
    if (P->dtype == HGL_BF16)
      hgl::k_export_q<double><<<256, 256, 0, st>>>(static_cast<const float*>(P->Q), nullptr, first, rows, P->k, Q);
    else
      hgl::k_export_q<double><<<256, 256, 0, st>>>(nullptr, static_cast<const double*>(P->Q), first, rows, P->k, Q);
    HGL_CHECK_CUDA(cudaGetLastError());
  }
  if (ev) HGL_CHECK_CUDA(cudaMemcpyAsync(ev, P->ev + (int64_t)b * P->k, sizeof(double) * P->k,
                                         cudaMemcpyDeviceToDevice, st));
  return HGL_OK;
}

extern "C" hgl_status hgl_precond_apply(const hgl_precond* P, const void* R, int64_t ldr, void* Z, int64_t ldz,
                                        int32_t c, hgl_dtype dtype, void* stream) {
  if (!P) return hgl::record_error(HGL_ERR_INVALID_ARG, "preconditioner is NULL");
  if (c < 1) return hgl::record_error(HGL_ERR_INVALID_ARG, "c must be >= 1");
  if (dtype != HGL_FP64 && dtype != HGL_FP32)
    return hgl::record_error(HGL_ERR_INVALID_ARG, "preconditioner panels must be FP64 or FP32");
  HGL_TRY(hgl::check_panel(R, ldr, c, hgl::dtype_size(dtype), "R"));
  HGL_TRY(hgl::check_panel(Z, ldz, c, hgl::dtype_size(dtype), "Z"));
  int rows = 0;
  return hgl::precond_apply_launch(P, P->g, R, ldr, Z, ldz, c, dtype, nullptr, hgl::as_stream(stream), &rows,
                                   nullptr);
}
