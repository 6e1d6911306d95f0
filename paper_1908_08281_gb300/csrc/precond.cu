// precond.cu -- the block preconditioner built by hgl_block_rsvd (Section 3, Eq. 15):
//   z_b = r_b / (1+lam) + Q_b diag(g_b) Q_b^T r_b,   g = ev / ((1+lam)(1+lam-ev)),
// applied block by block to an n x c panel: C_b = diag(g_b) Q_b^T R_b (k x c), then
// Z_b = R_b/(1+lam) + Q_b C_b.  FP32 panels with FP32 factors take the register-tiled
// kernels below (k_pc_*); FP64 panels or factors take the generic pair k_precond_*.
#include <algorithm>
#include <cstring>
#include <vector>

#include "rsvd_kernels.cuh"
#include "precond.cuh"
#include "solver.cuh"

namespace hgl {
namespace {

__global__ void k_gains(int nb, int k, int lpad, const double* __restrict__ ev_in, const int32_t* __restrict__ kb,
                        double lam, double* __restrict__ ev_out, double* __restrict__ gain,
                        float* __restrict__ gain32) {
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nb * k; q += gridDim.x * blockDim.x) {
    const int b = q / k, r = q % k;
    double e = r < kb[b] ? ev_in[(int64_t)b * lpad + r] : 0.0;
    e = e < 0.0 ? 0.0 : (e > 1.0 ? 1.0 : e);  // spec(Theta_bb) lies in [0, 1]
    ev_out[q] = e;
    gain[q] = r < kb[b] ? e / ((1.0 + lam) * (1.0 + lam - e)) : 0.0;
    if (gain32) gain32[q] = (float)gain[q];
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

// ---------------------------------------------------------------------------------
// FP32 panels with FP32 factors (the mixed-precision solvers), rank k <= 64, k % 4 == 0.
// Both contractions are register-tiled on the FP32 pipes: every thread owns an 8 x 8
// output tile fed by two float4 shared-memory loads per operand and step, so each
// step issues 64 FMAs per 4 shared loads.
//   projection: one CTA per (slab of <= PC_SLAB block rows, 128 columns) writes the
//               slab's 64 x 128 partial of Q_b^T R_b (double-buffered cp.async staging);
//   reduction:  C_b = diag(g_b) (sum of the block's slab partials, in slab order);
//   expansion:  one CTA per (128-row tile, 128 columns): Z = R/(1+lam) + Q_b C_b.
// Summation orders are fixed, so results are reproducible run to run.
constexpr int PF_R = 64;    // padded rank
constexpr int PF_C = 128;   // columns per CTA
constexpr int PF_RT = 32;   // block rows per staged projection step

__device__ __forceinline__ void cp_async16(void* dst, const void* src, int src_bytes) {
  const uint32_t d = static_cast<uint32_t>(__cvta_generic_to_shared(dst));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(src), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

__device__ __forceinline__ void fma_8x8(float (&acc)[8][8], const float4& a0, const float4& a1, const float4& b0,
                                        const float4& b1) {
  const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
  const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
}

// part[(slab * 64 + r) * ldp + col] = sum over the slab's rows i of Q[i, r] R[i, col]
__global__ void __launch_bounds__(128)
k_pc_proj_f32(const int32_t* __restrict__ slab_block, const int32_t* __restrict__ slab_row0,
              const int64_t* __restrict__ v0, const int32_t* __restrict__ rows, const float* __restrict__ Q, int k,
              const float* __restrict__ R, int64_t ldr, int c, float* __restrict__ part, int64_t ldp,
              const int32_t* __restrict__ run_flag) {
  if (run_flag && *run_flag == 0) return;
  __shared__ __align__(16) float sr[2][PF_RT][PF_C];   // 32 KB
  __shared__ __align__(16) float sq[2][PF_RT][PF_R];   // 16 KB
  const int slab = blockIdx.x;
  const int b = slab_block[slab];
  const int r0 = slab_row0[slab];
  const int nrows = min(PC_SLAB, rows[b] - r0);
  const int64_t base = v0[b] + r0;
  const int c0 = blockIdx.y * PF_C;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;  // tx: columns, ty: ranks
  auto stage = [&](int buf, int t0) {
#pragma unroll
    for (int q = tid; q < PF_RT * (PF_C / 4); q += 128) {
      const int i = q >> 5, j = (q & 31) * 4;
      const int row = t0 + i, col = c0 + j;
      const float* src = R;
      int bytes = 0;
      if (row < nrows && col < c) {
        src = R + (base + row) * ldr + col;
        bytes = 4 * min(4, c - col);  // the rest of the 16 bytes is zero-filled
      }
      cp_async16(&sr[buf][i][j], src, bytes);
    }
#pragma unroll
    for (int q = tid; q < PF_RT * (PF_R / 4); q += 128) {
      const int i = q >> 4, r = (q & 15) * 4;
      const int row = t0 + i;
      const float* src = Q;
      int bytes = 0;
      if (row < nrows && r < k) {
        src = Q + (base + row) * k + r;
        bytes = 16;
      }
      cp_async16(&sq[buf][i][r], src, bytes);
    }
    cp_async_commit();
  };
  float acc[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;
  const int nsteps = (nrows + PF_RT - 1) / PF_RT;
  stage(0, 0);
  for (int s = 0; s < nsteps; ++s) {
    if (s + 1 < nsteps) {
      stage((s + 1) & 1, (s + 1) * PF_RT);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
    const int buf = s & 1;
#pragma unroll 4
    for (int i = 0; i < PF_RT; ++i) {
      const float4 a0 = *reinterpret_cast<const float4*>(&sq[buf][i][ty * 4]);
      const float4 a1 = *reinterpret_cast<const float4*>(&sq[buf][i][32 + ty * 4]);
      const float4 b0 = *reinterpret_cast<const float4*>(&sr[buf][i][tx * 4]);
      const float4 b1 = *reinterpret_cast<const float4*>(&sr[buf][i][64 + tx * 4]);
      fma_8x8(acc, a0, a1, b0, b1);
    }
    __syncthreads();
  }
  // columns c..ldp-1 hold zeros (zero-filled R), so whole float4 stores are safe
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int r = i < 4 ? ty * 4 + i : 32 + ty * 4 + (i - 4);
    float* dst = part + ((int64_t)slab * PF_R + r) * ldp;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int col = c0 + h * 64 + tx * 4;
      if (col < ldp)
        *reinterpret_cast<float4*>(dst + col) =
            make_float4(acc[i][4 * h], acc[i][4 * h + 1], acc[i][4 * h + 2], acc[i][4 * h + 3]);
    }
  }
}

// C[(b * 64 + r) * ldp + col] = gain[b, r] * sum_{slabs of b, in order} part[...]
__global__ void k_pc_reduce_f32(int nb, const int32_t* __restrict__ blk_slab0, const double* __restrict__ gain,
                                int k, const float* __restrict__ part, int64_t ldp, float* __restrict__ C) {
  const int64_t nvec = ldp / 4;
  const int64_t total = (int64_t)nb * PF_R * nvec;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t row = q / nvec;  // b * 64 + r
    const int col = (int)(q % nvec) * 4;
    const int b = (int)(row / PF_R), r = (int)(row % PF_R);
    float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int sl = blk_slab0[b]; sl < blk_slab0[b + 1]; ++sl) {
      const float4 p = *reinterpret_cast<const float4*>(part + ((int64_t)sl * PF_R + r) * ldp + col);
      s.x += p.x;
      s.y += p.y;
      s.z += p.z;
      s.w += p.w;
    }
    const float g = r < k ? (float)gain[(int64_t)b * k + r] : 0.f;
    *reinterpret_cast<float4*>(C + row * ldp + col) = make_float4(g * s.x, g * s.y, g * s.z, g * s.w);
  }
}

// Z[rows of one 128-row tile, 128 columns] = R / (1+lam) + Q_b C_b
__global__ void __launch_bounds__(256, 2)
k_pc_expand_f32(const int32_t* __restrict__ exp_block, const int32_t* __restrict__ exp_tile,
                const int64_t* __restrict__ v0, const int32_t* __restrict__ rows, const float* __restrict__ Q, int k,
                const float* __restrict__ R, int64_t ldr, float* __restrict__ Z, int64_t ldz, int c, float inv1l,
                const float* __restrict__ C, int64_t ldp, const int32_t* __restrict__ run_flag) {
  if (run_flag && *run_flag == 0) return;
  extern __shared__ __align__(16) float smx[];
  float* qt = smx;                  // [64 ranks][128 rows]  (Q tile transposed)
  float* cs = smx + PF_R * PC_TILE;  // [64 ranks][128 columns]
  const int u = blockIdx.x;
  const int b = exp_block[u];
  const int i0 = exp_tile[u] * PC_TILE;
  const int nrows = rows[b];
  const int64_t base = v0[b] + i0;
  const int c0 = blockIdx.y * PF_C;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;  // tx: columns, ty: rows
  const int kk = (k + 3) & ~3;
  // the accumulators start at R / (1+lam): these loads are issued first so that their
  // latency overlaps the staging of the Q and C tiles
  float acc[8][8];
  const float* rbase = R + (base + ty * 4) * ldr + c0 + tx * 4;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int row = i < 4 ? ty * 4 + i : 64 + ty * 4 + (i - 4);
    const float* rrow = rbase + (int64_t)(i < 4 ? i : 60 + i) * ldr;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int col = c0 + h * 64 + tx * 4;
      // ldr is a multiple of 4 and col of 4, so col < c keeps the whole vector inside
      // the row; padding columns only reach accumulators that are never stored
      float4 rv = make_float4(0.f, 0.f, 0.f, 0.f);
      if (i0 + row < nrows && col < c) rv = __ldg(reinterpret_cast<const float4*>(rrow + h * 64));
      acc[i][4 * h] = inv1l * rv.x;
      acc[i][4 * h + 1] = inv1l * rv.y;
      acc[i][4 * h + 2] = inv1l * rv.z;
      acc[i][4 * h + 3] = inv1l * rv.w;
    }
  }
  for (int q = tid; q < PC_TILE * (PF_R / 4); q += 256) {
    const int i = q & (PC_TILE - 1), r = (q >> 7) * 4;
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (i0 + i < nrows && r < k) v = __ldg(reinterpret_cast<const float4*>(Q + (base + i) * k + r));
    qt[(r + 0) * PC_TILE + i] = v.x;
    qt[(r + 1) * PC_TILE + i] = v.y;
    qt[(r + 2) * PC_TILE + i] = v.z;
    qt[(r + 3) * PC_TILE + i] = v.w;
  }
  for (int q = tid; q < PF_R * (PF_C / 4); q += 256) {
    const int r = q >> 5, j = (q & 31) * 4;
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (c0 + j < ldp) v = __ldg(reinterpret_cast<const float4*>(C + ((int64_t)b * PF_R + r) * ldp + c0 + j));
    *reinterpret_cast<float4*>(&cs[r * PF_C + j]) = v;
  }
  __syncthreads();
#pragma unroll 4
  for (int r = 0; r < kk; ++r) {
    const float4 a0 = *reinterpret_cast<const float4*>(&qt[r * PC_TILE + ty * 4]);
    const float4 a1 = *reinterpret_cast<const float4*>(&qt[r * PC_TILE + 64 + ty * 4]);
    const float4 b0 = *reinterpret_cast<const float4*>(&cs[r * PF_C + tx * 4]);
    const float4 b1 = *reinterpret_cast<const float4*>(&cs[r * PF_C + 64 + tx * 4]);
    fma_8x8(acc, a0, a1, b0, b1);
  }
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int row = i < 4 ? ty * 4 + i : 64 + ty * 4 + (i - 4);
    if (i0 + row >= nrows) continue;
    float* zrow = Z + (base + row) * ldz;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int col = c0 + h * 64 + tx * 4;
      if (col + 3 < c) {
        *reinterpret_cast<float4*>(zrow + col) =
            make_float4(acc[i][4 * h], acc[i][4 * h + 1], acc[i][4 * h + 2], acc[i][4 * h + 3]);
      } else {
#pragma unroll
        for (int j = 0; j < 4; ++j)
          if (col + j < c) zrow[col + j] = acc[i][4 * h + j];
      }
    }
  }
}

hgl_status apply_fast_f32(hgl_precond* P, const float* R, int64_t ldr, float* Z, int64_t ldz, int c, cudaStream_t st,
                          const int32_t* run_flag) {
  ProfScope prof(HGL_PROF_PRECOND, st);
  const int64_t ldp = (c + 3) / 4 * 4;
  hgl_status s = HGL_OK;
  float* part = static_cast<float*>(buffer_get(P->pbuf, sizeof(float) * (size_t)P->nslabs * PF_R * ldp, &s));
  if (!part) return s;
  float* C = static_cast<float*>(buffer_get(P->cbuf, sizeof(float) * (size_t)P->nb * PF_R * ldp, &s));
  if (!C) return s;
  const int cchunks = (c + PF_C - 1) / PF_C;
  const size_t sm_exp = sizeof(float) * 2 * PF_R * PC_TILE;
  HGL_CHECK_CUDA(cudaFuncSetAttribute(k_pc_expand_f32, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_exp));
  hgl::count_launch(3);
  k_pc_proj_f32<<<dim3(P->nslabs, cchunks), 128, 0, st>>>(P->slab_block, P->slab_row0, P->d_v0, P->d_rows,
                                                          static_cast<const float*>(P->Q), P->k, R, ldr, c, part,
                                                          ldp, run_flag);
  const int64_t nred = (int64_t)P->nb * PF_R * (ldp / 4);
  const int gred = (int)std::min<int64_t>((nred + 255) / 256, (int64_t)device_sm_count() * 8);
  k_pc_reduce_f32<<<gred, 256, 0, st>>>(P->nb, P->blk_slab0, P->gain, P->k, part, ldp, C);
  k_pc_expand_f32<<<dim3(P->nexp, cchunks), 256, sm_exp, st>>>(
      P->exp_block, P->exp_tile, P->d_v0, P->d_rows, static_cast<const float*>(P->Q), P->k, R, ldr, Z, ldz, c,
      (float)(1.0 / (1.0 + P->lam)), C, ldp, run_flag);
  HGL_CHECK_CUDA(cudaGetLastError());
  return HGL_OK;
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
  hgl::count_launch(); k_gains<<<(P->nb * P->k + 255) / 256, 256, 0, st>>>(P->nb, P->k, lpad, ev_lpad, P->d_kb, P->lam, P->ev, P->gain,
                                                                             P->gain32);
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

hgl_status precond_reserve(hgl_precond* P, int c, int dt) {
  hgl_status s = HGL_OK;
  const bool f32q = P->dtype == HGL_BF16;
  if (dt == HGL_FP32 && P->tc) {  // the tensor-core apply's C hi/lo
    const int64_t c128 = (c + 127) / 128 * 128;
    if (!buffer_get(P->cbuf, sizeof(float) * 2 * (size_t)P->nb * c128 * P->kp, &s)) return s;
  }
  if (dt == HGL_FP32 && f32q && P->k <= PF_R && P->k % 4 == 0) {
    const int64_t ldp = (c + 3) / 4 * 4;
    if (!buffer_get(P->pbuf, sizeof(float) * (size_t)P->nslabs * PF_R * ldp, &s)) return s;
    if (!buffer_get(P->cbuf, sizeof(float) * (size_t)P->nb * PF_R * ldp, &s)) return s;
  } else {
    const size_t a = dt == HGL_FP64 ? sizeof(double) : sizeof(float);
    if (!buffer_get(P->cbuf, a * (size_t)P->nb * P->k * c, &s)) return s;
  }
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
    if (precond_tc_usable(P, R, ldr, Z, ldz)) {
      // tensor cores; the projection also gives the per-block r.z partials when the
      // caller's partial array has room for nb rows
      const bool rz_here = partials_rz && P->nb <= solver_partial_rows(g);
      HGL_TRY(precond_tc_apply(P, (const float*)R, ldr, (float*)Z, ldz, c, rz_here ? partials_rz : nullptr, st,
                               run_flag));
      if (rz_here) {
        *rows = P->nb;
        return HGL_OK;
      }
    } else if (f32q && P->k <= PF_R && P->k % 4 == 0)
      HGL_TRY(apply_fast_f32(P, (const float*)R, ldr, (float*)Z, ldz, c, st, run_flag));
    else if (f32q)
      HGL_TRY((apply_typed<float, float>(P, (const float*)R, ldr, (float*)Z, ldz, c, st, run_flag)));
    else
      HGL_TRY((apply_typed<float, double>(P, (const float*)R, ldr, (float*)Z, ldz, c, st, run_flag)));
  } else {
    return record_error(HGL_ERR_INVALID_ARG, "preconditioner panels must be FP64 or FP32");
  }
  if (partials_rz) HGL_TRY(panel_dot_launch(g, c, dt, R, ldr, Z, ldz, partials_rz, st, rows, run_flag));
  return HGL_OK;
}

}  // namespace hgl

extern "C" hgl_status hgl_set_block_product(hgl_graph* g, int32_t mode) {
  if (!g) return hgl::record_error(HGL_ERR_INVALID_ARG, "graph is NULL");
  if (mode != HGL_BLOCKS_AUTO && mode != HGL_BLOCKS_DENSE && mode != HGL_BLOCKS_SPARSE)
    return hgl::record_error(HGL_ERR_INVALID_ARG, "unknown block product route %d", (int)mode);
  g->block_product = mode;
  return HGL_OK;
}

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
  hgl::buffer_free(P->pbuf);
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
