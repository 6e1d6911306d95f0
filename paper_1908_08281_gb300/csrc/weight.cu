// weight.cu -- the weight sub-problem of Section 2 (Eqs. 4 and 5): the gradient of
// P(w) = tr(F^T Delta F) + mu ||w||^2 at fixed F, and the projected steepest-descent
// step onto the simplex {w >= 0, 1^T w = 1}.
//
// Gradient (bilinear form, Z = F for P):
//   d/dw_e tr(Z^T Theta F) = <sF_e, sZ_e>/de_e - sum_{v in e} phi_v,
//   sX_e = sum_{v in e} s_v X[v,:]           (H^T Dv^-1/2 X, row e)
//   UX_v = sum_{e ni v} t_e sX_e             (H W De^-1 H^T Dv^-1/2 X, row v)
//   phi_v = 1/2 s_v^3 (<F_v, UZ_v> + <Z_v, UF_v>)     (from d dv_v / d w_e = H(v,e))
// computed by a hyperedge gather pass (sX, and T = t sX for the next pass), a vertex
// gather pass (phi) and a scalar hyperedge pass; columns are processed in chunks and
// the row dot products are accumulated chunk by chunk in FP64.
#include <algorithm>
#include <vector>

#include "solver.cuh"
#include "theta_launch.cuh"

namespace hgl {

namespace {

// Heavy hyperedges (the first nheavy of `order`) get one block each, the others one
// warp each, longest first.
template <class TX, int LG, int NV, bool DUAL>
__global__ void __launch_bounds__(OP_THREADS)
k_grad_edge(int64_t m, const int64_t* __restrict__ csc_ptr, const int32_t* __restrict__ csc_idx,
            const int32_t* __restrict__ order, int64_t nheavy, const typename AccOf<TX>::type* __restrict__ s,
            const double* __restrict__ t, const TX* __restrict__ F, const TX* __restrict__ Zb, int64_t ld, int c0,
            int cw, typename AccOf<TX>::type* __restrict__ TF, typename AccOf<TX>::type* __restrict__ TZ, int64_t ldt,
            double* __restrict__ ex) {
  using A = typename AccOf<TX>::type;
  constexpr int E = 16 / (int)sizeof(TX);
  constexpr int G = 32 / LG;
  constexpr int TILE = LG * NV * E;
  const int lane = threadIdx.x & 31, grp = lane / LG, l = lane % LG, wid = threadIdx.x >> 5;
  const bool heavy = blockIdx.x < nheavy;
  const int64_t warp = heavy ? 0 : (((int64_t)blockIdx.x - nheavy) * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = heavy ? 1 : (((int64_t)gridDim.x - nheavy) * blockDim.x) >> 5;
  for (int64_t q = heavy ? blockIdx.x : nheavy + warp; q < (heavy ? (int64_t)blockIdx.x + 1 : m); q += nwarps) {
    const int32_t e = order[q];
    const int64_t beg = csc_ptr[e], end = csc_ptr[e + 1];
    A sf[NV][E], sz[NV][E];
#pragma unroll
    for (int k = 0; k < NV; ++k)
#pragma unroll
      for (int j = 0; j < E; ++j) sf[k][j] = sz[k][j] = A(0);
    const int64_t first = heavy ? beg + wid * G + grp : beg + grp;
    const int64_t step = heavy ? (int64_t)OP_WARPS * G : G;
    for (int64_t i = first; i < end; i += step) {
      const int32_t v = __ldg(csc_idx + i);
      const A sv = (A)__ldg(s + v);
#pragma unroll
      for (int k = 0; k < NV; ++k) {
        const int col = (k * LG + l) * E;
        if (col < cw) {
          A x[E];
          vload<A, TX, E>(F + (int64_t)v * ld + c0 + col, x);
#pragma unroll
          for (int j = 0; j < E; ++j) sf[k][j] = fma(sv, x[j], sf[k][j]);
          if (DUAL) {
            vload<A, TX, E>(Zb + (int64_t)v * ld + c0 + col, x);
#pragma unroll
            for (int j = 0; j < E; ++j) sz[k][j] = fma(sv, x[j], sz[k][j]);
          }
        }
      }
    }
#pragma unroll
    for (int off = LG; off < 32; off <<= 1)
#pragma unroll
      for (int k = 0; k < NV; ++k)
#pragma unroll
        for (int j = 0; j < E; ++j) {
          sf[k][j] += __shfl_xor_sync(0xffffffffu, sf[k][j], off);
          if (DUAL) sz[k][j] += __shfl_xor_sync(0xffffffffu, sz[k][j], off);
        }
    if (heavy) {
      __shared__ A red_f[OP_WARPS][TILE];
      __shared__ A red_z[DUAL ? OP_WARPS : 1][DUAL ? TILE : 1];
      if (grp == 0)
#pragma unroll
        for (int k = 0; k < NV; ++k)
#pragma unroll
          for (int j = 0; j < E; ++j) {
            red_f[wid][(k * LG + l) * E + j] = sf[k][j];
            if (DUAL) red_z[wid][(k * LG + l) * E + j] = sz[k][j];
          }
      __syncthreads();
      if (wid != 0) return;
#pragma unroll
      for (int k = 0; k < NV; ++k)
#pragma unroll
        for (int j = 0; j < E; ++j) {
          A a = A(0), b = A(0);
          for (int w = 0; w < OP_WARPS; ++w) {
            a += red_f[w][(k * LG + l) * E + j];
            if (DUAL) b += red_z[w][(k * LG + l) * E + j];
          }
          sf[k][j] = a;
          sz[k][j] = b;
        }
    }
    double d = 0.0;
    const A te = (A)t[e];
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      const int col = (k * LG + l) * E;
      if (col < cw) {
        A o[E];
#pragma unroll
        for (int j = 0; j < E; ++j) {
          d += (double)sf[k][j] * (double)(DUAL ? sz[k][j] : sf[k][j]);
          o[j] = te * sf[k][j];
        }
        if (grp == 0) {
          vstore<A, A, E>(TF + e * ldt + col, o, E);
          if (DUAL) {
#pragma unroll
            for (int j = 0; j < E; ++j) o[j] = te * sz[k][j];
            vstore<A, A, E>(TZ + e * ldt + col, o, E);
          }
        }
      }
    }
#pragma unroll
    for (int off = 1; off < LG; off <<= 1) d += __shfl_xor_sync(0xffffffffu, d, off);
    if (lane == 0) ex[e] = (c0 == 0 ? 0.0 : ex[e]) + d;
  }
}

template <class TX, int LG, int NV, bool DUAL>
__global__ void __launch_bounds__(OP_THREADS)
k_grad_vertex(int64_t n, const int64_t* __restrict__ csr_ptr, const int32_t* __restrict__ csr_idx,
              const double* __restrict__ s, const typename AccOf<TX>::type* __restrict__ TF,
              const typename AccOf<TX>::type* __restrict__ TZ, int64_t ldt, const TX* __restrict__ F,
              const TX* __restrict__ Zb, int64_t ld, int c0, int cw, double* __restrict__ phi) {
  using A = typename AccOf<TX>::type;
  constexpr int E = 16 / (int)sizeof(TX);
  constexpr int G = 32 / LG;
  const int lane = threadIdx.x & 31, grp = lane / LG, l = lane % LG;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t v = warp; v < n; v += nwarps) {
    const int64_t beg = csr_ptr[v], end = csr_ptr[v + 1];
    A uf[NV][E], uz[NV][E];
#pragma unroll
    for (int k = 0; k < NV; ++k)
#pragma unroll
      for (int j = 0; j < E; ++j) uf[k][j] = uz[k][j] = A(0);
    for (int64_t i = beg + grp; i < end; i += G) {
      const int32_t e = __ldg(csr_idx + i);
#pragma unroll
      for (int k = 0; k < NV; ++k) {
        const int col = (k * LG + l) * E;
        if (col < cw) {
          A x[E];
          vload<A, A, E>(TF + (int64_t)e * ldt + col, x);
#pragma unroll
          for (int j = 0; j < E; ++j) uf[k][j] += x[j];
          if (DUAL) {
            vload<A, A, E>(TZ + (int64_t)e * ldt + col, x);
#pragma unroll
            for (int j = 0; j < E; ++j) uz[k][j] += x[j];
          }
        }
      }
    }
#pragma unroll
    for (int off = LG; off < 32; off <<= 1)
#pragma unroll
      for (int k = 0; k < NV; ++k)
#pragma unroll
        for (int j = 0; j < E; ++j) {
          uf[k][j] += __shfl_xor_sync(0xffffffffu, uf[k][j], off);
          if (DUAL) uz[k][j] += __shfl_xor_sync(0xffffffffu, uz[k][j], off);
        }
    double d = 0.0;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      const int col = (k * LG + l) * E;
      if (col < cw) {
        A f[E];
        vload<A, TX, E>(F + v * ld + c0 + col, f);
        if (DUAL) {
          A z[E];
          vload<A, TX, E>(Zb + v * ld + c0 + col, z);
#pragma unroll
          for (int j = 0; j < E; ++j) d += 0.5 * ((double)f[j] * (double)uz[k][j] + (double)z[j] * (double)uf[k][j]);
        } else {
#pragma unroll
          for (int j = 0; j < E; ++j) d += (double)f[j] * (double)uf[k][j];
        }
      }
    }
#pragma unroll
    for (int off = 1; off < LG; off <<= 1) d += __shfl_xor_sync(0xffffffffu, d, off);
    if (lane == 0) {
      const double sv = s[v];
      phi[v] = (c0 == 0 ? 0.0 : phi[v]) + sv * sv * sv * d;
    }
  }
}

// grad_e = -(ex_e / de_e - sum_{v in e} phi_v) + 2 mu w_e   (phi omitted when dv is frozen)
__global__ void k_grad_final(int64_t m, const int64_t* __restrict__ csc_ptr, const int32_t* __restrict__ csc_idx,
                             const int32_t* __restrict__ de, const double* __restrict__ ex,
                             const double* __restrict__ phi, const double* __restrict__ w, double mu,
                             double theta_sign, double* __restrict__ grad) {
  // groups of 8 lanes per hyperedge (most hyperedges have a few members), a fixed
  // lane-to-member assignment and a fixed butterfly: the sum order depends on nothing
  // but the hyperedge
  constexpr int GL = 8;
  const int sub = threadIdx.x % GL;
  const int64_t grp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / GL;
  const int64_t ngrp = ((int64_t)gridDim.x * blockDim.x) / GL;
  const int64_t rounds = (m + ngrp - 1) / ngrp;  // every lane runs the same number of rounds
  for (int64_t r = 0; r < rounds; ++r) {
    const int64_t e = grp + r * ngrp;
    double acc = 0.0;
    if (phi && e < m)
      for (int64_t i = csc_ptr[e] + sub, end = csc_ptr[e + 1]; i < end; i += GL) acc += phi[csc_idx[i]];
#pragma unroll
    for (int o = GL / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (sub == 0 && e < m) grad[e] = -theta_sign * (ex[e] / (double)de[e] - acc) + 2.0 * mu * w[e];
  }
}

template <class TX, bool DUAL>
hgl_status grad_launch_typed(hgl_graph* g, const TX* F, const TX* Zb, int64_t ld, int c, double mu, bool frozen,
                             const double* w, double* grad, cudaStream_t st, double theta_sign) {
  using A = typename AccOf<TX>::type;
  constexpr int E = 16 / (int)sizeof(TX);
  const int nvec = (c + E - 1) / E;
  int chunk_vec = std::min(nvec, 128);
  int lg = 1, nv = 1;
  pick_tile(chunk_vec, &lg, &nv);
  const int cc = lg * nv * E;
  hgl_status stt = HGL_OK;
  A* TF = static_cast<A*>(buffer_get(g->scratch, sizeof(A) * (size_t)g->m * cc, &stt));
  if (!TF) return stt;
  A* TZ = nullptr;
  if (DUAL) {
    TZ = static_cast<A*>(buffer_get(g->scratch2, sizeof(A) * (size_t)g->m * cc, &stt));
    if (!TZ) return stt;
  }
  double* vecs = static_cast<double*>(buffer_get(g->misc, sizeof(double) * (size_t)(g->m + g->n + 2), &stt));
  if (!vecs) return stt;
  double* ex = vecs;
  double* phi = vecs + g->m;
  const int64_t cap = (int64_t)g->num_sms * 8;
  const int grid1 = (int)std::max<int64_t>(1, std::min<int64_t>((g->m + OP_WARPS - 1) / OP_WARPS, cap));
  ProfScope prof(HGL_PROF_GRADIENT, st);
  for (int c0 = 0; c0 < c; c0 += cc) {
    const int cw = std::min(cc, c - c0);
#define HGL_GE(LG_, NV_)                                                                                        \
  else if (lg == LG_ && nv == NV_) {                                                                            \
    auto fn = k_grad_edge<TX, LG_, NV_, DUAL>;                                                                  \
    const int gr = edge_grid(g, resident_blocks(reinterpret_cast<const void*>(fn), OP_THREADS, 0));             \
    hgl::count_launch();                                                                                        \
    fn<<<gr, OP_THREADS, 0, st>>>(g->m, g->csc_ptr, g->csc_idx, g->edge_order, g->nheavy, scal_s<A>(g), g->t, F, \
                                  Zb, ld, c0, cw, TF, TZ, (int64_t)cc, ex);                                     \
  }
#define HGL_GV(LG_, NV_)                                                                                        \
  else if (lg == LG_ && nv == NV_) {                                                                            \
    auto fn = k_grad_vertex<TX, LG_, NV_, DUAL>;                                                                \
    const int gr = vertex_grid(g, resident_blocks(reinterpret_cast<const void*>(fn), OP_THREADS, 0));           \
    hgl::count_launch();                                                                                        \
    fn<<<gr, OP_THREADS, 0, st>>>(g->n, g->csr_ptr, g->csr_idx, g->s, TF, TZ, (int64_t)cc, F, Zb, ld, c0, cw,    \
                                  phi);                                                                         \
  }
    if (false) {
    }
    HGL_FOR_EACH_TILE(HGL_GE)
    if (!frozen) {
      if (false) {
      }
      HGL_FOR_EACH_TILE(HGL_GV)
    }
#undef HGL_GE
#undef HGL_GV
    HGL_CHECK_CUDA(cudaGetLastError());
  }
  hgl::count_launch(); k_grad_final<<<grid1, OP_THREADS, 0, st>>>(g->m, g->csc_ptr, g->csc_idx, g->de, ex, frozen ? nullptr : phi, w, mu,
                                             theta_sign, grad);
  HGL_CHECK_CUDA(cudaGetLastError());
  return HGL_OK;
}

// ---- simplex projection (Michelot's support-shrinking iteration) -----------------

struct ProjState {
  double tau;
  double prev_count;
  int32_t done;
  unsigned counter;
};

constexpr int PROJ_THREADS = 256;

__global__ void k_proj_init(double* __restrict__ v, const double* __restrict__ w, const double* __restrict__ grad,
                            double eta, int64_t m, double* __restrict__ part_sum) {
  __shared__ double red[PROJ_THREADS / 32];
  double acc = 0.0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x) {
    const double x = w[e] - (grad ? eta * grad[e] : 0.0);
    v[e] = x;
    acc += x;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < PROJ_THREADS / 32; ++i) s += red[i];
    part_sum[blockIdx.x] = s;
  }
}

// tau_0 = (sum v - 1) / m
__global__ void k_proj_tau0(const double* __restrict__ part_sum, int nparts, int64_t m, ProjState* ps) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < nparts; ++i) s += part_sum[i];
    ps->tau = (s - 1.0) / (double)m;
    ps->prev_count = (double)m;
    ps->done = 0;
    ps->counter = 0u;
  }
}

// One Michelot step: S = {e : v_e > tau}; if |S| unchanged, done; else tau = (sum_S v - 1)/|S|.
__global__ void k_proj_step(const double* __restrict__ v, int64_t m, double* __restrict__ part_sum,
                            double* __restrict__ part_cnt, ProjState* ps) {
  if (((volatile ProjState*)ps)->done) return;
  __shared__ double rs[PROJ_THREADS / 32], rc[PROJ_THREADS / 32];
  __shared__ bool last;
  const double tau = ps->tau;
  double s = 0.0, cnt = 0.0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x) {
    const double x = v[e];
    if (x > tau) {
      s += x;
      cnt += 1.0;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    s += __shfl_xor_sync(0xffffffffu, s, o);
    cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
  }
  if ((threadIdx.x & 31) == 0) {
    rs[threadIdx.x >> 5] = s;
    rc[threadIdx.x >> 5] = cnt;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int i = 0; i < PROJ_THREADS / 32; ++i) {
      a += rs[i];
      b += rc[i];
    }
    part_sum[blockIdx.x] = a;
    part_cnt[blockIdx.x] = b;
    __threadfence();
    last = atomicAdd(&ps->counter, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (last && threadIdx.x == 0) {
    __threadfence();
    double a = 0.0, b = 0.0;
    for (unsigned i = 0; i < gridDim.x; ++i) {
      a += ((volatile double*)part_sum)[i];
      b += ((volatile double*)part_cnt)[i];
    }
    if (b == ps->prev_count || b <= 0.0) {
      ps->done = 1;
    } else {
      ps->tau = (a - 1.0) / b;
      ps->prev_count = b;
    }
    ps->counter = 0u;
  }
}

__global__ void k_proj_apply(const double* __restrict__ v, int64_t m, const ProjState* ps, double* __restrict__ w) {
  const double tau = ps->tau;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x) {
    const double x = v[e] - tau;
    w[e] = x > 0.0 ? x : 0.0;
  }
}

// ---- active-set steepest descent (Eq. 5 read literally) --------------------------
// Pinned weights (w_e = 0) stay 0; free ones move by -eta (g_e - mean over free of g),
// are clamped at 0 and rescaled to sum 1.  Three launches, block reductions in a fixed
// order (every block re-adds the previous kernel's partials in index order), no host
// reads.  work layout: v[m] | stats[2 * blocks] | sums[blocks]

__device__ __forceinline__ void block_sum2(double& a, double& b, double (*red)[PROJ_THREADS / 32]) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
  }
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = a;
    red[1][threadIdx.x >> 5] = b;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    a = 0.0;
    b = 0.0;
    for (int i = 0; i < PROJ_THREADS / 32; ++i) {
      a += red[0][i];
      b += red[1][i];
    }
  }
}

__global__ void k_as_stats(const double* __restrict__ w, const double* __restrict__ g, int64_t m,
                           double* __restrict__ stats) {
  __shared__ double red[2][PROJ_THREADS / 32];
  double s = 0.0, cnt = 0.0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x)
    if (w[e] > 0.0) {
      s += g[e];
      cnt += 1.0;
    }
  block_sum2(s, cnt, red);
  if (threadIdx.x == 0) {
    stats[2 * blockIdx.x] = s;
    stats[2 * blockIdx.x + 1] = cnt;
  }
}

__global__ void k_as_update(const double* __restrict__ w, const double* __restrict__ g, double eta, int64_t m,
                            const double* __restrict__ stats, double* __restrict__ v, double* __restrict__ sums) {
  __shared__ double red[2][PROJ_THREADS / 32];
  __shared__ double mean_s, cnt_s;
  if (threadIdx.x == 0) {
    double s = 0.0, c = 0.0;
    for (unsigned i = 0; i < gridDim.x; ++i) {
      s += stats[2 * i];
      c += stats[2 * i + 1];
    }
    mean_s = c > 0.0 ? s / c : 0.0;
    cnt_s = c;
  }
  __syncthreads();
  const double mean = mean_s;
  double tot = 0.0, unused = 0.0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x) {
    const double we = w[e];
    double x = 0.0;
    if (we > 0.0) {
      x = we - eta * (g[e] - mean);
      x = x > 0.0 ? x : 0.0;
    }
    v[e] = x;
    tot += x;
  }
  block_sum2(tot, unused, red);
  if (threadIdx.x == 0) sums[blockIdx.x] = cnt_s > 0.0 ? tot : 0.0;
}

__global__ void k_as_scale(double* __restrict__ w, const double* __restrict__ v, int64_t m,
                           const double* __restrict__ sums) {
  __shared__ double total_s;
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (unsigned i = 0; i < gridDim.x; ++i) t += sums[i];
    total_s = t;
  }
  __syncthreads();
  const double total = total_s;
  if (!(total > 0.0)) return;  // nothing free, or nothing left after clamping: w unchanged
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x)
    w[e] = v[e] / total;
}

}  // namespace

double* grad_vectors(hgl_graph* g, hgl_status* st) {
  return static_cast<double*>(buffer_get(g->misc, sizeof(double) * (size_t)(g->m + g->n + 2), st));
}

// The gradient's vertex pass and final sum from a first pass done elsewhere (TF, ex).
hgl_status weight_grad_from_edges(hgl_graph* g, const double* w, const float* TF, int64_t ldtf, const float* F,
                                  int64_t ld, int c, double mu, int flags, double* grad, cudaStream_t st) {
  constexpr int E = 4;
  const bool frozen = (flags & HGL_GRAD_DV_FROZEN) != 0;
  const int nvec = (c + E - 1) / E;
  int lg = 1, nv = 1;
  pick_tile(std::min(nvec, 128), &lg, &nv);
  const int cc = lg * nv * E;
  hgl_status stt = HGL_OK;
  double* vecs = grad_vectors(g, &stt);
  if (!vecs) return stt;
  double* ex = vecs;
  double* phi = vecs + g->m;
  const int64_t cap = (int64_t)g->num_sms * 8;
  const int grid1 = (int)std::max<int64_t>(1, std::min<int64_t>((g->m + OP_WARPS - 1) / OP_WARPS, cap));
  ProfScope prof(HGL_PROF_GRADIENT, st);
  if (!frozen) {
    for (int c0 = 0; c0 < c; c0 += cc) {
      const int cw = std::min(cc, c - c0);
#define HGL_GV(LG_, NV_)                                                                                        \
  else if (lg == LG_ && nv == NV_) {                                                                            \
    auto fn = k_grad_vertex<float, LG_, NV_, false>;                                                            \
    const int gr = vertex_grid(g, resident_blocks(reinterpret_cast<const void*>(fn), OP_THREADS, 0));           \
    hgl::count_launch();                                                                                        \
    fn<<<gr, OP_THREADS, 0, st>>>(g->n, g->csr_ptr, g->csr_idx, g->s, TF + c0, nullptr, ldtf, F, nullptr, ld,    \
                                  c0, cw, phi);                                                                 \
  }
      if (false) {
      }
      HGL_FOR_EACH_TILE(HGL_GV)
#undef HGL_GV
      HGL_CHECK_CUDA(cudaGetLastError());
    }
  }
  hgl::count_launch();
  k_grad_final<<<grid1, OP_THREADS, 0, st>>>(g->m, g->csc_ptr, g->csc_idx, g->de, ex, frozen ? nullptr : phi, w, mu,
                                             1.0, grad);
  HGL_CHECK_CUDA(cudaGetLastError());
  return HGL_OK;
}

hgl_status weight_grad_launch(hgl_graph* g, const double* w, const void* F, const void* Zb, int64_t ld, int c,
                              int dtype, double mu, int flags, double* grad, cudaStream_t st, double theta_sign) {
  const bool frozen = (flags & HGL_GRAD_DV_FROZEN) != 0;
  const double sg = theta_sign;
  if (dtype == HGL_FP64) {
    if (Zb)
      return grad_launch_typed<double, true>(g, (const double*)F, (const double*)Zb, ld, c, mu, frozen, w, grad, st, sg);
    return grad_launch_typed<double, false>(g, (const double*)F, nullptr, ld, c, mu, frozen, w, grad, st, sg);
  }
  if (dtype == HGL_FP32) {
    if (Zb)
      return grad_launch_typed<float, true>(g, (const float*)F, (const float*)Zb, ld, c, mu, frozen, w, grad, st, sg);
    return grad_launch_typed<float, false>(g, (const float*)F, nullptr, ld, c, mu, frozen, w, grad, st, sg);
  }
  return record_error(HGL_ERR_INVALID_ARG, "gradient panels must be FP64 or FP32");
}

hgl_status project_launch(double* w, const double* grad, double eta, int64_t m, double* work, int sms,
                          cudaStream_t st, int max_steps) {
  ProfScope prof(HGL_PROF_PROJECT, st);
  // work layout: v[m] | part_sum[blocks] | part_cnt[blocks] | ProjState
  const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((m + PROJ_THREADS - 1) / PROJ_THREADS, sms * 2));
  double* v = work;
  double* ps_sum = v + m;
  double* ps_cnt = ps_sum + blocks;
  ProjState* ps = reinterpret_cast<ProjState*>(ps_cnt + blocks);
  hgl::count_launch(); k_proj_init<<<blocks, PROJ_THREADS, 0, st>>>(v, w, grad, eta, m, ps_sum);
  hgl::count_launch(); k_proj_tau0<<<1, 32, 0, st>>>(ps_sum, blocks, m, ps);
  HGL_CHECK_CUDA(cudaGetLastError());
  int steps = 0;
  for (;;) {
    const int batch = 16;
    for (int k = 0; k < batch; ++k) { hgl::count_launch(); k_proj_step<<<blocks, PROJ_THREADS, 0, st>>>(v, m, ps_sum, ps_cnt, ps); }
    HGL_CHECK_CUDA(cudaGetLastError());
    steps += batch;
    if (max_steps > 0) {
      // a fixed number of steps (capturable: no host reads; converged steps return at once)
      if (steps >= max_steps) break;
      continue;
    }
    int32_t done = 0;
    HGL_CHECK_CUDA(cudaMemcpyAsync(&done, &ps->done, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    HGL_CHECK_CUDA(cudaStreamSynchronize(st));
    if (done || steps > m + 16) break;
  }
  hgl::count_launch(); k_proj_apply<<<blocks, PROJ_THREADS, 0, st>>>(v, m, ps, w);
  HGL_CHECK_CUDA(cudaGetLastError());
  return HGL_OK;
}

// After a projection launched with a fixed number of steps: if its iteration had not
// settled, continue it (host-checked batches) from the state in `work` and apply the
// final threshold again.  Synchronises the stream.
hgl_status project_finish(double* w, int64_t m, double* work, int sms, cudaStream_t st, bool* continued) {
  const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((m + PROJ_THREADS - 1) / PROJ_THREADS, sms * 2));
  double* v = work;
  double* ps_sum = v + m;
  double* ps_cnt = ps_sum + blocks;
  ProjState* ps = reinterpret_cast<ProjState*>(ps_cnt + blocks);
  int32_t done = 0;
  HGL_CHECK_CUDA(cudaMemcpyAsync(&done, &ps->done, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  HGL_CHECK_CUDA(cudaStreamSynchronize(st));
  *continued = !done;
  if (done) return HGL_OK;
  for (int64_t steps = 0; !done && steps <= m + 16; steps += 16) {
    for (int k = 0; k < 16; ++k) {
      hgl::count_launch();
      k_proj_step<<<blocks, PROJ_THREADS, 0, st>>>(v, m, ps_sum, ps_cnt, ps);
    }
    HGL_CHECK_CUDA(cudaGetLastError());
    HGL_CHECK_CUDA(cudaMemcpyAsync(&done, &ps->done, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    HGL_CHECK_CUDA(cudaStreamSynchronize(st));
  }
  hgl::count_launch();
  k_proj_apply<<<blocks, PROJ_THREADS, 0, st>>>(v, m, ps, w);
  HGL_CHECK_CUDA(cudaGetLastError());
  HGL_CHECK_CUDA(cudaStreamSynchronize(st));
  return HGL_OK;
}

size_t active_set_work_doubles(int64_t m, int sms) {
  const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>((m + PROJ_THREADS - 1) / PROJ_THREADS, sms * 2));
  return (size_t)(m + 3 * blocks + 4);
}

hgl_status active_set_launch(double* w, const double* grad, double eta, int64_t m, double* work, int sms,
                             cudaStream_t st) {
  ProfScope prof(HGL_PROF_PROJECT, st);
  const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((m + PROJ_THREADS - 1) / PROJ_THREADS, sms * 2));
  double* v = work;
  double* stats = v + m;
  double* sums = stats + 2 * blocks;
  hgl::count_launch(3);
  k_as_stats<<<blocks, PROJ_THREADS, 0, st>>>(w, grad, m, stats);
  k_as_update<<<blocks, PROJ_THREADS, 0, st>>>(w, grad, eta, m, stats, v, sums);
  k_as_scale<<<blocks, PROJ_THREADS, 0, st>>>(w, v, m, sums);
  HGL_CHECK_CUDA(cudaGetLastError());
  return HGL_OK;
}

size_t project_work_doubles(int64_t m, int sms) {
  const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>((m + PROJ_THREADS - 1) / PROJ_THREADS, sms * 2));
  return (size_t)(m + 2 * blocks + 4);
}

}  // namespace hgl

extern "C" hgl_status hgl_weight_grad(const hgl_graph* g, const double* w, const void* F, const void* Z, int64_t ld,
                                      int32_t c, hgl_dtype dtype, double mu, int32_t flags, double* grad,
                                      void* stream) {
  if (!g || !w || !grad) return hgl::record_error(HGL_ERR_INVALID_ARG, "NULL argument");
  if (c < 1) return hgl::record_error(HGL_ERR_INVALID_ARG, "c must be >= 1");
  if (dtype != HGL_FP64 && dtype != HGL_FP32)
    return hgl::record_error(HGL_ERR_INVALID_ARG, "gradient panels must be FP64 or FP32");
  HGL_TRY(hgl::check_panel(F, ld, c, hgl::dtype_size(dtype), "F"));
  if (Z) HGL_TRY(hgl::check_panel(Z, ld, c, hgl::dtype_size(dtype), "Z"));
  cudaStream_t st = hgl::as_stream(stream);
  hgl_graph* gg = const_cast<hgl_graph*>(g);
  HGL_TRY(hgl::degrees_launch(gg, w, st));
  return hgl::weight_grad_launch(gg, w, F, Z, ld, c, dtype, mu, flags, grad, st);
}

extern "C" hgl_status hgl_active_set_step(double* w, const double* grad, double eta, int64_t m, void* stream) {
  if (!w || !grad || m < 1) return hgl::record_error(HGL_ERR_INVALID_ARG, "w or grad is NULL, or m < 1");
  if (!(eta >= 0.0)) return hgl::record_error(HGL_ERR_INVALID_ARG, "eta must be >= 0");
  cudaStream_t st = hgl::as_stream(stream);
  const int sms = hgl::device_sm_count();
  double* work = nullptr;
  HGL_CHECK_CUDA(cudaMallocAsync(&work, sizeof(double) * hgl::active_set_work_doubles(m, sms), st));
  hgl_status s = hgl::active_set_launch(w, grad, eta, m, work, sms, st);
  cudaFreeAsync(work, st);
  return s;
}

extern "C" hgl_status hgl_project_simplex(double* w, const double* grad, double eta, int64_t m, void* stream) {
  if (!w || m < 1) return hgl::record_error(HGL_ERR_INVALID_ARG, "w is NULL or m < 1");
  cudaStream_t st = hgl::as_stream(stream);
  const int sms = hgl::device_sm_count();
  double* work = nullptr;
  HGL_CHECK_CUDA(cudaMallocAsync(&work, sizeof(double) * hgl::project_work_doubles(m, sms), st));
  hgl_status s = hgl::project_launch(w, grad, eta, m, work, sms, st, 0);
  cudaFreeAsync(work, st);
  return s;
}
