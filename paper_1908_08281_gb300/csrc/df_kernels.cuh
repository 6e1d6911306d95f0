// df_kernels.cuh -- FP64-accurate residual lam Y - M F without FP64 arithmetic.
//
// GB300 runs FP64 FMAs ~58x slower than FP32, so an FP64 operator apply over the
// full panel is arithmetic-bound.  Here every FP64 quantity is held as an unevaluated
// pair of floats x = hi + lo (|lo| <= 2^-24 |hi|, ~48 significant bits) and the two
// gather passes of the operator run in pair arithmetic built from the error-free
// transformations TwoSum (Knuth) and TwoProduct via FMA (Dekker), as in the
// double-float libraries of Dekker (1971) and Hida, Li and Bailey (2001).  The passes
// then move the same bytes as FP64 (two FP32 panels) and stay bandwidth-bound.
#pragma once

#include "hgl_internal.cuh"
#include "panel.cuh"

namespace hgl {
namespace df {

struct f2 {
  float hi, lo;
};

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
}

__device__ __forceinline__ f2 split(double x) {
  f2 r;
  r.hi = __double2float_rn(x);
  r.lo = __double2float_rn(x - (double)r.hi);
  return r;
}

// ---- conversions between FP64 and the FP32 pair without FP64 arithmetic ----
// The panels are converted at the start and end of every mixed-precision solve; with
// the FP64 pipe ~58x slower than FP32, three or four FP64 operations per element made
// those passes FP64-bound.  These work on the IEEE-754 binary64 / binary32 bit fields
// and give the same results as the FP64 conversions; values outside the fast range
// (zero, subnormal, very large or small, infinite, NaN) take the FP64 conversions.

// split(x) from the bits: hi = x rounded to nearest-even at 24 significant bits, lo = the
// exact remainder (an integer of at most 29 bits times 2^(e-52)) rounded to FP32.
__device__ __forceinline__ f2 split_bits(double x) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  const int e = (int)((u >> 52) & 0x7FF) - 1023;
  if (e < -70 || e > 120) return split(x);
  const unsigned long long M = (u & 0xFFFFFFFFFFFFFull) | (1ull << 52);
  unsigned long long H = M >> 29;
  const unsigned long long rem = M & ((1ull << 29) - 1), half = 1ull << 28;
  if (rem > half || (rem == half && (H & 1ull))) ++H;
  const long long R = (long long)M - (long long)(H << 29);  // |R| <= 2^28
  int eh = e;
  if (H == (1ull << 24)) {  // the rounding carried into the next binade
    H >>= 1;
    ++eh;
  }
  const unsigned sign = (unsigned)(u >> 63) << 31;
  f2 r;
  r.hi = __uint_as_float(sign | ((unsigned)(eh + 127) << 23) | (unsigned)(H & 0x7FFFFFull));
  const float scale = __uint_as_float((unsigned)(e - 52 + 127) << 23);  // 2^(e-52), a normal float
  const float lo = __int2float_rn((int)R) * scale;                         // exact scaling
  r.lo = R == 0 ? 0.f : (sign ? -lo : lo);
  return r;
}

// (double)f from the bits (exact).
__device__ __forceinline__ double f2d_bits(float f) {
  const unsigned b = __float_as_uint(f);
  const unsigned long long s = (unsigned long long)(b >> 31) << 63;
  const unsigned eb = (b >> 23) & 0xFFu;
  if ((b & 0x7FFFFFFFu) == 0) return __longlong_as_double((long long)s);
  if (eb == 0 || eb == 0xFFu) return (double)f;
  return __longlong_as_double(
      (long long)(s | ((unsigned long long)(eb + 896u) << 52) | ((unsigned long long)(b & 0x7FFFFFu) << 29)));
}

// acc += a * b
__device__ __forceinline__ void fma2(f2& acc, f2 a, f2 b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float pe = __fmaf_rn(a.hi, b.hi, -p);
  pe = __fmaf_rn(a.hi, b.lo, pe);
  pe = __fmaf_rn(a.lo, b.hi, pe);
  float s, se;
  two_sum(acc.hi, p, s, se);
  const float lo = __fadd_rn(__fadd_rn(acc.lo, se), pe);
  fast_two_sum(s, lo, acc.hi, acc.lo);
}

// acc += a
__device__ __forceinline__ void add2(f2& acc, f2 a) {
  float s, se;
  two_sum(acc.hi, a.hi, s, se);
  const float lo = __fadd_rn(__fadd_rn(acc.lo, a.lo), se);
  fast_two_sum(s, lo, acc.hi, acc.lo);
}

__device__ __forceinline__ f2 mul2(f2 a, f2 b) {
  f2 r{0.f, 0.f};
  fma2(r, a, b);
  return r;
}

constexpr int THREADS = 256;

// hyperedge pass: T[e] = t_e sum_{v in e} s_v F[v]     (F, T as hi/lo panels)
// Heavy hyperedges (the first nheavy of `order`) get one block each; light ones one
// warp each, longest first (as in the operator's hyperedge pass).
// LO is the storage of the low parts that the passes gather (F's and T's): float, or
// bf16_t for the compact residual (the low parts rounded to BF16 cost at most 2^-9 of
// a low part, i.e. 2^-33 of the high part, instead of ~2^-48).
template <int LG, int NV, class LO>
__global__ void __launch_bounds__(THREADS)
k_edge(int64_t m, const int64_t* __restrict__ csc_ptr, const int32_t* __restrict__ csc_idx,
       const int32_t* __restrict__ order, int64_t nheavy, const float* __restrict__ s_hi,
       const float* __restrict__ s_lo, const float* __restrict__ t_hi, const float* __restrict__ t_lo,
       const float* __restrict__ Fh, int64_t ldf, const LO* __restrict__ Fl, int64_t ldfl, int c0, int cw,
       float* __restrict__ Th, LO* __restrict__ Tl, int64_t ldt, const int32_t* __restrict__ guard,
       float* __restrict__ tf, int64_t ldtf, double* __restrict__ ex) {
  if (guard && *guard == 0) return;
  constexpr int E = 4, G = 32 / LG, WARPS = THREADS / 32, TILE = LG * NV * E;
  const int lane = threadIdx.x & 31, grp = lane / LG, l = lane % LG, wid = threadIdx.x >> 5;
  f2 acc[NV][E];
  const bool heavy = blockIdx.x < nheavy;
  const int64_t warp = heavy ? 0 : (((int64_t)blockIdx.x - nheavy) * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = heavy ? 1 : (((int64_t)gridDim.x - nheavy) * blockDim.x) >> 5;
  for (int64_t q = heavy ? blockIdx.x : nheavy + warp; q < (heavy ? (int64_t)blockIdx.x + 1 : m); q += nwarps) {
    const int32_t e = order[q];
    const int64_t beg = __ldg(csc_ptr + e), end = __ldg(csc_ptr + e + 1);
#pragma unroll
    for (int k = 0; k < NV; ++k)
#pragma unroll
      for (int j = 0; j < E; ++j) acc[k][j] = f2{0.f, 0.f};
    const int64_t first = heavy ? beg + wid * G + grp : beg + grp;
    const int64_t step = heavy ? (int64_t)WARPS * G : G;
    for (int64_t i = first; i < end; i += step) {
      const int32_t v = __ldg(csc_idx + i);
      const f2 sv{__ldg(s_hi + v), __ldg(s_lo + v)};
#pragma unroll
      for (int k = 0; k < NV; ++k) {
        const int col = (k * LG + l) * E;
        if (col < cw) {
          float xh[E], xl[E];
          vload<float, float, E>(Fh + (int64_t)v * ldf + c0 + col, xh);
          vload<float, LO, E>(Fl + (int64_t)v * ldfl + c0 + col, xl);
#pragma unroll
          for (int j = 0; j < E; ++j) fma2(acc[k][j], sv, f2{xh[j], xl[j]});
        }
      }
    }
#pragma unroll
    for (int off = LG; off < 32; off <<= 1)
#pragma unroll
      for (int k = 0; k < NV; ++k)
#pragma unroll
        for (int j = 0; j < E; ++j) {
          f2 o{__shfl_xor_sync(0xffffffffu, acc[k][j].hi, off), __shfl_xor_sync(0xffffffffu, acc[k][j].lo, off)};
          add2(acc[k][j], o);
        }
    if (heavy) {
      __shared__ float red_hi[WARPS][TILE], red_lo[WARPS][TILE];
      if (grp == 0)
#pragma unroll
        for (int k = 0; k < NV; ++k)
#pragma unroll
          for (int j = 0; j < E; ++j) {
            red_hi[wid][(k * LG + l) * E + j] = acc[k][j].hi;
            red_lo[wid][(k * LG + l) * E + j] = acc[k][j].lo;
          }
      __syncthreads();
      if (wid != 0) return;
#pragma unroll
      for (int k = 0; k < NV; ++k)
#pragma unroll
        for (int j = 0; j < E; ++j) {
          f2 sum{0.f, 0.f};
          for (int w = 0; w < WARPS; ++w)
            add2(sum, f2{red_hi[w][(k * LG + l) * E + j], red_lo[w][(k * LG + l) * E + j]});
          acc[k][j] = sum;
        }
    }
    if (grp == 0) {
      const f2 te{t_hi[e], t_lo[e]};
      double d = 0.0;  // sum of sigma^2 over this lane's columns (for the gradient)
#pragma unroll
      for (int k = 0; k < NV; ++k) {
        const int col = (k * LG + l) * E;
        if (col < cw) {
          float oh[E], ol[E];
#pragma unroll
          for (int j = 0; j < E; ++j) {
            const f2 r = mul2(te, acc[k][j]);
            oh[j] = r.hi;
            ol[j] = r.lo;
            d += (double)acc[k][j].hi * (double)acc[k][j].hi;
          }
          vstore<float, float, E>(Th + e * ldt + col, oh, E);
          vstore<LO, float, E>(Tl + e * ldt + col, ol, E);
          // the gradient's t * sigma in FP32, full width, at the residual's (final) F
          if (tf) vstore<float, float, E>(tf + e * ldtf + c0 + col, oh, E);
        }
      }
      if (ex) {
        const unsigned gmask = LG == 32 ? 0xffffffffu : ((1u << LG) - 1u);
#pragma unroll
        for (int off = 1; off < LG; off <<= 1) d += __shfl_xor_sync(gmask, d, off);
        if (l == 0) ex[e] = (c0 == 0 ? 0.0 : ex[e]) + d;
      }
    }
  }
}

// vertex pass: z = gy Y[v] + a F[v] + b s_v sum_{e ni v} T[e];  R = fl32(z);
// partials of R.R per column (compensated FP32, FP64 across rows).
template <int LG, int NV, class LO>
__global__ void __launch_bounds__(THREADS)
k_vertex(int64_t n, const int64_t* __restrict__ csr_ptr, const int32_t* __restrict__ csr_idx,
         const float* __restrict__ s_hi, const float* __restrict__ s_lo, const float* __restrict__ Th,
         const LO* __restrict__ Tl, int64_t ldt, const float* __restrict__ Fh, const float* __restrict__ Fl,
         int64_t ldf, const double* __restrict__ Y, int64_t ldy, double a, double b, double gy, int c0, int cw, int c,
         float* __restrict__ R, int64_t ldr, double* __restrict__ partials, const int32_t* __restrict__ guard) {
  if (guard && *guard == 0) return;
  constexpr int E = 4, G = 32 / LG, TILE = LG * NV * E;
  const int lane = threadIdx.x & 31, grp = lane / LG, l = lane % LG, wid = threadIdx.x >> 5;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const f2 a2 = split(a), b2 = split(b), g2 = split(gy);
  DotAcc<float> dot[NV][E];
  for (int64_t v = warp; v < n; v += nwarps) {
    const int64_t beg = __ldg(csr_ptr + v), end = __ldg(csr_ptr + v + 1);
    f2 acc[NV][E];
#pragma unroll
    for (int k = 0; k < NV; ++k)
#pragma unroll
      for (int j = 0; j < E; ++j) acc[k][j] = f2{0.f, 0.f};
    for (int64_t i = beg + grp; i < end; i += G) {
      const int32_t e = __ldg(csr_idx + i);
#pragma unroll
      for (int k = 0; k < NV; ++k) {
        const int col = (k * LG + l) * E;
        if (col < cw) {
          float xh[E], xl[E];
          vload<float, float, E>(Th + (int64_t)e * ldt + col, xh);
          vload<float, LO, E>(Tl + (int64_t)e * ldt + col, xl);
#pragma unroll
          for (int j = 0; j < E; ++j) add2(acc[k][j], f2{xh[j], xl[j]});
        }
      }
    }
#pragma unroll
    for (int off = LG; off < 32; off <<= 1)
#pragma unroll
      for (int k = 0; k < NV; ++k)
#pragma unroll
        for (int j = 0; j < E; ++j) {
          f2 o{__shfl_xor_sync(0xffffffffu, acc[k][j].hi, off), __shfl_xor_sync(0xffffffffu, acc[k][j].lo, off)};
          add2(acc[k][j], o);
        }
    if (grp == 0) {
      const f2 sv{s_hi[v], s_lo[v]};
      const f2 sb = mul2(b2, sv);
#pragma unroll
      for (int k = 0; k < NV; ++k) {
        const int col = (k * LG + l) * E;
        if (col < cw) {
          float fh[E], fl[E], r[E];
          vload<float, float, E>(Fh + v * ldf + c0 + col, fh);
          vload<float, float, E>(Fl + v * ldf + c0 + col, fl);
          const int nv = cw - col < E ? cw - col : E;
#pragma unroll
          for (int j = 0; j < E; ++j) {
            const double y = j < nv ? Y[v * ldy + c0 + col + j] : 0.0;
            f2 z = mul2(g2, split(y));
            fma2(z, a2, f2{fh[j], fl[j]});
            fma2(z, sb, acc[k][j]);
            r[j] = __fadd_rn(z.hi, z.lo);
            dot[k][j].add(r[j], r[j]);
          }
          vstore<float, float, E>(R + v * ldr + c0 + col, r, nv);
        }
      }
    }
  }
  __shared__ double red[TILE];
  for (int q = threadIdx.x; q < TILE; q += blockDim.x) red[q] = 0.0;
  __syncthreads();
  for (int w = 0; w < THREADS / 32; ++w) {
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

// (hi, lo) <- FP64 vector
__global__ void k_split_vec(int64_t len, const double* __restrict__ x, float* __restrict__ hi, float* __restrict__ lo) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < len; i += (int64_t)gridDim.x * blockDim.x) {
    const f2 r = split(x[i]);
    hi[i] = r.hi;
    lo[i] = r.lo;
  }
}

// (Fh, Fl) <- F (FP64 panel), or (Fh, Fl) += D (FP32 panel), or F <- Fh + Fl.
// With Fl16, SPLIT and ACCUMULATE also store the low part rounded to BF16 (the copy the
// compact residual gathers).  One warp per row.
enum PanelOp : int { SPLIT = 0, ACCUMULATE = 1, COMBINE = 2 };

template <int OP>
__global__ void k_panel(int64_t n, int c, double* __restrict__ F, int64_t ldf, float* __restrict__ Fh,
                        float* __restrict__ Fl, int64_t ld32, const float* __restrict__ D,
                        const int32_t* __restrict__ guard, bf16_t* __restrict__ Fl16, int64_t ld16) {
  if (guard && *guard == 0) return;
  const int vecs = (c + 3) / 4;
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  // one warp per row, lanes over its 4-column vectors (coalesced; FP64 rows read and
  // written as 2 x 16 bytes per vector: ldf * 8 is a multiple of 16 and col of 4)
  for (int64_t r = warp; r < n; r += nwarps) {
    for (int vi = lane; vi < vecs; vi += 32) {
      const int col = vi * 4;
      const int nv = c - col < 4 ? c - col : 4;
      float h[4], lo[4];
      if (OP == SPLIT) {
        double x[4] = {0.0, 0.0, 0.0, 0.0};
        if (nv == 4) {
          const double2 a = reinterpret_cast<const double2*>(F + r * ldf + col)[0];
          const double2 b = reinterpret_cast<const double2*>(F + r * ldf + col)[1];
          x[0] = a.x;
          x[1] = a.y;
          x[2] = b.x;
          x[3] = b.y;
        } else {
          for (int j = 0; j < nv; ++j) x[j] = F[r * ldf + col + j];
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const f2 y = split_bits(x[j]);
          h[j] = y.hi;
          lo[j] = y.lo;
        }
        vstore<float, float, 4>(Fh + r * ld32 + col, h, 4);
        vstore<float, float, 4>(Fl + r * ld32 + col, lo, 4);
        if (Fl16) vstore<bf16_t, float, 4>(Fl16 + r * ld16 + col, lo, 4);
      } else if (OP == ACCUMULATE) {
        float d[4];
        vload<float, float, 4, false>(Fh + r * ld32 + col, h);
        vload<float, float, 4, false>(Fl + r * ld32 + col, lo);
        vload<float, float, 4, false>(D + r * ld32 + col, d);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          if (j >= nv) d[j] = 0.f;  // columns past c are padding
          f2 x{h[j], lo[j]};
          add2(x, f2{d[j], 0.f});
          h[j] = x.hi;
          lo[j] = x.lo;
        }
        vstore<float, float, 4>(Fh + r * ld32 + col, h, 4);
        vstore<float, float, 4>(Fl + r * ld32 + col, lo, 4);
        if (Fl16) vstore<bf16_t, float, 4>(Fl16 + r * ld16 + col, lo, 4);
      } else {
        vload<float, float, 4, false>(Fh + r * ld32 + col, h);
        vload<float, float, 4, false>(Fl + r * ld32 + col, lo);
        if (nv == 4) {
          reinterpret_cast<double2*>(F + r * ldf + col)[0] =
              make_double2(f2d_bits(h[0]) + f2d_bits(lo[0]), f2d_bits(h[1]) + f2d_bits(lo[1]));
          reinterpret_cast<double2*>(F + r * ldf + col)[1] =
              make_double2(f2d_bits(h[2]) + f2d_bits(lo[2]), f2d_bits(h[3]) + f2d_bits(lo[3]));
        } else {
          for (int j = 0; j < nv; ++j) F[r * ldf + col + j] = f2d_bits(h[j]) + f2d_bits(lo[j]);
        }
      }
    }
  }
}

}  // namespace df
}  // namespace hgl
