// panel.cuh -- element types, vector loads/stores and compensated dot accumulators
// shared by the panel kernels.
#pragma once

#include <cuda_bf16.h>

#include <cstdint>

namespace hgl {

// BF16 panel element (raw bits; converted to FP32 on load).
struct bf16_t {
  uint16_t x;
};

template <class T> struct AccOf { using type = float; };
template <> struct AccOf<double> { using type = double; };

template <class T> struct Elem;
template <> struct Elem<double> {
  template <class A> __device__ static __forceinline__ A get(const uint32_t* u, int i) {
    return (A)__hiloint2double((int)u[2 * i + 1], (int)u[2 * i]);
  }
  template <class A> __device__ static __forceinline__ void put(uint32_t* u, int i, A v) {
    double d = (double)v;
    u[2 * i] = (uint32_t)__double2loint(d);
    u[2 * i + 1] = (uint32_t)__double2hiint(d);
  }
};
template <> struct Elem<float> {
  template <class A> __device__ static __forceinline__ A get(const uint32_t* u, int i) {
    return (A)__uint_as_float(u[i]);
  }
  template <class A> __device__ static __forceinline__ void put(uint32_t* u, int i, A v) {
    u[i] = __float_as_uint((float)v);
  }
};
template <> struct Elem<bf16_t> {
  template <class A> __device__ static __forceinline__ A get(const uint32_t* u, int i) {
    return (A)__uint_as_float(((u[i >> 1] >> ((i & 1) * 16)) & 0xffffu) << 16);
  }
  template <class A> __device__ static __forceinline__ void put(uint32_t* u, int i, A v) {
    uint32_t bits = __bfloat16_as_ushort(__float2bfloat16_rn((float)v));
    if (i & 1)
      u[i >> 1] = (u[i >> 1] & 0x0000ffffu) | (bits << 16);
    else
      u[i >> 1] = (u[i >> 1] & 0xffff0000u) | bits;
  }
};

// Load B bytes (B in {4, 8, 16, 32, 64}) from an address aligned to min(B, 16).
template <int B, bool RO>
__device__ __forceinline__ void raw_load(const void* p, uint32_t* u) {
  if constexpr (B >= 16) {
#pragma unroll
    for (int i = 0; i < B / 16; ++i) {
      uint4 v = RO ? __ldg(reinterpret_cast<const uint4*>(p) + i) : reinterpret_cast<const uint4*>(p)[i];
      u[4 * i] = v.x;
      u[4 * i + 1] = v.y;
      u[4 * i + 2] = v.z;
      u[4 * i + 3] = v.w;
    }
  } else if constexpr (B == 8) {
    uint2 v = RO ? __ldg(reinterpret_cast<const uint2*>(p)) : *reinterpret_cast<const uint2*>(p);
    u[0] = v.x;
    u[1] = v.y;
  } else {
    static_assert(B == 4, "unsupported width");
    u[0] = RO ? __ldg(reinterpret_cast<const unsigned*>(p)) : *reinterpret_cast<const unsigned*>(p);
  }
}

template <int B>
__device__ __forceinline__ void raw_store(void* p, const uint32_t* u) {
  if constexpr (B >= 16) {
#pragma unroll
    for (int i = 0; i < B / 16; ++i)
      reinterpret_cast<uint4*>(p)[i] = make_uint4(u[4 * i], u[4 * i + 1], u[4 * i + 2], u[4 * i + 3]);
  } else if constexpr (B == 8) {
    *reinterpret_cast<uint2*>(p) = make_uint2(u[0], u[1]);
  } else {
    static_assert(B == 4, "unsupported width");
    *reinterpret_cast<unsigned*>(p) = u[0];
  }
}

// N consecutive elements of T as accumulator type A.
template <class A, class T, int N, bool RO = true>
__device__ __forceinline__ void vload(const T* p, A* o) {
  constexpr int B = N * (int)sizeof(T);
  uint32_t u[B / 4];
  raw_load<B, RO>(p, u);
#pragma unroll
  for (int i = 0; i < N; ++i) o[i] = Elem<T>::template get<A>(u, i);
}

// Store N elements; if nvalid < N only the first nvalid are written (element-wise).
template <class T, class A, int N>
__device__ __forceinline__ void vstore(T* p, const A* v, int nvalid) {
  constexpr int B = N * (int)sizeof(T);
  uint32_t u[B / 4];
#pragma unroll
  for (int i = 0; i < B / 4; ++i) u[i] = 0;
#pragma unroll
  for (int i = 0; i < N; ++i) Elem<T>::template put<A>(u, i, v[i]);
  if (nvalid >= N) {
    raw_store<B>(p, u);
  } else {
    for (int i = 0; i < nvalid; ++i) {
      if constexpr (sizeof(T) == 8) {
        reinterpret_cast<unsigned long long*>(p)[i] =
            ((unsigned long long)u[2 * i + 1] << 32) | (unsigned long long)u[2 * i];
      } else if constexpr (sizeof(T) == 4) {
        reinterpret_cast<unsigned*>(p)[i] = u[i];
      } else {
        reinterpret_cast<unsigned short*>(p)[i] = (unsigned short)((u[i >> 1] >> ((i & 1) * 16)) & 0xffffu);
      }
    }
  }
}

// Per-lane dot-product accumulator.  FP64 accumulates natively.  FP32 uses the
// compensated Dot2 scheme of Ogita, Rump and Oishi ("Accurate sum and dot product",
// SIAM J. Sci. Comput. 2005): the rounding error of every product (TwoProduct via
// FMA) and of every addition (TwoSum) is carried in a second float, so the result
// is as accurate as if the sum were formed in about twice the working precision.
template <class A> struct DotAcc;
template <> struct DotAcc<double> {
  double s = 0.0;
  __device__ __forceinline__ void add(double a, double b) { s = fma(a, b, s); }
  __device__ __forceinline__ double value() const { return s; }
};
template <> struct DotAcc<float> {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float a, float b) {
    float p = __fmul_rn(a, b);
    float pe = __fmaf_rn(a, b, -p);
    float t = __fadd_rn(s, p);
    float bp = __fsub_rn(t, s);
    float se = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(p, bp));
    s = t;
    c = __fadd_rn(c, __fadd_rn(se, pe));
  }
  __device__ __forceinline__ double value() const { return (double)s + (double)c; }
};

}  // namespace hgl
