// Complex element types of the grid product and their traits.
//   float2  : complex64 ("mixed" precision)
//   dfc     : double-float complex, FP64-class accuracy on the FP32 pipe (default FP64 mode)
//   double2 : IEEE binary64 complex (native FP64 mode)
#pragma once

#include "dfloat.cuh"
#include "fft_reg.cuh"

namespace aim {

template <typename CT> struct GridT;
// W: column-tile width (W * sizeof(CT) = 32 bytes); VT: type of restricted grid values handed
// to the gather; MaxThreads: launch bound (16-byte types hold 32 x 16 bytes per thread).
// MaxThreads is the launch bound with one transform of 16 elements per thread (TPT = 1); with two
// transforms per thread (TPT = 2) a CTA of the same work has half the threads, with 8 elements
// per thread twice as many (at most 1024).
template <> struct GridT<float2> {
  using VT = float2;
  static constexpr int W = 4, MaxThreads = 1024;
};
template <> struct GridT<double2> {
  using VT = double2;
  static constexpr int W = 2, MaxThreads = 512;
};
template <> struct GridT<dfc> {
  using VT = double2;
  static constexpr int W = 2, MaxThreads = 512;
};
// a double-float complex product is ~40 FP32-pipe instructions: twiddles come whole from the table
template <> struct TwiddleFromTable<dfc> { static constexpr bool value = true; };

template <typename CT, int TPT, int LOGE> struct LaunchMax {
  // fewer elements per thread: the same registers per thread hold the work of fewer elements,
  // so the same register file holds more threads
  static constexpr int base = TPT == 1 ? GridT<CT>::MaxThreads : GridT<CT>::MaxThreads / 2;
  static constexpr int value = (base << (4 - LOGE)) > 1024 ? 1024 : (base << (4 - LOGE));
};

template <typename CT> __device__ __forceinline__ CT czero();
template <> __device__ __forceinline__ float2 czero<float2>() { return float2{0.f, 0.f}; }
template <> __device__ __forceinline__ double2 czero<double2>() { return double2{0.0, 0.0}; }
template <> __device__ __forceinline__ dfc czero<dfc>() { return dfc{0.f, 0.f, 0.f, 0.f}; }

template <typename CT> __device__ __forceinline__ CT cfrom(double re, double im);
template <> __device__ __forceinline__ float2 cfrom<float2>(double re, double im) {
  return float2{(float)re, (float)im};
}
template <> __device__ __forceinline__ double2 cfrom<double2>(double re, double im) { return double2{re, im}; }
template <> __device__ __forceinline__ dfc cfrom<dfc>(double re, double im) {
  dfc r;
  df_split(re, r.xh, r.xl);
  df_split(im, r.yh, r.yl);
  return r;
}

__device__ __forceinline__ double2 cto_d2(float2 v, double s) { return double2{(double)v.x * s, (double)v.y * s}; }
__device__ __forceinline__ double2 cto_d2(double2 v, double s) { return double2{v.x * s, v.y * s}; }
__device__ __forceinline__ double2 cto_d2(dfc v, double s) {
  return double2{((double)v.xh + (double)v.xl) * s, ((double)v.yh + (double)v.yl) * s};
}

// value handed to the gather (restricted grid value times the 1/P^2 of the inverse DFT)
__device__ __forceinline__ float2 cto_vt(float2 v, double s) { return float2{v.x * (float)s, v.y * (float)s}; }
__device__ __forceinline__ double2 cto_vt(double2 v, double s) { return cto_d2(v, s); }
__device__ __forceinline__ double2 cto_vt(dfc v, double s) { return cto_d2(v, s); }

// tables of double-float values are float4 (xh, yh, xl, yl), the order of dfc
__device__ __forceinline__ dfc ldro(const dfc* p) {
  const float4 v = __ldg(reinterpret_cast<const float4*>(p));
  return dfc{v.x, v.y, v.z, v.w};
}

// value held by the partner lane (lane ^ 1); all 32 lanes must call it together
__device__ __forceinline__ float2 shfl_pair(float2 v) {
  return float2{__shfl_xor_sync(0xffffffffu, v.x, 1), __shfl_xor_sync(0xffffffffu, v.y, 1)};
}
__device__ __forceinline__ double2 shfl_pair(double2 v) {
  return double2{__shfl_xor_sync(0xffffffffu, v.x, 1), __shfl_xor_sync(0xffffffffu, v.y, 1)};
}
__device__ __forceinline__ dfc shfl_pair(dfc v) {
  dfc r;
  r.xh = __shfl_xor_sync(0xffffffffu, v.xh, 1);
  r.yh = __shfl_xor_sync(0xffffffffu, v.yh, 1);
  r.xl = __shfl_xor_sync(0xffffffffu, v.xl, 1);
  r.yl = __shfl_xor_sync(0xffffffffu, v.yl, 1);
  return r;
}

}  // namespace aim
