// Shared-memory FFT building blocks for the AIM grid product (Eq. 8 / Eq. 10).
//
// A CTA transforms `nfft` independent sequences of length 2^logH stored back to back in
// shared memory. Each pass is a Stockham auto-sort radix-R step (natural order in and out):
// butterfly j of a pass with current sub-transform length Ns reads X[j + r*H/R], applies the
// twiddles W_{Ns R}^{(j mod Ns) r}, a length-R DFT, and writes
// X[(j - j mod Ns) R + j mod Ns + r Ns]. Every butterfly of a pass is held in registers
// between one barrier and the next, so a pass runs in place. Twiddles come from a table
// tw[t] = exp(-2 pi i t / P) computed on the host in FP64 (no device sin/cos).
#pragma once

#include <cuda_runtime.h>

namespace aim {

template <typename T2> __device__ __forceinline__ T2 cadd(T2 a, T2 b) { return T2{a.x + b.x, a.y + b.y}; }
template <typename T2> __device__ __forceinline__ T2 csub(T2 a, T2 b) { return T2{a.x - b.x, a.y - b.y}; }
template <typename T2> __device__ __forceinline__ T2 cmul(T2 a, T2 b) {
  return T2{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
// a * conj(b)
template <typename T2> __device__ __forceinline__ T2 cmulc(T2 a, T2 b) {
  return T2{a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y};
}
// complex64 sums and differences as one paired FP32 instruction each (both parts in one lane pair)
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }
// complex64 products as a paired multiply and a paired fused multiply-add:
// a b = ax (bx, by) + (-ay by, ay bx),  a conj(b) = ax (bx, -by) + (ay by, ay bx)
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  const float2 p = __fmul2_rn(make_float2(a.y, a.y), make_float2(b.y, b.x));
  return __ffma2_rn(make_float2(a.x, a.x), b, make_float2(-p.x, p.y));
}
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {
  const float2 p = __fmul2_rn(make_float2(a.y, a.y), make_float2(b.y, b.x));
  return __ffma2_rn(make_float2(a.x, a.x), make_float2(b.x, -b.y), p);
}
template <typename T2> __device__ __forceinline__ T2 mul_minus_i(T2 a) { return T2{a.y, -a.x}; }
template <typename T2> __device__ __forceinline__ T2 mul_plus_i(T2 a) { return T2{-a.y, a.x}; }

template <bool INV, typename T2> __device__ __forceinline__ void dft_small(T2 (&v)[2]) {
  T2 a = v[0], b = v[1];
  v[0] = cadd(a, b);
  v[1] = csub(a, b);
}

template <bool INV, typename T2> __device__ __forceinline__ void dft_small(T2 (&v)[4]) {
  // forward uses W4 = -i, inverse W4 = +i
  T2 a0 = cadd(v[0], v[2]), a1 = csub(v[0], v[2]);
  T2 b0 = cadd(v[1], v[3]), b1 = csub(v[1], v[3]);
  b1 = INV ? mul_plus_i(b1) : mul_minus_i(b1);
  v[0] = cadd(a0, b0);
  v[2] = csub(a0, b0);
  v[1] = cadd(a1, b1);
  v[3] = csub(a1, b1);
}

// One radix-R Stockham pass over nfft sequences of length 2^logH at buf + f * 2^logH.
// NB bounds the butterflies a thread holds: nfft * 2^logH / R <= NB * blockDim.x.
template <int R, int NB, bool INV, typename T2>
__device__ __forceinline__ void stockham_pass(T2* __restrict__ buf, int logH, int nfft, int logNs,
                                              const T2* __restrict__ tw, int logP) {
  constexpr int logR = (R == 2) ? 1 : 2;
  const int lognb = logH - logR;
  const int nbmask = (1 << lognb) - 1;
  const int total = nfft << lognb;
  const int nsmask = (1 << logNs) - 1;
  const int twsh = logP - logNs - logR;
  T2 v[NB][R];
  int ob[NB];
#pragma unroll
  for (int t = 0; t < NB; ++t) {
    const int b = threadIdx.x + t * blockDim.x;
    ob[t] = -1;
    if (b < total) {
      const int f = b >> lognb;
      const int j = b & nbmask;
      const int k = j & nsmask;
      const T2* X = buf + (f << logH);
#pragma unroll
      for (int r = 0; r < R; ++r) v[t][r] = X[j + (r << lognb)];
      if (k != 0) {
#pragma unroll
        for (int r = 1; r < R; ++r) {
          const T2 w = tw[(k * r) << twsh];
          v[t][r] = INV ? cmulc(v[t][r], w) : cmul(v[t][r], w);
        }
      }
      dft_small<INV>(v[t]);
      ob[t] = (f << logH) + ((j - k) << logR) + k;
    }
  }
  __syncthreads();
#pragma unroll
  for (int t = 0; t < NB; ++t) {
    if (ob[t] >= 0) {
#pragma unroll
      for (int r = 0; r < R; ++r) buf[ob[t] + (r << logNs)] = v[t][r];
    }
  }
  __syncthreads();
}

// In-place unnormalised DFT (forward: exp(-2 pi i jk/H), inverse: exp(+2 pi i jk/H)) of nfft
// sequences of length H = 2^logH in shared memory. Requires nfft*H/4 <= NB*blockDim.x and
// H <= P (the twiddle table length, P = 2^logP). Starts and ends with a barrier-consistent
// buffer: callers must __syncthreads() after writing the input.
template <int NB, bool INV, typename T2>
__device__ __forceinline__ void smem_fft(T2* __restrict__ buf, int logH, int nfft,
                                         const T2* __restrict__ tw, int logP) {
  int logNs = 0;
  if (logH & 1) {
    stockham_pass<2, 2 * NB, INV>(buf, logH, nfft, 0, tw, logP);
    logNs = 1;
  }
  for (; logNs < logH; logNs += 2) stockham_pass<4, NB, INV>(buf, logH, nfft, logNs, tw, logP);
}

}  // namespace aim
