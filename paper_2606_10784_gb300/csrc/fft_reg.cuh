// Register-resident FFT passes for the AIM grid product (Eq. 8 / Eq. 10).
//
// Each thread owns E = 2^LOGE elements (E = 16 or 8) of every transform it works on. A
// length-H = 2^logH transform is split into radix-E passes plus at most one pass of a smaller
// radix (logH = q LOGE + rem); in a radix-R pass a thread does E/R butterflies. Butterflies
// follow the Stockham auto-sort indexing (natural order in and out): butterfly b of a pass with
// current sub-length Ns reads X[b + r H/R], multiplies by W_{Ns R}^{(b mod Ns) r}, does a
// length-R DFT in registers and writes X[(b - b mod Ns) R + b mod Ns + r Ns].
// Shared memory holds the exchange between passes, padded by one element every E so that the
// stride-E writes of the first pass do not collide in banks. Twiddles come from the
// host-computed FP64 table tw[t] = exp(-2 pi i t/P).
#pragma once

#include <cuda_runtime.h>

#include "fft.cuh"

namespace aim {

template <int LOGE>
__host__ __device__ __forceinline__ int padi(int i) { return i + (i >> LOGE); }
// Stride between the transforms of a CTA: the padded length plus 2, so that transforms whose
// lanes share a warp (the even/odd halves and the columns of a tile) start 2 elements apart.
template <int LOGE>
__host__ __device__ __forceinline__ int padded_len(int H) { return H + (H >> LOGE) + 2; }

// read-only load of a twiddle / spectrum entry
__device__ __forceinline__ float2 ldro(const float2* p) { return __ldg(p); }
__device__ __forceinline__ double2 ldro(const double2* p) { return __ldg(p); }

template <int R>
__host__ __device__ constexpr int bitrev_r(int k) {
  return R == 2 ? k
       : R == 4 ? ((k & 1) << 1) | ((k >> 1) & 1)
       : R == 8 ? ((k & 1) << 2) | (k & 2) | ((k >> 2) & 1)
                : ((k & 1) << 3) | ((k & 2) << 1) | ((k >> 1) & 2) | ((k >> 3) & 1);
}

// d * W16^e (forward W16 = exp(-2 pi i/16); inverse uses the conjugate), e in [0, 8)
template <bool INV, typename T2>
__device__ __forceinline__ T2 rot16(T2 d, int e) {
  using T = decltype(d.x);
  constexpr double C1 = 0.92387953251128675613, S1 = 0.38268343236508977173, C2 = 0.70710678118654752440;
  switch (e) {
    case 0: return d;
    case 4: return INV ? mul_plus_i(d) : mul_minus_i(d);
    default: {
      double c, s;   // exp(-i 2 pi e/16) = c - i s
      switch (e) {
        case 1: c = C1; s = S1; break;
        case 2: c = C2; s = C2; break;
        case 3: c = S1; s = C1; break;
        case 5: c = -S1; s = C1; break;
        case 6: c = -C2; s = C2; break;
        default: c = -C1; s = S1; break;   // 7
      }
      const T cc = (T)c, ss = INV ? (T)(-s) : (T)s;
      return T2{d.x * cc + d.y * ss, d.y * cc - d.x * ss};
    }
  }
}

// In-register DFT of length R (2, 4, 8, 16): radix-2 decimation in frequency, then the
// bit-reversal permutation (resolved at compile time).
template <int R, bool INV, typename T2>
__device__ __forceinline__ void dft_reg(T2 (&v)[R]) {
#pragma unroll
  for (int len = R; len >= 2; len >>= 1) {
    const int half = len >> 1;
#pragma unroll
    for (int o = 0; o < R; o += len) {
#pragma unroll
      for (int i = 0; i < half; ++i) {
        const T2 a = v[o + i], b = v[o + i + half];
        v[o + i] = cadd(a, b);
        v[o + i + half] = rot16<INV>(csub(a, b), i * (16 / len));
      }
    }
  }
  T2 t[R];
#pragma unroll
  for (int k = 0; k < R; ++k) t[k] = v[bitrev_r<R>(k)];
#pragma unroll
  for (int k = 0; k < R; ++k) v[k] = t[k];
}

// Where the twiddles of a pass come from. Complex64: only the powers r = 1, 2, 4, 8 are read
// from the table and the others are products of at most three of them (a scattered table read
// per power costs more L1 wavefronts than the products cost FMAs, and the complex64 passes keep
// L1 busy). Types whose complex product costs tens of FP32-pipe instructions (double-float) or
// runs on the slow FP64 pipe (binary64) read every factor from the table instead.
template <typename T2> struct TwiddleFromTable { static constexpr bool value = false; };
template <> struct TwiddleFromTable<double2> { static constexpr bool value = true; };

// The twiddles W_{Ns R}^{k r}, r = 1..R-1, of butterfly position k (k != 0): app(r, w) for each.
// All transforms a thread works on at the same butterfly position share them, so callers apply
// each factor to all of them before the next one is formed.
template <int LOGR, typename T2, typename App>
__device__ __forceinline__ void twiddles(int k, int logNs, const T2* __restrict__ tw, int logP, App app) {
  constexpr int R = 1 << LOGR;
  const int sh = logP - logNs - LOGR;
  if constexpr (TwiddleFromTable<T2>::value) {
    // (r k) << sh < R Ns 2^sh = P: inside the table
#pragma unroll
    for (int r = 1; r < R; ++r) app(r, ldro(&tw[(r * k) << sh]));
  } else {
    const T2 w1 = ldro(&tw[k << sh]);
    app(1, w1);
    if constexpr (R > 2) {
      const T2 w2 = ldro(&tw[(2 * k) << sh]);
      app(2, w2);
      const T2 w3 = cmul(w2, w1);
      app(3, w3);
      if constexpr (R > 4) {
        const T2 w4 = ldro(&tw[(4 * k) << sh]);
        app(4, w4);
        const T2 w5 = cmul(w4, w1);
        app(5, w5);
        const T2 w6 = cmul(w4, w2);
        app(6, w6);
        const T2 w7 = cmul(w4, w3);
        app(7, w7);
        if constexpr (R > 8) {
          const T2 w8 = ldro(&tw[(8 * k) << sh]);
          app(8, w8);
          app(9, cmul(w8, w1));
          app(10, cmul(w8, w2));
          app(11, cmul(w8, w3));
          app(12, cmul(w8, w4));
          app(13, cmul(w8, w5));
          app(14, cmul(w8, w6));
          app(15, cmul(w8, w7));
        }
      }
    }
  }
}

// Twiddles of position k applied to the NF transforms v[f][t][.] (one set of factors for all),
// then their length-R DFTs.
template <int LOGR, bool INV, int NF, int NB, typename T2>
__device__ __forceinline__ void bfly_shared(T2 (&v)[NF][NB][1 << LOGR], int t, int k, int logNs,
                                            const T2* __restrict__ tw, int logP) {
  if (k != 0)
    twiddles<LOGR>(k, logNs, tw, logP, [&](int r, const T2& w) {
#pragma unroll
      for (int f = 0; f < NF; ++f) v[f][t][r] = INV ? cmulc(v[f][t][r], w) : cmul(v[f][t][r], w);
    });
#pragma unroll
  for (int f = 0; f < NF; ++f) dft_reg<1 << LOGR, INV>(v[f][t]);
}

template <int LOGE>
__device__ __forceinline__ int fft_npass(int logH) { return logH / LOGE + (logH % LOGE != 0); }
template <int LOGE>
__device__ __forceinline__ int fft_logr(int pass, int logH) { return pass < logH / LOGE ? LOGE : logH % LOGE; }

// One pass over NF transforms owned by this thread group, shared memory in and out.
// Each thread works on butterflies b = j + t*tpf (t < E/R) of each of its transforms, whose
// padded bases in shared memory are fb[f]. `post(f, out_index, value)` may rewrite a value
// before it is stored (identity for plain passes). Barrier before and after the stores.
template <int LOGR, bool INV, int NF, int LOGE, typename T2, typename Post>
__device__ __forceinline__ void smem_pass(T2* __restrict__ sm, const int (&fb)[NF], int j, int tpf, int logH,
                                          int logNs, const T2* __restrict__ tw, int logP, Post post) {
  constexpr int R = 1 << LOGR, NB = (1 << LOGE) >> LOGR;
  const int lognb = logH - LOGR;
  const int nsm = (1 << logNs) - 1;
  T2 v[NF][NB][R];
#pragma unroll
  for (int t = 0; t < NB; ++t) {
    const int b = j + t * tpf;
#pragma unroll
    for (int f = 0; f < NF; ++f)
#pragma unroll
      for (int r = 0; r < R; ++r) v[f][t][r] = sm[fb[f] + padi<LOGE>(b + (r << lognb))];
    bfly_shared<LOGR, INV>(v, t, b & nsm, logNs, tw, logP);
  }
  __syncthreads();
#pragma unroll
  for (int f = 0; f < NF; ++f)
#pragma unroll
    for (int t = 0; t < NB; ++t) {
      const int b = j + t * tpf;
      const int k = b & nsm;
      const int base = ((b - k) << LOGR) + k;
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int o = base + (r << logNs);
        sm[fb[f] + padi<LOGE>(o)] = post(f, o, v[f][t][r]);
      }
    }
  __syncthreads();
}

// Last pass: shared memory in, `emit(t, r, out_index, values[NF])` out (no stores to shared
// memory here; callers that write shared memory in `emit` must place a barrier first).
template <int LOGR, bool INV, int NF, int LOGE, typename T2, typename Emit>
__device__ __forceinline__ void last_pass(const T2* __restrict__ sm, const int (&fb)[NF], int j, int tpf, int logH,
                                          int logNs, const T2* __restrict__ tw, int logP, Emit emit) {
  constexpr int R = 1 << LOGR, NB = (1 << LOGE) >> LOGR;
  const int lognb = logH - LOGR;
  const int nsm = (1 << logNs) - 1;
#pragma unroll
  for (int t = 0; t < NB; ++t) {
    const int b = j + t * tpf;
    const int k = b & nsm;
    T2 v[NF][1][R];
#pragma unroll
    for (int f = 0; f < NF; ++f)
#pragma unroll
      for (int r = 0; r < R; ++r) v[f][0][r] = sm[fb[f] + padi<LOGE>(b + (r << lognb))];
    bfly_shared<LOGR, INV>(v, 0, k, logNs, tw, logP);
    const int base = ((b - k) << LOGR) + k;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      T2 vals[NF];
#pragma unroll
      for (int f = 0; f < NF; ++f) vals[f] = v[f][0][r];
      emit(base + (r << logNs), vals);
    }
  }
}

// Runs passes [p0, p1) of a length-2^logH transform in shared memory, dispatching the radix.
template <bool INV, int NF, int LOGE, typename T2, typename Post>
__device__ __forceinline__ void smem_passes(T2* sm, const int (&fb)[NF], int j, int tpf, int logH, int p0, int p1,
                                            int logNs, const T2* tw, int logP, Post post) {
  for (int p = p0; p < p1; ++p) {
    const int lr = fft_logr<LOGE>(p, logH);
    if (lr == LOGE) {
      smem_pass<LOGE, INV, NF, LOGE>(sm, fb, j, tpf, logH, logNs, tw, logP, post);
    } else {
      switch (lr) {
        case 3: if constexpr (LOGE > 3) smem_pass<3, INV, NF, LOGE>(sm, fb, j, tpf, logH, logNs, tw, logP, post); break;
        case 2: smem_pass<2, INV, NF, LOGE>(sm, fb, j, tpf, logH, logNs, tw, logP, post); break;
        default: smem_pass<1, INV, NF, LOGE>(sm, fb, j, tpf, logH, logNs, tw, logP, post); break;
      }
    }
    logNs += lr;
  }
}

template <bool INV, int NF, int LOGE, typename T2, typename Emit>
__device__ __forceinline__ void last_pass_dispatch(const T2* sm, const int (&fb)[NF], int j, int tpf, int logH,
                                                   int logNs, const T2* tw, int logP, Emit emit) {
  const int lr = fft_logr<LOGE>(fft_npass<LOGE>(logH) - 1, logH);
  if (lr == LOGE) {
    last_pass<LOGE, INV, NF, LOGE>(sm, fb, j, tpf, logH, logNs, tw, logP, emit);
  } else {
    switch (lr) {
      case 3: if constexpr (LOGE > 3) last_pass<3, INV, NF, LOGE>(sm, fb, j, tpf, logH, logNs, tw, logP, emit); break;
      case 2: last_pass<2, INV, NF, LOGE>(sm, fb, j, tpf, logH, logNs, tw, logP, emit); break;
      default: last_pass<1, INV, NF, LOGE>(sm, fb, j, tpf, logH, logNs, tw, logP, emit); break;
    }
  }
}

// The middle of a convolution: the last forward pass, the pointwise product, and the first
// pass of the inverse transform, in registers. The last Stockham pass (Ns = H/R) of butterfly b
// writes the outputs X[b + r H/R], which are exactly the inputs of butterfly b of an inverse
// pass with the same radix R and Ns = 1. So when the inverse runs its radices in the reverse
// order (R first, then the radix-E passes), nothing goes through shared memory between the
// two. `mul(f, k, value)` multiplies forward output k of transform f. The inverse pass writes
// its outputs (index b R + r) to shared memory: barrier before and after the stores.
template <int LOGR, int NF, int LOGE, typename T2, typename Mul>
__device__ __forceinline__ void conv_mid_pass(T2* __restrict__ sm, const int (&fb)[NF], int j, int tpf, int logH,
                                              const T2* __restrict__ tw, int logP, Mul mul) {
  constexpr int R = 1 << LOGR, NB = (1 << LOGE) >> LOGR;
  const int lognb = logH - LOGR;
  T2 v[NF][NB][R];
#pragma unroll
  for (int t = 0; t < NB; ++t) {
    const int b = j + t * tpf;
#pragma unroll
    for (int f = 0; f < NF; ++f)
#pragma unroll
      for (int r = 0; r < R; ++r) v[f][t][r] = sm[fb[f] + padi<LOGE>(b + (r << lognb))];
    bfly_shared<LOGR, false>(v, t, b, lognb, tw, logP);   // Ns = H/R, so b mod Ns = b
#pragma unroll
    for (int f = 0; f < NF; ++f) {
#pragma unroll
      for (int r = 0; r < R; ++r) v[f][t][r] = mul(f, b + (r << lognb), v[f][t][r]);
      dft_reg<R, true>(v[f][t]);                          // inverse pass with Ns = 1: no twiddles
    }
  }
  __syncthreads();
#pragma unroll
  for (int f = 0; f < NF; ++f)
#pragma unroll
    for (int t = 0; t < NB; ++t) {
      const int b = j + t * tpf;
#pragma unroll
      for (int r = 0; r < R; ++r) sm[fb[f] + padi<LOGE>((b << LOGR) + r)] = v[f][t][r];
    }
  __syncthreads();
}

// conv_mid_pass for the radix lr of the last forward pass
template <int NF, int LOGE, typename T2, typename Mul>
__device__ __forceinline__ void conv_mid_dispatch(int lr, T2* sm, const int (&fb)[NF], int j, int tpf, int logH,
                                                  const T2* tw, int logP, Mul mul) {
  if (lr == LOGE) {
    conv_mid_pass<LOGE, NF, LOGE>(sm, fb, j, tpf, logH, tw, logP, mul);
  } else {
    switch (lr) {
      case 3: if constexpr (LOGE > 3) conv_mid_pass<3, NF, LOGE>(sm, fb, j, tpf, logH, tw, logP, mul); break;
      case 2: conv_mid_pass<2, NF, LOGE>(sm, fb, j, tpf, logH, tw, logP, mul); break;
      default: conv_mid_pass<1, NF, LOGE>(sm, fb, j, tpf, logH, tw, logP, mul); break;
    }
  }
}

struct Identity {
  template <typename T2>
  __device__ __forceinline__ T2 operator()(int, int, T2 v) const { return v; }
};

}  // namespace aim
