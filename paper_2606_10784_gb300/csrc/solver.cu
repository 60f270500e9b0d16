// Restarted GMRES for the AIM systems (the iterative solver of Sec. I; the Calderon system of
// Eq. 3). Arnoldi runs in FP64 on the device with classical Gram-Schmidt applied twice, the
// second pass delayed into the next step (DCGS2, below); the small Hessenberg least-squares
// problem (Givens rotations) is solved on the host, one device-to-host copy of the newly final
// Hessenberg column per iteration. Several right-hand sides run in lock step, each with its own
// Krylov basis.
//
// Mixed precision: the outer loop computes r = b - A x with the FP64 grid product, an inner
// GMRES with the FP32 grid product solves A d = r to a looser tolerance, and x += d, until
// the FP64 residual meets the target (iterative refinement).
//
// The Krylov basis is stored in double-float (hi + lo floats per real, 16 bytes per complex like
// complex128) and the Gram-Schmidt projections V^H w and updates w - V h run their products and
// per-thread sums in double-float arithmetic on the FP32 pipe, with FP64 only for the block
// reductions and the chunk sums. In binary64 they would be bound by GB300's FP64 rate (16 FP64
// operations per basis element and iteration, about 3x the time of their HBM traffic).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>

#include "aim_internal.h"
#include "dfloat.cuh"

namespace aim {

// out[j*nrhs + r] = sum_i conj(V[j][r][i]) * w[r][i]   (j < J), one block per (j, r)
__global__ void k_multidot(const double2* __restrict__ V, const double2* __restrict__ w, int n, int nrhs,
                           double2* __restrict__ out) {
  const int j = blockIdx.x, r = blockIdx.y;
  const double2* v = V + ((size_t)j * nrhs + r) * n;
  const double2* x = w + (size_t)r * n;
  double re = 0.0, im = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double2 a = v[i], b = x[i];
    re += a.x * b.x + a.y * b.y;
    im += a.x * b.y - a.y * b.x;
  }
  __shared__ double sre[32], sim[32];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    re += __shfl_xor_sync(0xffffffffu, re, off);
    im += __shfl_xor_sync(0xffffffffu, im, off);
  }
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) { sre[wid] = re; sim[wid] = im; }
  __syncthreads();
  if (wid == 0) {
    const int nw = blockDim.x >> 5;
    re = lane < nw ? sre[lane] : 0.0;
    im = lane < nw ? sim[lane] : 0.0;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      re += __shfl_xor_sync(0xffffffffu, re, off);
      im += __shfl_xor_sync(0xffffffffu, im, off);
    }
    if (lane == 0) out[(size_t)j * nrhs + r] = double2{re, im};
  }
}

// The same inner products split over chunks of kDotChunk elements, so that short Krylov bases
// still fill the GPU: part[(z J + j) nrhs + r] is the sum over chunk z; k_multidot_finish adds
// the chunks in order (deterministic).
constexpr int kDotChunk = 2048;

__global__ void k_multidot_partial(const double2* __restrict__ V, const double2* __restrict__ w, int n, int nrhs,
                                   int J, double2* __restrict__ part) {
  const int j = blockIdx.x, r = blockIdx.y, z = blockIdx.z;
  const int i0 = z * kDotChunk, i1 = min(n, i0 + kDotChunk);
  const double2* v = V + ((size_t)j * nrhs + r) * n;
  const double2* x = w + (size_t)r * n;
  double re = 0.0, im = 0.0;
  for (int i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
    const double2 a = v[i], b = x[i];
    re += a.x * b.x + a.y * b.y;
    im += a.x * b.y - a.y * b.x;
  }
  __shared__ double sre[32], sim[32];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    re += __shfl_xor_sync(0xffffffffu, re, off);
    im += __shfl_xor_sync(0xffffffffu, im, off);
  }
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) { sre[wid] = re; sim[wid] = im; }
  __syncthreads();
  if (wid == 0) {
    const int nw = blockDim.x >> 5;
    re = lane < nw ? sre[lane] : 0.0;
    im = lane < nw ? sim[lane] : 0.0;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      re += __shfl_xor_sync(0xffffffffu, re, off);
      im += __shfl_xor_sync(0xffffffffu, im, off);
    }
    if (lane == 0) part[((size_t)z * J + j) * nrhs + r] = double2{re, im};
  }
}

__global__ void k_multidot_finish(const double2* __restrict__ part, int nz, int count, double2* __restrict__ out) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= count) return;
  double re = 0.0, im = 0.0;
  for (int z = 0; z < nz; ++z) {
    const double2 p = part[(size_t)z * count + t];
    re += p.x;
    im += p.y;
  }
  out[t] = double2{re, im};
}

// Basis updates out[r][i] += sign * sum_j V[j][r][i] c[j*nrhs + r] run over chunks of kCgsChunk
// Krylov vectors: stage 1 (k_vcombine_partial_df) sums each chunk, stage 2 adds the chunk sums in
// chunk order, so the result does not depend on scheduling.
constexpr int kCgsChunk = 32;

__device__ __forceinline__ dfc to_dfc(double2 d) {
  dfc r;
  df_split(d.x, r.xh, r.xl);
  df_split(d.y, r.yh, r.yl);
  return r;
}
__device__ __forceinline__ double2 to_d2(float h_re, float l_re, float h_im, float l_im) {
  return double2{(double)h_re + (double)l_re, (double)h_im + (double)l_im};
}

__global__ void k_to_dfc(const double2* __restrict__ src, int count, dfc* __restrict__ dst) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < count) dst[t] = to_dfc(src[t]);
}

// Sum of a complex double-float value over the 32 lanes of a warp (fixed xor tree: every lane
// ends with the same, deterministic result)
__device__ __forceinline__ void warp_sum_df(float& rh, float& rl, float& ih, float& il) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const float orh = __shfl_xor_sync(0xffffffffu, rh, off), orl = __shfl_xor_sync(0xffffffffu, rl, off);
    const float oih = __shfl_xor_sync(0xffffffffu, ih, off), oil = __shfl_xor_sync(0xffffffffu, il, off);
    df_add(rh, rl, orh, orl, rh, rl);
    df_add(ih, il, oih, oil, ih, il);
  }
}

// Stage 1 of the basis update: part[chunk][r][i] = sum over the chunk of V[j][r][i] c[j*nrhs + r],
// kept in double-float (converting every chunk sum to FP64 and adding them on the FP64 pipe, at
// 1/64 of the FP32 rate here, cost more than the additions in double-float)
__global__ void k_vcombine_partial_df(const dfc* __restrict__ V, const dfc* __restrict__ c, int J, int n, int nrhs,
                                      dfc* __restrict__ part) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int chunk = blockIdx.y, r = blockIdx.z;
  if (i >= n) return;
  const int j0 = chunk * kCgsChunk, j1 = min(J, j0 + kCgsChunk);
  float rh = 0.f, rl = 0.f, ih = 0.f, il = 0.f;
  for (int j = j0; j < j1; ++j) {
    const dfc v = V[((size_t)j * nrhs + r) * n + i];
    const dfc h = c[(size_t)j * nrhs + r];
    float ph, pl;
    df_dot2<-1>(v.xh, v.xl, h.xh, h.xl, v.yh, v.yl, h.yh, h.yl, ph, pl);   // vx hx - vy hy
    df_add(rh, rl, ph, pl, rh, rl);
    df_dot2<+1>(v.xh, v.xl, h.yh, h.yl, v.yh, v.yl, h.xh, h.xl, ph, pl);   // vx hy + vy hx
    df_add(ih, il, ph, pl, ih, il);
  }
  dfc o;
  o.xh = rh;
  o.xl = rl;
  o.yh = ih;
  o.yl = il;
  part[((size_t)chunk * nrhs + r) * n + i] = o;
}

// Stage 2: out += sign * sum of the chunk partials (double-float, in chunk order, then FP64);
// out_df (may be null) receives the double-float copy of the updated out
__global__ void k_vcombine_finish_df(const dfc* __restrict__ part, int nchunks, int n, int nrhs, double sign,
                                     double2* __restrict__ out, dfc* __restrict__ out_df) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * nrhs) return;
  float rh = 0.f, rl = 0.f, ih = 0.f, il = 0.f;
  for (int ch = 0; ch < nchunks; ++ch) {
    const dfc p = part[(size_t)ch * n * nrhs + t];
    df_add(rh, rl, p.xh, p.xl, rh, rl);
    df_add(ih, il, p.yh, p.yl, ih, il);
  }
  const double2 sum = to_d2(rh, rl, ih, il);
  const double2 o = double2{out[t].x + sign * sum.x, out[t].y + sign * sum.y};
  out[t] = o;
  if (out_df != nullptr) out_df[t] = to_dfc(o);
}

// ------------------------------------------------------------------------------------
// Arnoldi with delayed reorthogonalisation (DCGS2: classical Gram-Schmidt applied twice, the
// second pass of step j-1 carried out in step j; Swirydowicz, Langou, Ananthan, Yang, Thomas,
// "Low synchronization Gram-Schmidt and GMRES algorithms", 2020; Bielich et al., "Low-synch
// Gram-Schmidt with delayed reorthogonalization for Krylov solvers", 2022).
//
// Step j starts from the orthonormal v_0..v_{j-1} and the candidate u for v_j (projected once,
// not normalised), kept in basis slot j. With w = A u, one read of the basis gives
//   s = V^H u, q = u^H u, t = V^H w, p = u^H w,
// and then (V = [v_0..v_{j-1}], H the Hessenberg matrix, <v, v_l> = 0 used throughout):
//   beta = sqrt(q - |s|^2),  v_j = (u - V s) / beta        (the delayed second pass of u)
//   H[l][j-1] += s_l, H[j][j-1] = beta                     (column j-1 is now final)
//   A v_j = (w - V (H s) - s_{j-1} (u - V s)) / beta      (A V = V H + beta v_j e_{j-1}^T)
//   c = V^H A v_j = (t - H s) / beta,  d = v_j^H A v_j = (p - s^H t) / beta^2 - s_{j-1}
//   u_{j+1} = A v_j - V c - v_j d = w / beta - kappa u - V g,
//   kappa = (s_{j-1} + d) / beta,  g = H s / beta + c - kappa s,
// so H[.][j] = (c, d) is column j's first pass, and v_j and u_{j+1} come from one more read of
// the basis. The basis is read twice per step instead of four times.
// ------------------------------------------------------------------------------------

// Offset of Hessenberg entry (l, m), l <= m + 1, in the column-packed upper Hessenberg matrix
// (column m holds rows 0..m+1), and the entries of a restart length's matrix
__host__ __device__ __forceinline__ size_t hess_index(int l, int m) { return (size_t)m * (m + 3) / 2 + l; }
__host__ __device__ __forceinline__ size_t hess_entries(int restart) { return (size_t)restart * (restart + 3) / 2; }

// part0[(z J + l) nrhs + r] = sum over chunk z of conj(V[l][r][i]) R0[r][i]; part1 likewise with
// R1 (not written when R1 is null): both projections over one read of the basis. One warp per
// (basis vector, chunk): each lane sums every 32nd element of the chunk (64 of them), then a fixed
// shuffle tree adds the lanes, so the reduction is a small part of a warp's work. A block's eight
// warps take eight consecutive basis vectors over the same chunk, so they read the same R0 and R1
// elements at about the same time and all but the first find them in L1. (One warp per block and
// eight elements per thread before a block-wide reduction ran at 2.5 TB/s of basis reads.)
constexpr int kDot2Warps = 8;

__global__ void __launch_bounds__(32 * kDot2Warps) k_multidot2_partial_df(const dfc* __restrict__ V,
                                                                          const dfc* __restrict__ R0,
                                                                          const dfc* __restrict__ R1, int n, int nrhs,
                                                                          int J, double2* __restrict__ part0,
                                                                          double2* __restrict__ part1) {
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int l = blockIdx.x * kDot2Warps + wid, r = blockIdx.y, z = blockIdx.z;
  if (l >= J) return;   // whole warps; the kernel has no block-wide barrier
  const int i0 = z * kDotChunk, i1 = min(n, i0 + kDotChunk);
  const dfc* v = V + ((size_t)l * nrhs + r) * n;
  const dfc* x0 = R0 + (size_t)r * n;
  const dfc* x1 = R1 != nullptr ? R1 + (size_t)r * n : nullptr;
  // products and sums as paired instructions on the (re, im) lanes (cconjmul, cadd)
  dfc acc0 = dfc{0.f, 0.f, 0.f, 0.f}, acc1 = dfc{0.f, 0.f, 0.f, 0.f};
  if (x1 != nullptr) {
#pragma unroll 4
    for (int i = i0 + lane; i < i1; i += 32) {
      const dfc a = v[i];
      acc0 = cadd(acc0, cconjmul(a, x0[i]));
      acc1 = cadd(acc1, cconjmul(a, x1[i]));
    }
  } else {
#pragma unroll 4
    for (int i = i0 + lane; i < i1; i += 32) acc0 = cadd(acc0, cconjmul(v[i], x0[i]));
  }
  float a_rh = acc0.xh, a_rl = acc0.xl, a_ih = acc0.yh, a_il = acc0.yl;
  warp_sum_df(a_rh, a_rl, a_ih, a_il);
  const size_t o = ((size_t)z * J + l) * nrhs + r;
  if (x1 != nullptr) {
    float b_rh = acc1.xh, b_rl = acc1.xl, b_ih = acc1.yh, b_il = acc1.yl;
    warp_sum_df(b_rh, b_rl, b_ih, b_il);
    if (lane == 0) part1[o] = to_d2(b_rh, b_rl, b_ih, b_il);
  }
  if (lane == 0) part0[o] = to_d2(a_rh, a_rl, a_ih, a_il);
}

// D0[l nrhs + r], D1[...] = chunk sums in chunk order (FP64), D0's double-float copy, and the
// delayed second pass of column j-1: H[l][j-1] += s_l = D0[l] for l < j
__global__ void k_dcgs2_finish(const double2* __restrict__ part0, const double2* __restrict__ part1, int nz, int J,
                               int nrhs, int j, int restart, double2* __restrict__ D0, double2* __restrict__ D1,
                               dfc* __restrict__ D0df, dfc* __restrict__ H) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int count = J * nrhs;
  if (t >= count) return;
  double re = 0.0, im = 0.0, re1 = 0.0, im1 = 0.0;
#pragma unroll 5
  for (int z = 0; z < nz; ++z) {
    const double2 a = part0[(size_t)z * count + t];
    re += a.x;
    im += a.y;
    if (part1 != nullptr) {
      const double2 b = part1[(size_t)z * count + t];
      re1 += b.x;
      im1 += b.y;
    }
  }
  D0[t] = double2{re, im};
  if (part1 != nullptr) D1[t] = double2{re1, im1};
  const dfc sd = to_dfc(double2{re, im});
  D0df[t] = sd;
  const int l = t / nrhs, r = t - l * nrhs;
  if (j >= 1 && l < j) {
    dfc& h = H[(size_t)r * hess_entries(restart) + hess_index(l, j - 1)];
    dfc o;
    df_add(h.xh, h.xl, sd.xh, sd.xl, o.xh, o.xl);
    df_add(h.yh, h.yl, sd.yh, sd.yl, o.yh, o.yl);
    h = o;
  }
}

__device__ __forceinline__ double2 zmul(double2 a, double2 b) { return double2{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x}; }
__device__ __forceinline__ double2 zconjmul(double2 a, double2 b) { return double2{a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x}; }

// Block sum (fixed tree) of three values over the threads of a block; every thread gets it
__device__ __forceinline__ void block_sum3(double& a, double& b, double& c, double (*sh)[3]) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, off);
    b += __shfl_xor_sync(0xffffffffu, b, off);
    c += __shfl_xor_sync(0xffffffffu, c, off);
  }
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) { sh[wid][0] = a; sh[wid][1] = b; sh[wid][2] = c; }
  __syncthreads();
  const int nw = blockDim.x >> 5;
  a = b = c = 0.0;
  for (int w = 0; w < nw; ++w) { a += sh[w][0]; b += sh[w][1]; c += sh[w][2]; }
}

// Blocks x < ceil(j/8): hs[l nrhs + r] = (H s)_l = sum_{m >= l-1} H[l][m] s_m for 8 rows l each
// (double-float; 32 slices of m per row, added in slice order). H s is small next to t (s is the
// second pass's correction), so its rounding matters less than that of t.
// Block x = ceil(j/8): the step's scalars for rhs r: beta = sqrt(q - |s|^2) (colout row j and
// H[j][j-1]), and unless final_step d = (p - s^H t)/beta^2 - s_{j-1}, kappa = (s_{j-1} + d)/beta,
// into scal = (1/beta, kappa, d).
constexpr int kHsRows = 8, kHsSlices = 32;

__global__ void __launch_bounds__(256) k_dcgs2_hs_scal(const dfc* H, const dfc* __restrict__ sdf,
                                                       const double2* __restrict__ D0, const double2* __restrict__ D1,
                                                       const int* __restrict__ active, int j, int nrhs, int restart,
                                                       int final_step, double2* __restrict__ hs,
                                                       double2* __restrict__ colout, dfc* Hw,
                                                       double2* __restrict__ scal) {
  const int r = blockIdx.y;
  const int nrow_blocks = final_step ? 0 : (j + kHsRows - 1) / kHsRows;
  const size_t hb = (size_t)r * hess_entries(restart);
  if ((int)blockIdx.x < nrow_blocks) {
    const int rl = threadIdx.x % kHsRows, sl = threadIdx.x / kHsRows;
    const int l0 = blockIdx.x * kHsRows, l = l0 + rl;
    float rh = 0.f, rlo = 0.f, ih = 0.f, il = 0.f;
#pragma unroll 4
    for (int m = max(l0 - 1, 0) + sl; m < j; m += kHsSlices) {
      if (l < j && l <= m + 1) {
        const dfc a = H[hb + hess_index(l, m)], b = sdf[(size_t)m * nrhs + r];
        float ph, pl;
        df_dot2<-1>(a.xh, a.xl, b.xh, b.xl, a.yh, a.yl, b.yh, b.yl, ph, pl);
        df_add(rh, rlo, ph, pl, rh, rlo);
        df_dot2<+1>(a.xh, a.xl, b.yh, b.yl, a.yh, a.yl, b.xh, b.xl, ph, pl);
        df_add(ih, il, ph, pl, ih, il);
      }
    }
    __shared__ float part[kHsSlices][kHsRows][4];
    part[sl][rl][0] = rh;
    part[sl][rl][1] = rlo;
    part[sl][rl][2] = ih;
    part[sl][rl][3] = il;
    __syncthreads();
    if (sl == 0 && l < j) {
      for (int k = 1; k < kHsSlices; ++k) {
        df_add(rh, rlo, part[k][rl][0], part[k][rl][1], rh, rlo);
        df_add(ih, il, part[k][rl][2], part[k][rl][3], ih, il);
      }
      hs[(size_t)l * nrhs + r] = to_d2(rh, rlo, ih, il);
    }
    return;
  }
  __shared__ double sh[32][3];
  double ss = 0.0, st_re = 0.0, st_im = 0.0;
  for (int l = threadIdx.x; l < j; l += blockDim.x) {
    const double2 sv = D0[(size_t)l * nrhs + r];
    ss += sv.x * sv.x + sv.y * sv.y;
    if (!final_step) {
      const double2 c = zconjmul(sv, D1[(size_t)l * nrhs + r]);
      st_re += c.x;
      st_im += c.y;
    }
  }
  block_sum3(ss, st_re, st_im, sh);
  if (threadIdx.x != 0) return;
  const double q = D0[(size_t)j * nrhs + r].x;
  const double b2 = q - ss;
  // a non-finite value reaches the host through beta (the norm it checks); b2 <= 0 is a breakdown
  const double beta = !active[r] ? 0.0 : !isfinite(b2) ? b2 : b2 > 0.0 ? sqrt(b2) : 0.0;
  const double ib = beta > 0.0 ? 1.0 / beta : 0.0;
  if (j >= 1) {
    colout[(size_t)j * nrhs + r] = double2{beta, 0.0};
    Hw[hb + hess_index(j, j - 1)] = to_dfc(double2{beta, 0.0});
  }
  if (final_step) return;
  const double2 p = D1[(size_t)j * nrhs + r];
  const double2 slast = j >= 1 ? D0[(size_t)(j - 1) * nrhs + r] : double2{0.0, 0.0};
  double2 d = double2{(p.x - st_re) * ib * ib - slast.x, (p.y - st_im) * ib * ib - slast.y};
  if (beta == 0.0) d = double2{0.0, 0.0};
  const double2 kappa = double2{(slast.x + d.x) * ib, (slast.y + d.y) * ib};
  scal[r] = double2{ib, 0.0};
  scal[nrhs + r] = kappa;
  scal[2 * nrhs + r] = d;
  Hw[hb + hess_index(j, j)] = to_dfc(d);
}

// Per entry l < j of rhs r (t = l nrhs + r): the final column j-1 for the host (colout, from H
// after the delayed pass), and unless final_step c_l = (t_l - (H s)_l)/beta into H[l][j],
// g_l = (H s)_l / beta + c_l - kappa s_l and a1_l = s_l / beta (double-float, for the updates)
__global__ void k_dcgs2_coeffs(const double2* __restrict__ D0, const double2* __restrict__ D1,
                               const double2* __restrict__ hs, const double2* __restrict__ scal, int j, int nrhs,
                               int restart, int final_step, dfc* __restrict__ H, double2* __restrict__ colout,
                               dfc* __restrict__ a1, dfc* __restrict__ g) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= j * nrhs) return;
  const int l = t / nrhs, r = t - l * nrhs;
  const size_t hb = (size_t)r * hess_entries(restart);
  if (j >= 1) {
    const dfc h = H[hb + hess_index(l, j - 1)];
    colout[t] = to_d2(h.xh, h.xl, h.yh, h.yl);
  }
  if (final_step) return;
  const double ib = scal[r].x;
  const double2 kappa = scal[nrhs + r];
  const double2 sv = D0[t], tv = D1[t], hv = hs[t];
  const double2 c = double2{(tv.x - hv.x) * ib, (tv.y - hv.y) * ib};
  const double2 ks = zmul(kappa, sv);
  g[t] = to_dfc(double2{hv.x * ib + c.x - ks.x, hv.y * ib + c.y - ks.y});
  a1[t] = to_dfc(double2{sv.x * ib, sv.y * ib});
  H[hb + hess_index(l, j)] = to_dfc(c);
}

// Stage 1 of the two updates of a step, over one read of the basis: part1[chunk][r][i] =
// sum over the chunk of V[l][r][i] a1[l], part2 the same with g
__global__ void k_vcombine2_partial_df(const dfc* __restrict__ V, const dfc* __restrict__ a1, const dfc* __restrict__ g,
                                       int J, int n, int nrhs, dfc* __restrict__ part1, dfc* __restrict__ part2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int chunk = blockIdx.y, r = blockIdx.z;
  if (i >= n) return;
  const int j0 = chunk * kCgsChunk, j1 = min(J, j0 + kCgsChunk);
  // products and sums as paired instructions on the (re, im) lanes (cmul, cadd)
  dfc acc1 = dfc{0.f, 0.f, 0.f, 0.f}, acc2 = dfc{0.f, 0.f, 0.f, 0.f};
#pragma unroll 4
  for (int l = j0; l < j1; ++l) {
    const dfc v = V[((size_t)l * nrhs + r) * n + i];
    acc1 = cadd(acc1, cmul(v, a1[(size_t)l * nrhs + r]));
    acc2 = cadd(acc2, cmul(v, g[(size_t)l * nrhs + r]));
  }
  const size_t o = ((size_t)chunk * nrhs + r) * n + i;
  part1[o] = acc1;
  part2[o] = acc2;
}

// Stage 2: v_j = u / beta - V a1 into slot j (u is read there first), u_{j+1} = w / beta - kappa u -
// V g into slot j+1 and, in binary64, into cur (the next product's input). Eight adjacent threads
// per element sum every eighth chunk; a fixed shuffle tree adds their sums.
constexpr int kFinishLanes = 8;

__global__ void k_vcombine2_finish_df(const dfc* __restrict__ part1, const dfc* __restrict__ part2, int nchunks, int n,
                                      int nrhs, const double2* __restrict__ scal, dfc* __restrict__ Vj,
                                      const double2* __restrict__ w, dfc* __restrict__ Vnext, double2* __restrict__ cur) {
  const long long gt = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int t = (int)(gt / kFinishLanes), q = (int)(gt % kFinishLanes);
  const bool live = t < n * nrhs;   // whole groups of four: the shuffles below need every lane
  float a_rh = 0.f, a_rl = 0.f, a_ih = 0.f, a_il = 0.f;
  float b_rh = 0.f, b_rl = 0.f, b_ih = 0.f, b_il = 0.f;
  if (live) {
#pragma unroll 2
    for (int ch = q; ch < nchunks; ch += kFinishLanes) {
      const dfc p = part1[(size_t)ch * n * nrhs + t], pp = part2[(size_t)ch * n * nrhs + t];
      df_add(a_rh, a_rl, p.xh, p.xl, a_rh, a_rl);
      df_add(a_ih, a_il, p.yh, p.yl, a_ih, a_il);
      df_add(b_rh, b_rl, pp.xh, pp.xl, b_rh, b_rl);
      df_add(b_ih, b_il, pp.yh, pp.yl, b_ih, b_il);
    }
  }
#pragma unroll
  for (int off = 1; off < kFinishLanes; off <<= 1) {
    const float o0 = __shfl_xor_sync(0xffffffffu, a_rh, off), o1 = __shfl_xor_sync(0xffffffffu, a_rl, off);
    const float o2 = __shfl_xor_sync(0xffffffffu, a_ih, off), o3 = __shfl_xor_sync(0xffffffffu, a_il, off);
    const float o4 = __shfl_xor_sync(0xffffffffu, b_rh, off), o5 = __shfl_xor_sync(0xffffffffu, b_rl, off);
    const float o6 = __shfl_xor_sync(0xffffffffu, b_ih, off), o7 = __shfl_xor_sync(0xffffffffu, b_il, off);
    df_add(a_rh, a_rl, o0, o1, a_rh, a_rl);
    df_add(a_ih, a_il, o2, o3, a_ih, a_il);
    df_add(b_rh, b_rl, o4, o5, b_rh, b_rl);
    df_add(b_ih, b_il, o6, o7, b_ih, b_il);
  }
  if (!live || q != 0) return;
  const int r = t / n;
  const double2 P1 = to_d2(a_rh, a_rl, a_ih, a_il), P2 = to_d2(b_rh, b_rl, b_ih, b_il);
  const double ib = scal[r].x;
  const double2 kappa = scal[nrhs + r];
  const dfc ud = Vj[t];
  const double2 u = to_d2(ud.xh, ud.xl, ud.yh, ud.yl);
  const double2 wv = w[t];
  const double2 vj = double2{u.x * ib - P1.x, u.y * ib - P1.y};
  const double2 ku = zmul(kappa, u);
  const double2 un = double2{wv.x * ib - ku.x - P2.x, wv.y * ib - ku.y - P2.y};
  Vj[t] = to_dfc(vj);
  Vnext[t] = to_dfc(un);
  cur[t] = un;
}

// v = w[r] / sqrt(nrm2[r].x) (zero if the norm vanished, or active[r] == 0): the new basis
// vector in double-float (dst) and in binary64 (cur, the next matrix-vector product's input)
__global__ void k_normalize(const double2* __restrict__ w, const double2* __restrict__ nrm2, const int* __restrict__ active,
                            int n, int nrhs, dfc* __restrict__ dst, double2* __restrict__ cur) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * nrhs) return;
  const int r = t / n;
  const double nv = sqrt(fmax(nrm2[r].x, 0.0));
  const double s = (active[r] && nv > 0.0) ? 1.0 / nv : 0.0;
  const double2 v = double2{w[t].x * s, w[t].y * s};
  cur[t] = v;
  dst[t] = to_dfc(v);
}

// r = b - Ax
__global__ void k_residual(const double2* __restrict__ b, const double2* __restrict__ Ax, int total, double2* __restrict__ r) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < total) r[t] = double2{b[t].x - Ax[t].x, b[t].y - Ax[t].y};
}

__global__ void k_add_vec(double2* __restrict__ x, const double2* __restrict__ d, int total) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < total) { x[t].x += d[t].x; x[t].y += d[t].y; }
}

namespace {

struct Zc {
  double re, im;
};
inline Zc cm(Zc a, Zc b) { return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }
inline Zc cconj(Zc a) { return {a.re, -a.im}; }
inline double cabs2(Zc a) { return a.re * a.re + a.im * a.im; }

struct Workspace {
  dfc* V;                      // basis, double-float
  double2 *w, *r, *cur, *tmp, *dots, *dots2, *nrm;
  dfc *wdf, *dots_df, *dots2_df;
  int* active;
  // delayed reorthogonalisation: Hessenberg matrix (row-packed, per rhs), H s, the final column
  // staged for the host, the update coefficients and the two scalars (1/beta, kappa) per rhs
  dfc* H;
  double2 *hs, *colout, *scal;
  dfc* g;
};

inline int blocks_for(long long total, int tpb) { return (int)((total + tpb - 1) / tpb); }

// two timing-free events, destroyed with the scope
struct EventPair {
  cudaEvent_t e[2] = {nullptr, nullptr};
  aim_status create() {
    for (auto& ev : e) AIM_CUDA_TRY(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    return AIM_OK;
  }
  ~EventPair() {
    for (auto& ev : e)
      if (ev) cudaEventDestroy(ev);
  }
};

// out[j*nrhs + r] = <V[j][r], w[r]> for j < J (two launches); part holds ceil(n/kDotChunk)*J*nrhs values
aim_status multidot(const double2* V, const double2* w, int J, int n, int nrhs, double2* out, double2* part,
                    cudaStream_t st) {
  const int nz = (n + kDotChunk - 1) / kDotChunk;
  count_launches(K_GMRES, 2);
  k_multidot_partial<<<dim3(J, nrhs, nz), 256, 0, st>>>(V, w, n, nrhs, J, part);
  k_multidot_finish<<<blocks_for((long long)J * nrhs, 256), 256, 0, st>>>(part, nz, J * nrhs, out);
  AIM_CUDA_TRY(cudaGetLastError());
  return AIM_OK;
}

aim_status dot_norms(const double2* vecs, int n, int nrhs, double2* out, double2* part, cudaStream_t st) {
  return multidot(vecs, vecs, 1, n, nrhs, out, part, st);
}

}  // namespace

// The solver's operator products: through the calling thread's batcher when aim_solve_batched
// attached one (the product then joins other solves' products in a multi-context launch), else
// directly.
static aim_status solver_apply(aim_ctx* ctx, aim_op op, int nrhs, const double2* x, double2* y, int precision,
                               cudaStream_t st) {
  if (aim_batcher* b = current_batcher()) return batcher_product(b, ctx, op, nrhs, x, y, precision, st);
  return apply_op(ctx, op, nrhs, x, y, precision, st);
}

// The operator product of an Arnoldi step always reads the current vector and writes w, so it is
// captured once as a CUDA graph and replayed each iteration: one host call instead of ~10 kernel
// launches, which is what limits small problems. Not while kernels are being timed (a replay
// would not record their events); if capture fails for any reason the step launches directly.
struct OpGraph {
  cudaGraphExec_t exec = nullptr;
  bool tried = false;
  long long counts[K_COUNT] = {};   // launches one replay stands for, per kernel id
  void capture(aim_ctx* ctx, aim_op op, int nrhs, const double2* x, double2* y, int precision, cudaStream_t st) {
    tried = true;
    if (profiling_active() || current_batcher() != nullptr) return;   // batched products are not captured
    long long before[K_COUNT], after[K_COUNT];
    thread_launch_counts(before);
    if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      cudaGetLastError();
      return;
    }
    const aim_status s = apply_op(ctx, op, nrhs, x, y, precision, st);
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(st, &g);
    thread_launch_counts(after);
    for (int i = 0; i < K_COUNT; ++i) {
      counts[i] = after[i] - before[i];
      if (counts[i]) count_launches(i, (int)-counts[i]);   // a capture runs nothing
    }
    if (s == AIM_OK && e == cudaSuccess && g != nullptr && cudaGraphInstantiate(&exec, g, 0) != cudaSuccess)
      exec = nullptr;
    if (g != nullptr) cudaGraphDestroy(g);
    cudaGetLastError();
  }
  aim_status replay(cudaStream_t st) {
    AIM_CUDA_TRY(cudaGraphLaunch(exec, st));
    for (int i = 0; i < K_COUNT; ++i)
      if (counts[i]) count_launches(i, (int)counts[i]);
    return AIM_OK;
  }
  ~OpGraph() {
    if (exec != nullptr) cudaGraphExecDestroy(exec);
  }
};

// out += sign * V c over J vectors of the double-float basis (two launches, deterministic order)
static void vcombine_df(const dfc* V, const dfc* c, int J, int n, int nrhs, double sign, double2* out, dfc* out_df,
                        double2* part, cudaStream_t st) {
  const int nch = (J + kCgsChunk - 1) / kCgsChunk;
  count_launches(K_GMRES, 2);
  dfc* part_df = reinterpret_cast<dfc*>(part);   // same 16-byte elements
  k_vcombine_partial_df<<<dim3((n + 255) / 256, nch, nrhs), 256, 0, st>>>(V, c, J, n, nrhs, part_df);
  k_vcombine_finish_df<<<(n * nrhs + 255) / 256, 256, 0, st>>>(part_df, nch, n, nrhs, sign, out, out_df);
}

size_t krylov_bytes(size_t n, int nrhs, int restart) {
  // partial sums of the two basis updates of a step (chunks of kCgsChunk vectors) or of its two
  // sets of inner products (chunks of kDotChunk elements), whichever needs more
  const size_t nz = (n + kDotChunk - 1) / kDotChunk;
  const size_t part_vecs =
      std::max(2 * ((size_t)(restart + kCgsChunk) / kCgsChunk), (2 * nz * (restart + 1) + n - 1) / n);
  // basis (restart + 1, double-float), w, r, the current vector, w in double-float, partial sums
  const size_t nvec = (size_t)(restart + 1) + 4 + part_vecs;
  // and the Hessenberg matrix of each right-hand side (double-float, row-packed)
  return nvec * nrhs * n * sizeof(double2) + (size_t)nrhs * hess_entries(restart) * sizeof(dfc);
}

size_t reduction_bytes(int nrhs, int restart) {
  // dots, dots2, norms, double-float copies, H s, the staged column, g, the step scalars, and
  // the active flags
  return ((size_t)(restart + 2) * 8 + 3) * nrhs * sizeof(double2) + nrhs * sizeof(int);
}

static aim_status ensure_krylov(aim_ctx* ctx, int nrhs, int restart) {
  const size_t need = krylov_bytes((size_t)ctx->n, nrhs, restart);
  if (ctx->kry_bytes < need) {
    if (ctx->kry) cudaFree(ctx->kry);
    ctx->kry = nullptr;
    ctx->kry_bytes = 0;
    void* p = nullptr;
    AIM_CUDA_TRY(cudaMalloc(&p, need));
    ctx->kry = static_cast<double2*>(p);
    ctx->kry_bytes = need;
  }
  const size_t rneed = reduction_bytes(nrhs, restart);
  if (ctx->red_bytes < rneed) {
    if (ctx->red) cudaFree(ctx->red);
    if (ctx->red_host) cudaFreeHost(ctx->red_host);
    ctx->red = nullptr;
    ctx->red_host = nullptr;
    ctx->red_bytes = 0;
    void* p = nullptr;
    AIM_CUDA_TRY(cudaMalloc(&p, rneed));
    ctx->red = static_cast<double*>(p);
    AIM_CUDA_TRY(cudaMallocHost(&p, rneed));
    ctx->red_host = static_cast<double*>(p);
    ctx->red_bytes = rneed;
  }
  return AIM_OK;
}

// Core restarted GMRES on A (op, precision) for b -> x, all right-hand sides in lock step.
// tol: relative to ||b_r||. Updates per-rhs iteration counters and convergence flags.
// single_cycle: stop after one Krylov cycle (at most `restart` iterations, ended by the Arnoldi
// residual estimate) without the true-residual check. The inner solves of the mixed-precision
// refinement use it: the true residual under the complex64 operator cannot fall below that
// operator's own noise, so a restart decided on it would stall; the outer FP64 residual decides.
static aim_status gmres_core(aim_ctx* ctx, aim_op op, int precision, int nrhs, const double2* b, double2* x,
                             double tol, int restart, int max_iter, std::vector<int>* iters,
                             std::vector<double>* relres, std::vector<int>* conv,
                             std::chrono::steady_clock::time_point deadline, bool has_deadline,
                             cudaStream_t st, bool single_cycle = false) {
  const int n = ctx->n;
  const size_t vsz = (size_t)nrhs * n;
  AIM_TRY(ensure_krylov(ctx, nrhs, restart));
  static_assert(sizeof(dfc) == sizeof(double2), "double-float complex must be 16 bytes");
  Workspace ws;
  ws.V = reinterpret_cast<dfc*>(ctx->kry);
  ws.w = ctx->kry + (size_t)(restart + 1) * vsz;
  ws.r = ws.w + vsz;
  ws.cur = ws.r + vsz;
  ws.wdf = reinterpret_cast<dfc*>(ws.cur + vsz);
  ws.tmp = ws.cur + 2 * vsz;
  double2* red = reinterpret_cast<double2*>(ctx->red);
  ws.dots = red;                                   // (restart+1) * nrhs
  ws.dots2 = red + (size_t)(restart + 2) * nrhs;   // (restart+1) * nrhs
  ws.nrm = red + (size_t)(restart + 2) * 2 * nrhs; // nrhs
  ws.dots_df = reinterpret_cast<dfc*>(red + (size_t)(restart + 2) * 3 * nrhs);   // (restart+1) * nrhs
  ws.dots2_df = reinterpret_cast<dfc*>(red + (size_t)(restart + 2) * 4 * nrhs);  // (restart+1) * nrhs
  ws.hs = red + (size_t)(restart + 2) * 5 * nrhs;                                  // (restart+1) * nrhs
  ws.colout = red + (size_t)(restart + 2) * 6 * nrhs;                              // (restart+2) * nrhs
  ws.g = reinterpret_cast<dfc*>(red + (size_t)(restart + 2) * 7 * nrhs);           // (restart+1) * nrhs
  ws.scal = red + (size_t)(restart + 2) * 8 * nrhs;                                // 2 * nrhs
  ws.active = reinterpret_cast<int*>(red + ((size_t)(restart + 2) * 8 + 3) * nrhs);
  {
    const size_t nz = ((size_t)n + kDotChunk - 1) / kDotChunk;
    const size_t part_vecs =
        std::max(2 * ((size_t)(restart + kCgsChunk) / kCgsChunk), (2 * nz * (restart + 1) + n - 1) / n);
    ws.H = reinterpret_cast<dfc*>(ws.tmp + part_vecs * vsz);
  }
  double2* hred = reinterpret_cast<double2*>(ctx->red_host);
  const int tpb = 256;
  const int nb = blocks_for((long long)vsz, tpb);

  // ||b||
  AIM_TRY(dot_norms(b, n, nrhs, ws.nrm, ws.tmp, st));
  AIM_CUDA_TRY(cudaMemcpyAsync(hred, ws.nrm, nrhs * sizeof(double2), cudaMemcpyDeviceToHost, st));
  AIM_CUDA_TRY(cudaStreamSynchronize(st));
  std::vector<double> bnorm(nrhs);
  for (int r = 0; r < nrhs; ++r) {
    bnorm[r] = std::sqrt(hred[r].x);
    if (!std::isfinite(bnorm[r])) return fail(AIM_ENUMERIC, "non-finite right-hand side");
  }

  std::vector<int> active(nrhs, 1);
  // Hessenberg columns as they are produced: column j holds rows 0..j+1 for every rhs
  std::vector<std::vector<Zc>> Hcol;
  Hcol.reserve(restart);
  std::vector<Zc> cs((size_t)restart * nrhs), sn((size_t)restart * nrhs), g((size_t)(restart + 1) * nrhs),
      yv((size_t)restart * nrhs);
  std::vector<double> beta(nrhs);
  std::vector<int> jconv(nrhs);
  EventPair col_ready;
  AIM_TRY(col_ready.create());
  OpGraph op_graph;

  while (true) {
    // true residual r = b - A x
    AIM_TRY(solver_apply(ctx, op, nrhs, x, ws.w, precision, st));
    count_launches(K_GMRES, 1);
    k_residual<<<nb, tpb, 0, st>>>(b, ws.w, (int)vsz, ws.r);
    AIM_CUDA_TRY(cudaGetLastError());
    AIM_TRY(dot_norms(ws.r, n, nrhs, ws.nrm, ws.tmp, st));
    AIM_CUDA_TRY(cudaMemcpyAsync(hred, ws.nrm, nrhs * sizeof(double2), cudaMemcpyDeviceToHost, st));
    AIM_CUDA_TRY(cudaStreamSynchronize(st));
    bool any = false;
    for (int r = 0; r < nrhs; ++r) {
      beta[r] = std::sqrt(hred[r].x);
      if (!std::isfinite(beta[r])) return fail(AIM_ENUMERIC, "non-finite residual");
      const double rel = bnorm[r] > 0 ? beta[r] / bnorm[r] : 0.0;
      (*relres)[r] = rel;
      if (rel <= tol || bnorm[r] == 0.0) { active[r] = 0; (*conv)[r] = 1; }
      else if ((*iters)[r] >= max_iter) active[r] = 0;
      else active[r] = 1;
      any = any || active[r];
    }
    if (!any) break;
    if (has_deadline && std::chrono::steady_clock::now() > deadline) return fail(AIM_ETIMEOUT, "solve time limit reached");

    AIM_CUDA_TRY(cudaMemcpyAsync(ws.active, active.data(), nrhs * sizeof(int), cudaMemcpyHostToDevice, st));
    count_launches(K_GMRES, 1);
    k_normalize<<<nb, tpb, 0, st>>>(ws.r, ws.nrm, ws.active, n, nrhs, ws.V, ws.cur);
    AIM_CUDA_TRY(cudaGetLastError());
    for (int r = 0; r < nrhs; ++r) {
      g[(size_t)0 * nrhs + r] = {beta[r], 0.0};
      for (int j = 1; j <= restart; ++j) g[(size_t)j * nrhs + r] = {0.0, 0.0};
      jconv[r] = 0;
    }
    // Arnoldi step j (delayed reorthogonalisation, see the kernels above): w = A u_j, both sets of
    // projections over one read of the basis, the coefficients, and v_j and u_{j+1} from one more
    // read; step j (j >= 1) finalises Hessenberg column j - 1 and copies it to host slot
    // (j - 1) % 2. Step `restart` only finalises the last column (no product). A step needs
    // nothing from the host, so steps c + 1 and c + 2 are queued before the host waits for column
    // c: the Givens updates overlap the device work, and at most two queued steps are discarded
    // when a cycle ends early (they write only basis slots and columns past the ones in use).
    auto arnoldi_step = [&](int j) -> aim_status {
      const bool final_step = j == restart;
      dfc* Vj = ws.V + (size_t)j * vsz;
      if (!final_step) {
        // w = A u_j (cur = u_j)
        if (!op_graph.tried) op_graph.capture(ctx, op, nrhs, ws.cur, ws.w, precision, st);
        if (op_graph.exec != nullptr) {
          AIM_TRY(op_graph.replay(st));
        } else {
          AIM_TRY(solver_apply(ctx, op, nrhs, ws.cur, ws.w, precision, st));
        }
      }
      // 7 launches (4 in the final step), timed as one group when profiling
      ProfScope group(K_GMRES, st, /*count_launch=*/false);
      const int J = j + 1;   // v_0..v_{j-1} and the candidate u_j in slot j
      const int nz = (n + kDotChunk - 1) / kDotChunk;
      double2* part0 = ws.tmp;
      double2* part1 = ws.tmp + (size_t)nz * J * nrhs;
      if (!final_step) {
        count_launches(K_GMRES, 1);
        k_to_dfc<<<nb, tpb, 0, st>>>(ws.w, (int)vsz, ws.wdf);
      }
      count_launches(K_GMRES, 3);
      k_multidot2_partial_df<<<dim3((J + kDot2Warps - 1) / kDot2Warps, nrhs, nz), 32 * kDot2Warps, 0, st>>>(
          ws.V, Vj, final_step ? nullptr : ws.wdf, n, nrhs, J, part0, final_step ? nullptr : part1);
      k_dcgs2_finish<<<blocks_for((long long)J * nrhs, tpb), tpb, 0, st>>>(part0, final_step ? nullptr : part1, nz, J,
                                                                          nrhs, j, restart, ws.dots, ws.dots2,
                                                                          ws.dots_df, ws.H);
      const int hs_blocks = final_step ? 0 : (j + kHsRows - 1) / kHsRows;
      k_dcgs2_hs_scal<<<dim3(hs_blocks + 1, nrhs), 256, 0, st>>>(ws.H, ws.dots_df, ws.dots, ws.dots2, ws.active, j, nrhs,
                                                                 restart, final_step ? 1 : 0, ws.hs, ws.colout, ws.H,
                                                                 ws.scal);
      if (j >= 1) {
        count_launches(K_GMRES, 1);
        k_dcgs2_coeffs<<<blocks_for((long long)j * nrhs, tpb), tpb, 0, st>>>(ws.dots, ws.dots2, ws.hs, ws.scal, j, nrhs,
                                                                             restart, final_step ? 1 : 0, ws.H,
                                                                             ws.colout, ws.dots2_df, ws.g);
      }
      if (!final_step) {
        const int nch = (j + kCgsChunk - 1) / kCgsChunk;
        dfc* p1 = reinterpret_cast<dfc*>(ws.tmp);
        dfc* p2 = p1 + (size_t)nch * vsz;
        if (nch > 0) {
          count_launches(K_GMRES, 1);
          k_vcombine2_partial_df<<<dim3((n + 255) / 256, nch, nrhs), 256, 0, st>>>(ws.V, ws.dots2_df, ws.g, j, n, nrhs,
                                                                                   p1, p2);
        }
        count_launches(K_GMRES, 1);
        k_vcombine2_finish_df<<<blocks_for((long long)vsz * kFinishLanes, tpb), tpb, 0, st>>>(p1, p2, nch, n, nrhs, ws.scal,
                                                                                             Vj, ws.w, Vj + vsz, ws.cur);
      }
      AIM_CUDA_TRY(cudaGetLastError());
      if (j >= 1) {
        double2* slot = hred + (size_t)((j - 1) & 1) * (restart + 2) * nrhs;
        AIM_CUDA_TRY(cudaMemcpyAsync(slot, ws.colout, (size_t)(j + 1) * nrhs * sizeof(double2), cudaMemcpyDeviceToHost, st));
        AIM_CUDA_TRY(cudaEventRecord(col_ready.e[(j - 1) & 1], st));
      }
      return AIM_OK;
    };
    int jdone = 0;
    AIM_TRY(arnoldi_step(0));
    AIM_TRY(arnoldi_step(1));
    for (int j = 0; j < restart; ++j) {
      // column j is finalised by step j + 1, already queued
      if (j + 2 <= restart) AIM_TRY(arnoldi_step(j + 2));
      AIM_CUDA_TRY(cudaEventSynchronize(col_ready.e[j & 1]));
      const double2* hcol = hred + (size_t)(j & 1) * (restart + 2) * nrhs;
      jdone = j + 1;
      bool all_done = true;
      if ((int)Hcol.size() <= j) Hcol.resize(j + 1);
      Hcol[j].assign((size_t)(j + 2) * nrhs, Zc{0.0, 0.0});
      Zc* col = Hcol[j].data();   // column j, rows 0..j+1
      for (int r = 0; r < nrhs; ++r) {
        if (!active[r] || jconv[r]) continue;
        for (int i = 0; i <= j; ++i) {
          const double2 h = hcol[(size_t)i * nrhs + r];
          if (!std::isfinite(h.x) || !std::isfinite(h.y)) return fail(AIM_ENUMERIC, "non-finite Hessenberg entry");
          col[(size_t)i * nrhs + r] = {h.x, h.y};
        }
        const double hn = hcol[(size_t)(j + 1) * nrhs + r].x;
        if (!std::isfinite(hn)) return fail(AIM_ENUMERIC, "non-finite Arnoldi norm");
        col[(size_t)(j + 1) * nrhs + r] = {hn, 0.0};
        for (int i = 0; i < j; ++i) {
          const Zc c = cs[(size_t)i * nrhs + r], s = sn[(size_t)i * nrhs + r];
          const Zc a = col[(size_t)i * nrhs + r], bb = col[(size_t)(i + 1) * nrhs + r];
          const Zc t1 = cm(c, a), t2 = cm(s, bb);
          const Zc t3 = cm(cconj(s), a), t4 = cm(cconj(c), bb);
          col[(size_t)i * nrhs + r] = {t1.re + t2.re, t1.im + t2.im};
          col[(size_t)(i + 1) * nrhs + r] = {-t3.re + t4.re, -t3.im + t4.im};
        }
        const Zc a = col[(size_t)j * nrhs + r], bb = col[(size_t)(j + 1) * nrhs + r];
        const double den = std::sqrt(cabs2(a) + cabs2(bb));
        Zc c{1.0, 0.0}, s{0.0, 0.0};
        if (den > 0.0) {
          c = {a.re / den, -a.im / den};
          s = {bb.re / den, -bb.im / den};
        }
        cs[(size_t)j * nrhs + r] = c;
        sn[(size_t)j * nrhs + r] = s;
        col[(size_t)j * nrhs + r] = {den, 0.0};
        col[(size_t)(j + 1) * nrhs + r] = {0.0, 0.0};
        const Zc gj = g[(size_t)j * nrhs + r];
        const Zc ng = cm(cconj(s), gj);
        g[(size_t)(j + 1) * nrhs + r] = {-ng.re, -ng.im};
        g[(size_t)j * nrhs + r] = cm(c, gj);
        (*iters)[r] += 1;
        const double est = std::sqrt(cabs2(g[(size_t)(j + 1) * nrhs + r])) / bnorm[r];
        if (est <= tol || (*iters)[r] >= max_iter || hn == 0.0) jconv[r] = j + 1;
        if (!jconv[r]) all_done = false;
      }
      if (all_done) break;
      if (has_deadline && std::chrono::steady_clock::now() > deadline) return fail(AIM_ETIMEOUT, "solve time limit reached");
    }
    // back substitution per rhs, using its own Krylov length
    std::fill(yv.begin(), yv.end(), Zc{0.0, 0.0});
    for (int r = 0; r < nrhs; ++r) {
      if (!active[r]) continue;
      const int J = jconv[r] ? jconv[r] : jdone;
      for (int i = J - 1; i >= 0; --i) {
        Zc acc = g[(size_t)i * nrhs + r];
        for (int l = i + 1; l < J; ++l) {
          const Zc t = cm(Hcol[l][(size_t)i * nrhs + r], yv[(size_t)l * nrhs + r]);
          acc.re -= t.re;
          acc.im -= t.im;
        }
        const Zc d = Hcol[i][(size_t)i * nrhs + r];
        const double dd = cabs2(d);
        yv[(size_t)i * nrhs + r] = dd > 0 ? Zc{(acc.re * d.re + acc.im * d.im) / dd, (acc.im * d.re - acc.re * d.im) / dd}
                                          : Zc{0.0, 0.0};
      }
    }
    AIM_CUDA_TRY(cudaMemcpyAsync(ws.dots, yv.data(), (size_t)jdone * nrhs * sizeof(double2), cudaMemcpyHostToDevice, st));
    count_launches(K_GMRES, 1);
    k_to_dfc<<<blocks_for((long long)jdone * nrhs, tpb), tpb, 0, st>>>(ws.dots, jdone * nrhs, ws.dots_df);
    vcombine_df(ws.V, ws.dots_df, jdone, n, nrhs, 1.0, x, nullptr, ws.tmp, st);
    AIM_CUDA_TRY(cudaGetLastError());
    if (single_cycle) break;
  }
  return AIM_OK;
}

aim_status gmres_solve(aim_ctx* ctx, aim_op system, int nrhs, const double2* b, double2* x,
                       const aim_solve_opts* opts, aim_solve_info* info, cudaStream_t st) {
  const int n = ctx->n;
  const size_t vsz = (size_t)nrhs * n;
  const bool has_deadline = opts->timeout_ms > 0;
  const auto deadline = std::chrono::steady_clock::now() + std::chrono::milliseconds(has_deadline ? opts->timeout_ms : 0);
  std::vector<int> iters(nrhs, 0), conv(nrhs, 0), outer(nrhs, 0);
  std::vector<double> relres(nrhs, 1.0);
  aim_status st_out = AIM_OK;
  if (opts->precision != AIM_MIXED) {
    aim_status s = gmres_core(ctx, system, opts->precision, nrhs, b, x, opts->tol, opts->restart, opts->max_iter, &iters,
                              &relres, &conv, deadline, has_deadline, st);
    if (s != AIM_OK) return s;
    for (int r = 0; r < nrhs; ++r) outer[r] = 1;
  } else {
    // iterative refinement: FP64 residual outside, FP32 grid product inside
    AIM_TRY(reserve(ctx, nrhs, AIM_FP64));
    AIM_TRY(reserve(ctx, nrhs, AIM_MIXED));
    // the residual and the correction of the refinement: a stream-ordered temporary
    double2* rr = nullptr;
    double2* dd = nullptr;
    AIM_CUDA_TRY(cudaMallocAsync(reinterpret_cast<void**>(&rr), 2 * vsz * sizeof(double2), st));
    dd = rr + vsz;
    std::vector<double> bn(nrhs);
    aim_status s = AIM_OK;
    for (int outer_it = 0; outer_it < 60; ++outer_it) {
      // r = b - A x (FP64)
      s = solver_apply(ctx, system, nrhs, x, rr, AIM_FP64, st);
      if (s != AIM_OK) break;
      count_launches(K_GMRES, 3);
      k_residual<<<blocks_for((long long)vsz, 256), 256, 0, st>>>(b, rr, (int)vsz, rr);
      // norms of r and b
      std::vector<int> it_inner(nrhs, 0), conv_inner(nrhs, 0);
      std::vector<double> rel_inner(nrhs, 1.0);
      double2* nrm = reinterpret_cast<double2*>(ctx->red);
      s = ensure_krylov(ctx, nrhs, opts->restart);
      if (s != AIM_OK) break;
      nrm = reinterpret_cast<double2*>(ctx->red);
      double2* hred = reinterpret_cast<double2*>(ctx->red_host);
      k_multidot<<<dim3(1, nrhs), 256, 0, st>>>(rr, rr, n, nrhs, nrm);
      k_multidot<<<dim3(1, nrhs), 256, 0, st>>>(b, b, n, nrhs, nrm + nrhs);
      cudaMemcpyAsync(hred, nrm, 2 * nrhs * sizeof(double2), cudaMemcpyDeviceToHost, st);
      if (cudaStreamSynchronize(st) != cudaSuccess) { s = fail(AIM_ECUDA, "stream sync failed"); break; }
      bool all = true;
      double worst = 0.0;   // largest relative residual among the right-hand sides still running
      for (int r = 0; r < nrhs; ++r) {
        const double rn = std::sqrt(hred[r].x), bnr = std::sqrt(hred[nrhs + r].x);
        if (!std::isfinite(rn) || !std::isfinite(bnr)) { s = fail(AIM_ENUMERIC, "non-finite residual"); break; }
        relres[r] = bnr > 0 ? rn / bnr : 0.0;
        conv[r] = relres[r] <= opts->tol;
        all = all && (conv[r] || iters[r] >= opts->max_iter);
        if (!conv[r]) worst = std::max(worst, relres[r]);
      }
      if (s != AIM_OK || all) break;
      if (has_deadline && std::chrono::steady_clock::now() > deadline) { s = fail(AIM_ETIMEOUT, "solve time limit reached"); break; }
      // inner solve A d = r with the FP32 grid product
      cudaMemsetAsync(dd, 0, vsz * sizeof(double2), st);
      // inner tolerance (on the Arnoldi estimate, relative to ||r||): fixed, or half the reduction
      // still needed by the right-hand side that is furthest from tol, so that one inner cycle
      // usually ends the solve
      const double itol = opts->inner_tol > 0
                              ? opts->inner_tol
                              : std::min(0.5, std::max(1e-7, 0.5 * opts->tol / std::max(worst, 1e-300)));
      s = gmres_core(ctx, system, AIM_MIXED, nrhs, rr, dd, itol, opts->restart, opts->max_iter, &it_inner, &rel_inner,
                     &conv_inner, deadline, has_deadline, st, /*single_cycle=*/true);
      if (s != AIM_OK) break;
      // only right-hand sides that have not converged take the correction
      for (int r = 0; r < nrhs; ++r) {
        iters[r] += it_inner[r];
        outer[r] += 1;
        if (conv[r]) cudaMemsetAsync(dd + (size_t)r * n, 0, n * sizeof(double2), st);
      }
      count_launches(K_GMRES, 1);
      k_add_vec<<<blocks_for((long long)vsz, 256), 256, 0, st>>>(x, dd, (int)vsz);
    }
    cudaFreeAsync(rr, st);
    if (s != AIM_OK) return s;
  }
  for (int r = 0; r < nrhs; ++r) {
    if (info) {
      info[r].iters = iters[r];
      info[r].outer_iters = outer[r];
      info[r].rel_res = relres[r];
      info[r].converged = conv[r];
    }
    if (!conv[r]) st_out = AIM_ENOCONV;
  }
  if (st_out != AIM_OK) return fail(st_out, "GMRES did not reach the tolerance within max_iter");
  return AIM_OK;
}

}  // namespace aim
