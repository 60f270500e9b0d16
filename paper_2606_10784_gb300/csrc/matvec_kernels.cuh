// The AIM matrix-vector product on the grid (Sec. III-A, Eq. 8; filtered: Sec. III-B, Eq. 10).
//
// For each channel (one projection of one right-hand side) the product
//     y = P_t^T [ F^-1( F(c) .* F(b) ) ]_restr ,   b = zero-padded P_s x
// runs as three grid passes and a gather:
//   k_row_fwd   sparse anterpolation of x onto grid row iy (u = P_s x, deterministic,
//               no atomics) fused with the forward P-point row DFT. The row has nonzeros
//               only in its first m <= P/2 entries, so X[2k] = DFT_H(a)[k] and
//               X[2k+1] = DFT_H(a w^n)[k], H = P/2, w = exp(-2 pi i/P).
//   k_col_conv  per column q: the same pruned forward DFT along the rows, the product with
//               the stored spectrum column F(c)[., q] (even symmetric, so only
//               (P/2+1)^2 values are stored), and the inverse DFT keeping rows < P/2 only:
//               y[n] = IDFT_H(Y_even)[n] + w^-n IDFT_H(Y_odd)[n].
//   k_row_inv   the inverse row DFT with the same split, scaled by 1/P^2, evaluated at the
//               grid points the test projection reads (the restriction [.]_restr): the two
//               half-transforms are recombined only at those points.
//   k_gather    y_i = sum over projections of coef * (P_t^T v)_i plus the near-field row
//               (C x)_i, eight lanes per unknown, deterministic.
// Each length-H transform runs as register-resident radix-E passes (fft_reg.cuh, E = 16 or 8
// elements per thread, a schedule choice): the first
// pass reads its operands straight from global memory (column and inverse row passes) and the
// last pass writes straight to global memory (forward row and column passes; the inverse row
// pass keeps its last pass in shared memory for the restriction), so shared memory carries only
// the exchanges between passes. A thread owns TPT transforms: with TPT = 2 the even- and odd-half transforms
// of a line sit in the same thread; with TPT = 1 they sit in adjacent lanes and recombine
// through a lane shuffle (half the registers per thread, twice the threads). Which one is
// faster depends on the element type; the autotuner measures both.
// The intermediate m x P grid of a channel is stored as column tiles of W entries
// (W * sizeof(complex) = 32 bytes) so that the column pass reads contiguous blocks and the
// row passes touch whole 32-byte sectors. Only grid rows that hold active points are stored.
#pragma once

#include <algorithm>
#include <type_traits>
#include <vector>

#include "aim_internal.h"
#include "gridtypes.cuh"

namespace aim {

// ------------------------------------------------------------------------------------
// row pass, forward
// ------------------------------------------------------------------------------------
struct RowFwdArgs {
  const double2* x;     // sparse mode: n * nrhs vectors; dense mode: m*m grid per channel
  int dense;
  int n, m, nrhs;
  const int* row_ptr;
  const int* act_ix;
  const int* sc_ptr;
  const int* sc_col;
  const double* w[kMaxProj];
  void* inter;
  const void* tw;
  int logH, logP, row_lo, nrows;
  int rows_per_cta;
};

// CTA: rows_per_cta rows of one channel; (3 - TPT) * H/E threads per row (E = 2^LOGE elements each).
constexpr int kAntChunk = 8;

// One work item of the forward row pass: rows [row_block * rows_per_cta, +rows_per_cta) of channel c.
// Every thread of the CTA calls it (it holds barriers); `smraw` is the CTA's dynamic shared memory.
template <typename CT, int TPT, int LOGE>
__device__ __forceinline__ void row_fwd_item(const RowFwdArgs& a, int row_block, int c, unsigned char* smraw) {
  using T2 = CT;
  constexpr int W = GridT<CT>::W, NF = TPT, LPT = 3 - TPT;
  T2* sm = reinterpret_cast<T2*>(smraw);
  const int H = 1 << a.logH, P = 1 << a.logP, tpf = H >> LOGE, HS = padded_len<LOGE>(H);
  const int per_row = LPT * tpf;
  const int g = threadIdx.x / per_row, rem = threadIdx.x - g * per_row;
  const int half = TPT == 1 ? (rem & 1) : 0, j = TPT == 1 ? (rem >> 1) : rem;
  const int rloc = row_block * a.rows_per_cta + g;
  const bool live = rloc < a.nrows;
  const int iy = a.row_lo + rloc;
  const T2* tw = static_cast<const T2*>(a.tw);
  const int fbA = (2 * g) * HS;
  int fb[NF];
#pragma unroll
  for (int f = 0; f < NF; ++f) fb[f] = (2 * g + (TPT == 1 ? half : f)) * HS;
  // zero the row buffer, then anterpolate u = P_s x into it (the row's active-point range is
  // loaded first so that its latency overlaps the zeroing). Forming u w^n here, at the active
  // points only and into a second zeroed buffer, was measured: 0.6 % faster in double-float and
  // 3 % slower in complex64, so pass 0 keeps the products.
  int a0 = 0, a1 = 0;
  if (live && !a.dense) {
    a0 = a.row_ptr[iy];
    a1 = a.row_ptr[iy + 1];
  }
  for (int i = rem; i < HS; i += per_row) sm[fbA + i] = czero<T2>();
  __syncthreads();
  if (live) {
    if (a.dense) {
      const double2* u = a.x + (size_t)c * a.m * a.m + (size_t)iy * a.m;
      for (int ix = rem; ix < a.m; ix += per_row) {
        const double2 v = u[ix];
        sm[fbA + padi<LOGE>(ix)] = cfrom<T2>(v.x, v.y);
      }
    } else {
      const int pj = c / a.nrhs, r = c - pj * a.nrhs;
      // projection weights by unrolled compare (indexing the argument array with a runtime
      // index would copy it to local memory)
      const double* w = a.w[0];
#pragma unroll
      for (int q = 1; q < kMaxProj; ++q)
        if (q == pj) w = a.w[q];
      const double2* xv = a.x + (size_t)r * a.n;
      for (int ap = a0 + rem; ap < a1; ap += per_row) {
        // a grid row holds few active points (tens), each with a handful of entries, so most of
        // the CTA waits here: the loads of up to kAntChunk entries are issued together before
        // their FMAs, which run in entry order as a plain loop would
        double re = 0.0, im = 0.0;
        const int e0 = a.sc_ptr[ap], e1 = a.sc_ptr[ap + 1];
        for (int e = e0; e < e1; e += kAntChunk) {
          int col[kAntChunk];
          double ww[kAntChunk];
          double2 xx[kAntChunk];
#pragma unroll
          for (int u = 0; u < kAntChunk; ++u) {
            col[u] = e + u < e1 ? a.sc_col[e + u] : 0;
            ww[u] = e + u < e1 ? w[e + u] : 0.0;
          }
#pragma unroll
          for (int u = 0; u < kAntChunk; ++u) xx[u] = e + u < e1 ? xv[col[u]] : double2{0.0, 0.0};
#pragma unroll
          for (int u = 0; u < kAntChunk; ++u) {
            if (e + u < e1) {
              re = fma(ww[u], xx[u].x, re);
              im = fma(ww[u], xx[u].y, im);
            }
          }
        }
        sm[fbA + padi<LOGE>(a.act_ix[ap])] = cfrom<T2>(re, im);
      }
    }
  }
  __syncthreads();
  // pass 0 (radix E, Ns = 1): the transform of a and/or of a w^n
  {
    const int lognb = a.logH - LOGE;
    T2 v[NF][1 << LOGE];
#pragma unroll
    for (int r = 0; r < (1 << LOGE); ++r) {
      const int nn = j + (r << lognb);
      const T2 x = sm[fbA + padi<LOGE>(nn)];
#pragma unroll
      for (int f = 0; f < NF; ++f) v[f][r] = (TPT == 1 ? half : f) ? cmul(x, ldro(&tw[nn])) : x;
    }
#pragma unroll
    for (int f = 0; f < NF; ++f) dft_reg<(1 << LOGE), false>(v[f]);
    __syncthreads();
#pragma unroll
    for (int f = 0; f < NF; ++f)
#pragma unroll
      for (int r = 0; r < (1 << LOGE); ++r) sm[fb[f] + padi<LOGE>((j << LOGE) + r)] = v[f][r];
    __syncthreads();
  }
  const int np = fft_npass<LOGE>(a.logH);
  smem_passes<false, NF, LOGE>(sm, fb, j, tpf, a.logH, 1, np - 1, LOGE, tw, a.logP, Identity{});
  int logNs = 0;
  for (int p = 0; p < np - 1; ++p) logNs += fft_logr<LOGE>(p, a.logH);
  // last pass: X[2k + half] straight to the tiled intermediate
  T2* out = static_cast<T2*>(a.inter) + (size_t)c * P * a.nrows;
  last_pass_dispatch<false, NF, LOGE>(sm, fb, j, tpf, a.logH, logNs, tw, a.logP, [&](int k, const T2 (&v)[NF]) {
    if (!live) return;
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      const int q = 2 * k + (TPT == 1 ? half : f);
      out[((size_t)(q / W) * a.nrows + rloc) * W + (q % W)] = v[f];
    }
  });
}

template <typename CT, int TPT, int LOGE>
__global__ void __launch_bounds__(LaunchMax<CT, TPT, LOGE>::value) k_row_fwd(RowFwdArgs a) {
  extern __shared__ __align__(16) unsigned char smraw[];
  row_fwd_item<CT, TPT, LOGE>(a, blockIdx.x, blockIdx.y, smraw);
}

// ------------------------------------------------------------------------------------
// column pass: forward DFT x spectrum x inverse DFT
// ------------------------------------------------------------------------------------
struct ColArgs {
  void* inter;
  const void* spec;
  const int* live;     // filtered spectrum: per column q' <= P/2, 0 where the mask zeroes it; else null
  const void* tw;
  int logH, logP, row_lo, nrows;
  int log_cols;        // log2 of the columns of one channel per CTA
  int chan_x;          // grid order: channels along x (1) or column tiles along x (0)
};

// Recombination of the even- and odd-half inverse transforms: with TPT = 2 both are in the
// thread; with TPT = 1 the partner lane holds the other one (all lanes must call this).
template <int TPT, typename T2>
__device__ __forceinline__ T2 recombine(const T2 (&v)[TPT], int half, const T2* __restrict__ tw, int nn) {
  if constexpr (TPT == 2) {
    return cadd(v[0], cmulc(v[1], ldro(&tw[nn])));
  } else {
    const T2 other = shfl_pair(v[0]);
    return half ? other : cadd(v[0], cmulc(other, ldro(&tw[nn])));
  }
}

// CTA: 2^log_cols consecutive columns of one channel; (3 - TPT) * H/E threads per column.
// Lane order puts the columns of a tile that the CTA holds (min(2^log_cols, W) of them) in
// adjacent lanes (lane pairs when TPT = 1), so with a whole tile per CTA the global loads and
// stores of a warp are whole 32-byte sectors; with fewer columns per CTA the CTAs of the
// neighbouring columns read the rest of each sector, through L2.
// One work item of the column pass: column tile `ctile` (2^log_cols columns) of channel c.
template <typename CT, int TPT, int LOGE>
__device__ __forceinline__ void col_conv_item(const ColArgs& a, int ctile, int c, unsigned char* smraw) {
  using T2 = CT;
  constexpr int W = GridT<CT>::W, NF = TPT, LPT = 3 - TPT;
  T2* sm = reinterpret_cast<T2*>(smraw);
  const int H = 1 << a.logH, P = 1 << a.logP, tpf = H >> LOGE, HS = padded_len<LOGE>(H);
  const int cw = min(1 << a.log_cols, W);               // columns side by side in the lanes
  const int per_grp = LPT * cw * tpf;
  const int g = threadIdx.x / per_grp, rem = threadIdx.x - g * per_grp;
  const int half = TPT == 1 ? (rem & 1) : 0;
  const int r2 = TPT == 1 ? (rem >> 1) : rem;
  const int wl = r2 & (cw - 1), j = r2 / cw;
  const int colc = g * cw + wl;                         // column within the CTA
  const int qcol = (ctile << a.log_cols) + colc;   // column of the grid
  const int w = qcol & (W - 1), tile = qcol / W;
  if (a.live != nullptr) {
    // the filtered spectrum (Eq. 10) vanishes on columns beyond the mask radius: when it does on
    // every column of this CTA their product is zero, so write zeros and skip the transforms
    // (the same decision in every thread: the early return is uniform)
    bool any = false;
    for (int cc = 0; cc < (1 << a.log_cols); ++cc) {
      const int q = (ctile << a.log_cols) + cc;
      any = any || a.live[min(q, P - q)] != 0;
    }
    if (!any) {
      T2* base = static_cast<T2*>(a.inter) + (size_t)c * P * a.nrows;
      const int total = (1 << a.log_cols) * a.nrows;
      for (int e = threadIdx.x; e < total; e += blockDim.x) {
        const int cc = e / a.nrows, row = e - cc * a.nrows;
        const int q = (ctile << a.log_cols) + cc;
        base[((size_t)(q / W) * a.nrows + row) * W + (q & (W - 1))] = czero<T2>();
      }
      return;
    }
  }
  int fb[NF];
#pragma unroll
  for (int f = 0; f < NF; ++f) fb[f] = (2 * colc + (TPT == 1 ? half : f)) * HS;
  const T2* tw = static_cast<const T2*>(a.tw);
  T2* blk = static_cast<T2*>(a.inter) + (size_t)c * P * a.nrows + (size_t)tile * a.nrows * W;
  const int row_hi = a.row_lo + a.nrows - 1;
  // pass 0 from global: a[n] and/or a[n] w^n, n = j + (H/E)-stride
  {
    const int lognb = a.logH - LOGE;
    T2 v[NF][1 << LOGE];
#pragma unroll
    for (int r = 0; r < (1 << LOGE); ++r) {
      const int nn = j + (r << lognb);
      const T2 x = (nn >= a.row_lo && nn <= row_hi) ? blk[(nn - a.row_lo) * W + w] : czero<T2>();
#pragma unroll
      for (int f = 0; f < NF; ++f) v[f][r] = (TPT == 1 ? half : f) ? cmul(x, ldro(&tw[nn])) : x;
    }
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      dft_reg<(1 << LOGE), false>(v[f]);
#pragma unroll
      for (int r = 0; r < (1 << LOGE); ++r) sm[fb[f] + padi<LOGE>((j << LOGE) + r)] = v[f][r];
    }
    __syncthreads();
  }
  const int np = fft_npass<LOGE>(a.logH);
  // remaining forward passes but the last
  smem_passes<false, NF, LOGE>(sm, fb, j, tpf, a.logH, 1, np - 1, LOGE, tw, a.logP, Identity{});
  // last forward pass, product with the spectrum column, first inverse pass (same radix), in
  // registers; the inverse then runs its radix-E passes
  const int lr0 = fft_logr<LOGE>(np - 1, a.logH);
  {
    const int qq = min(qcol, P - qcol);
    const T2* col = static_cast<const T2*>(a.spec) + (size_t)qq * (H + 1);
    const int half_h = H >> 1;
    auto spec_mul = [&](int f, int k, T2 v) {
      const int odd = TPT == 1 ? half : f;
      const T2 s = odd ? ldro(&col[half_h + 1 + min(k, H - 1 - k)]) : ldro(&col[min(k, H - k)]);
      return cmul(v, s);
    };
    conv_mid_dispatch<NF, LOGE>(lr0, sm, fb, j, tpf, a.logH, tw, a.logP, spec_mul);
  }
  for (int p = 1; p < np - 1; ++p)
    smem_pass<LOGE, true, NF, LOGE>(sm, fb, j, tpf, a.logH, lr0 + LOGE * (p - 1), tw, a.logP, Identity{});
  // last inverse pass (radix E, Ns = H/E) recombines y[n] = A[n] + conj(w^n) B[n] for kept rows
  last_pass<LOGE, true, NF, LOGE>(sm, fb, j, tpf, a.logH, a.logH - LOGE, tw, a.logP, [&](int nn, const T2 (&v)[NF]) {
    const T2 y = recombine<TPT>(v, half, tw, nn);
    if (!half && nn >= a.row_lo && nn <= row_hi) blk[(nn - a.row_lo) * W + w] = y;
  });
}

template <typename CT, int TPT, int LOGE>
__global__ void __launch_bounds__(LaunchMax<CT, TPT, LOGE>::value) k_col_conv(ColArgs a) {
  extern __shared__ __align__(16) unsigned char smraw[];
  // with many channels they run along x: the channels of one column tile run back to back and
  // share its spectrum column through L2 (64 right-hand sides: 2.82 -> 2.67 ms per launch);
  // with few, column tiles run along x (no gain measured for 3 channels)
  col_conv_item<CT, TPT, LOGE>(a, a.chan_x ? blockIdx.y : blockIdx.x, a.chan_x ? blockIdx.x : blockIdx.y, smraw);
}

// ------------------------------------------------------------------------------------
// row pass, inverse + restriction
// ------------------------------------------------------------------------------------
struct RowInvArgs {
  const void* inter;
  const void* tw;
  void* vact;          // sparse mode output: channel-major, n_act per channel
  double2* dense_out;  // dense mode output: m*m per channel
  int dense;
  int m, n_act;
  const int* row_ptr;
  const int* act_ix;
  int logH, logP, row_lo, nrows;
  double scale;
  int rows_per_cta;
};

// One work item of the inverse row pass: rows [row_block * rows_per_cta, +rows_per_cta) of channel c.
template <typename CT, int TPT, int LOGE>
__device__ __forceinline__ void row_inv_item(const RowInvArgs& a, int row_block, int c, unsigned char* smraw) {
  using T2 = CT;
  using VT = typename GridT<CT>::VT;
  constexpr int W = GridT<CT>::W, NF = TPT, LPT = 3 - TPT;
  T2* sm = reinterpret_cast<T2*>(smraw);
  const int H = 1 << a.logH, P = 1 << a.logP, tpf = H >> LOGE, HS = padded_len<LOGE>(H);
  const int per_row = LPT * tpf;
  const int g = threadIdx.x / per_row, rem = threadIdx.x - g * per_row;
  const int half = TPT == 1 ? (rem & 1) : 0, j = TPT == 1 ? (rem >> 1) : rem;
  const int rloc = row_block * a.rows_per_cta + g;
  const bool live = rloc < a.nrows;
  const int iy = a.row_lo + rloc;
  const T2* tw = static_cast<const T2*>(a.tw);
  const int fbA = (2 * g) * HS;
  int fb[NF];
#pragma unroll
  for (int f = 0; f < NF; ++f) fb[f] = (2 * g + (TPT == 1 ? half : f)) * HS;
  const T2* blk = static_cast<const T2*>(a.inter) + (size_t)c * P * a.nrows;
  // pass 0 (inverse, radix E, Ns = 1) from global: Y[2k] and/or Y[2k+1]
  {
    const int lognb = a.logH - LOGE;
    T2 v[NF][1 << LOGE];
#pragma unroll
    for (int r = 0; r < (1 << LOGE); ++r) {
#pragma unroll
      for (int f = 0; f < NF; ++f) {
        const int q = 2 * (j + (r << lognb)) + (TPT == 1 ? half : f);
        v[f][r] = live ? blk[((size_t)(q / W) * a.nrows + rloc) * W + (q % W)] : czero<T2>();
      }
    }
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      dft_reg<(1 << LOGE), true>(v[f]);
#pragma unroll
      for (int r = 0; r < (1 << LOGE); ++r) sm[fb[f] + padi<LOGE>((j << LOGE) + r)] = v[f][r];
    }
    __syncthreads();
  }
  const int np = fft_npass<LOGE>(a.logH);
  smem_passes<true, NF, LOGE>(sm, fb, j, tpf, a.logH, 1, np - 1, LOGE, tw, a.logP, Identity{});
  int logNs = 0;
  for (int p = 0; p < np - 1; ++p) logNs += fft_logr<LOGE>(p, a.logH);
  const double sc = a.scale;
  if (a.dense) {
    double2* out = a.dense_out + (size_t)c * a.m * a.m + (size_t)iy * a.m;
    last_pass_dispatch<true, NF, LOGE>(sm, fb, j, tpf, a.logH, logNs, tw, a.logP, [&](int nn, const T2 (&v)[NF]) {
      const T2 y = recombine<TPT>(v, half, tw, nn);
      if (!half && live && nn < a.m) out[nn] = cto_d2(y, sc);
    });
    return;
  }
  // sparse mode: the last pass as one more shared-memory pass leaves both half-transforms in
  // natural order in their own buffers, and the recombination y = Y_even + w^-n Y_odd runs only
  // at the row's active points (tens of the H outputs)
  smem_passes<true, NF, LOGE>(sm, fb, j, tpf, a.logH, np - 1, np, logNs, tw, a.logP, Identity{});
  if (live) {
    VT* out = static_cast<VT*>(a.vact) + (size_t)c * a.n_act;
    const int a1 = a.row_ptr[iy + 1];
    for (int ap = a.row_ptr[iy] + rem; ap < a1; ap += per_row) {
      const int ix = a.act_ix[ap];
      const T2 y = cadd(sm[fbA + padi<LOGE>(ix)], cmulc(sm[fbA + HS + padi<LOGE>(ix)], ldro(&tw[ix])));
      out[ap] = cto_vt(y, sc);
    }
  }
}

template <typename CT, int TPT, int LOGE>
__global__ void __launch_bounds__(LaunchMax<CT, TPT, LOGE>::value) k_row_inv(RowInvArgs a) {
  extern __shared__ __align__(16) unsigned char smraw[];
  row_inv_item<CT, TPT, LOGE>(a, blockIdx.x, blockIdx.y, smraw);
}

// ------------------------------------------------------------------------------------
// gather + near field, Gram inverse
// ------------------------------------------------------------------------------------
struct GatherArgs {
  const void* vact;
  int n_act, n, nrhs, nproj;
  const int* ga_ptr;
  const int* ga_act;
  const double* w[kMaxProj];
  double2 coef[kMaxProj];
  const int* nptr;
  const int* ncol;
  const void* nval;
  const double2* x;
  double2 out_scale;
  double2* y;
  int accumulate;
};

// A group of kGatherLanes adjacent lanes per unknown i and block of up to kGatherRhs right-hand
// sides (1 when there is only one), four groups to a warp: the CSR entries of row i (weights,
// active-point indices, near-field values and columns) are loaded once and used for every
// right-hand side of the block. For each right-hand side, lane g of the group sums the entries
// e = e0 + g, e0 + g + 8, ... in order, and the group then adds its partial sums by xor shuffles,
// so the result does not depend on the block size. The FP64 pipe sets the cost here: a whole
// warp per unknown spent more FP64 instructions on coefficient products and its five-step
// shuffle tree than on the entries themselves. With a complex64 grid (mixed precision) the
// projection sums run in FP32 (Acc): converting every grid value to FP64 cost as much as the
// FP64 products, conversions running at the FP64 rate here. The coefficient products, the
// near-field rows and the sums over projections stay in FP64.
constexpr int kGatherLanes = 8;

// Gather for the threads of virtual block `vblock` (blockDim.x threads each); all 32 lanes of every
// warp call it (the group sums are shuffles).
template <typename T2, int kGatherRhs>
__device__ __forceinline__ void gather_item(const GatherArgs& a, long long vblock) {
  static_assert(kGatherRhs <= kGatherLanes, "lane g writes right-hand side r0 + g");
  using Acc = typename std::conditional<std::is_same<T2, float2>::value, float, double>::type;
  const long long grp = (vblock * blockDim.x + threadIdx.x) / kGatherLanes;
  const int g = threadIdx.x & (kGatherLanes - 1);
  const int nblk = (a.nrhs + kGatherRhs - 1) / kGatherRhs;
  const bool valid = grp < (long long)a.n * nblk;
  const int rb = valid ? (int)(grp / a.n) : 0, i = valid ? (int)(grp - (long long)rb * a.n) : 0;
  const int r0 = rb * kGatherRhs, nr = min(kGatherRhs, a.nrhs - r0);
  double re[kGatherRhs], im[kGatherRhs];
#pragma unroll
  for (int q = 0; q < kGatherRhs; ++q) re[q] = im[q] = 0.0;
  if (valid) {
    const int e0 = a.ga_ptr[i], e1 = a.ga_ptr[i + 1];
    for (int pj = 0; pj < a.nproj; ++pj) {
      const T2* v = static_cast<const T2*>(a.vact) + (size_t)(pj * a.nrhs + r0) * a.n_act;
      const double* w = a.w[pj];
      Acc cr[kGatherRhs], ci[kGatherRhs];
#pragma unroll
      for (int q = 0; q < kGatherRhs; ++q) cr[q] = ci[q] = Acc(0);
      for (int e = e0 + g; e < e1; e += kGatherLanes) {
        const Acc ww = static_cast<Acc>(w[e]);
        const int act = a.ga_act[e];
#pragma unroll
        for (int q = 0; q < kGatherRhs; ++q) {
          if (q < nr) {
            const T2 val = v[(size_t)q * a.n_act + act];
            cr[q] = fma(ww, static_cast<Acc>(val.x), cr[q]);
            ci[q] = fma(ww, static_cast<Acc>(val.y), ci[q]);
          }
        }
      }
      const double2 cf = a.coef[pj];
#pragma unroll
      for (int q = 0; q < kGatherRhs; ++q) {
        const double crq = cr[q], ciq = ci[q];
        re[q] += cf.x * crq - cf.y * ciq;
        im[q] += cf.x * ciq + cf.y * crq;
      }
    }
    if (a.nptr != nullptr) {
      const T2* val = static_cast<const T2*>(a.nval);
      const int n1 = a.nptr[i + 1];
      for (int e = a.nptr[i] + g; e < n1; e += kGatherLanes) {
        const T2 cv = val[e];
        const int col = a.ncol[e];
#pragma unroll
        for (int q = 0; q < kGatherRhs; ++q) {
          if (q < nr) {
            const double2 xx = a.x[(size_t)(r0 + q) * a.n + col];
            re[q] += (double)cv.x * xx.x - (double)cv.y * xx.y;
            im[q] += (double)cv.x * xx.y + (double)cv.y * xx.x;
          }
        }
      }
    }
  }
  // every lane of the warp takes part in the shuffles (groups past the end carry zeros)
#pragma unroll
  for (int q = 0; q < kGatherRhs; ++q) {
#pragma unroll
    for (int off = kGatherLanes / 2; off > 0; off >>= 1) {
      re[q] += __shfl_xor_sync(0xffffffffu, re[q], off);
      im[q] += __shfl_xor_sync(0xffffffffu, im[q], off);
    }
  }
  if (valid && g < nr) {
    // lane g writes right-hand side r0 + g (select by unrolled compare: no local-memory indexing)
    double xr = 0.0, xi = 0.0;
#pragma unroll
    for (int q = 0; q < kGatherRhs; ++q)
      if (q == g) { xr = re[q]; xi = im[q]; }
    const double2 s = a.out_scale;
    double2 o = double2{s.x * xr - s.y * xi, s.x * xi + s.y * xr};
    double2* dst = a.y + (size_t)(r0 + g) * a.n + i;
    if (a.accumulate) {
      const double2 prev = *dst;
      o.x += prev.x;
      o.y += prev.y;
    }
    *dst = o;
  }
}

template <typename T2, int kGatherRhs>
__global__ void k_gather(GatherArgs a) {
  gather_item<T2, kGatherRhs>(a, blockIdx.x);
}

// ------------------------------------------------------------------------------------
// launch configuration
// ------------------------------------------------------------------------------------
template <typename K>
static aim_status ensure_smem(K kernel, size_t bytes) {
  if (bytes > 48 * 1024) {
    AIM_CUDA_TRY(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
  }
  return AIM_OK;
}

// tables of the context in the element type of the grid product
static const void* twiddles(const aim_ctx* c, float2*) { return c->twf; }
static const void* twiddles(const aim_ctx* c, double2*) { return c->tw; }
static const void* twiddles(const aim_ctx* c, dfc*) { return c->twdf; }
static const void* spectrum(const aim_ctx* c, bool f, float2*) { return f ? (const void*)c->specAf : c->specUf; }
static const void* spectrum(const aim_ctx* c, bool f, double2*) { return f ? (const void*)c->specA : c->specU; }
static const void* spectrum(const aim_ctx* c, bool f, dfc*) { return f ? (const void*)c->specAdf : c->specUdf; }
static const void* near_values(const NearField* nf, int which, float2*) { return nf->valf[which]; }
static const void* near_values(const NearField* nf, int which, double2*) { return nf->val[which]; }
static const void* near_values(const NearField* nf, int which, dfc*) { return nf->val[which]; }
static int precision_of(float2*) { return AIM_MIXED; }
static int precision_of(double2*) { return AIM_FP64_NATIVE; }
static int precision_of(dfc*) { return AIM_FP64; }

constexpr size_t kMaxDynSmem = 227 * 1024;   // opt-in dynamic shared memory per CTA

// Which (transforms per thread, elements per thread) pairs are compiled for an element type:
// native binary64 keeps two transforms of 16 elements per thread
template <typename CT, int TPT, int LOGE>
struct Supports {
  static constexpr bool value = std::is_same<CT, double2>::value ? (TPT == 2 && LOGE == 4) : true;
};

inline int loge_of(const Schedule& sc) { return sc.elems == 8 ? 3 : 4; }

// columns per column-pass CTA: the schedule's choice, else the fewest whole tiles of W
// columns that give at least 128 threads
template <typename CT, int TPT, int LOGE>
static int col_cols_of(const Schedule& sc, int logH, int logP) {
  constexpr int W = GridT<CT>::W, LPT = 3 - TPT;
  if (sc.col_cols > 0) return sc.col_cols;
  const int tpf = (1 << logH) >> LOGE, ntiles = (1 << logP) / W;
  int tpc = 1;
  while (tpc * LPT * W * tpf < 128 && tpc < ntiles) tpc *= 2;
  return tpc * W;
}

template <typename CT, int TPT, int LOGE>
static bool feasible_tpt(const Schedule& sc, int logH, int logP) {
  if constexpr (!Supports<CT, TPT, LOGE>::value) {
    return false;
  } else {
    constexpr int LPT = 3 - TPT;
    if (logH < LOGE + 1) return false;   // at least two passes
    const int H = 1 << logH, tpf = H >> LOGE, cols = col_cols_of<CT, TPT, LOGE>(sc, logH, logP);
    if (cols < 1 || (cols & (cols - 1)) || cols > (1 << logP)) return false;
    if (LPT * cols * tpf > LaunchMax<CT, TPT, LOGE>::value || LPT * cols * tpf < 32) return false;
    if (2 * (size_t)cols * padded_len<LOGE>(H) * sizeof(CT) > kMaxDynSmem) return false;
    if (sc.min_row_threads < 32 || sc.min_row_threads > 1024) return false;
    // row passes: one row per CTA must fit too
    if (2 * (size_t)padded_len<LOGE>(H) * sizeof(CT) > kMaxDynSmem || LPT * tpf > LaunchMax<CT, TPT, LOGE>::value)
      return false;
    return true;
  }
}

template <typename CT>
static bool feasible_for(const Schedule& s, int logH, int logP) {
  if (s.tpt != 1 && s.tpt != 2) return false;
  if (s.elems != 0 && s.elems != 8 && s.elems != 16) return false;
  if (loge_of(s) == 3)
    return s.tpt == 1 ? feasible_tpt<CT, 1, 3>(s, logH, logP) : feasible_tpt<CT, 2, 3>(s, logH, logP);
  return s.tpt == 1 ? feasible_tpt<CT, 1, 4>(s, logH, logP) : feasible_tpt<CT, 2, 4>(s, logH, logP);
}

template <typename CT, int TPT, int LOGE>
static aim_status launch_tpt(aim_ctx* ctx, int channels, bool filtered, RowFwdArgs fa, RowInvArgs ia,
                             void* inter, const Schedule& sc, cudaStream_t st) {
  const int min_row_threads = sc.min_row_threads;
  using T2 = CT;
  constexpr int LPT = 3 - TPT;
  const int H = ctx->H, tpf = H >> LOGE, HS = padded_len<LOGE>(H);
  const void* tw = twiddles(ctx, (CT*)nullptr);
  const void* spec = spectrum(ctx, filtered, (CT*)nullptr);

  // rows per CTA: at least min_row_threads threads (fewer when the grid has fewer rows, but
  // never less than a full warp: the recombination shuffles need all 32 lanes; rows past the
  // last one load zeros and store nothing), within the launch bound
  int rpc = 1;
  while (((rpc * LPT * tpf < min_row_threads && rpc < ctx->nrows) || rpc * LPT * tpf < 32) &&
         2 * rpc * LPT * tpf <= LaunchMax<CT, TPT, LOGE>::value)
    rpc *= 2;
  const int row_blocks = (ctx->nrows + rpc - 1) / rpc;
  const size_t sm_row = 2 * (size_t)rpc * HS * sizeof(T2);

  fa.tw = tw;
  fa.logH = ctx->logH;
  fa.logP = ctx->logP;
  fa.row_lo = ctx->row_lo;
  fa.nrows = ctx->nrows;
  fa.inter = inter;
  fa.rows_per_cta = rpc;
  AIM_TRY(ensure_smem(k_row_fwd<CT, TPT, LOGE>, sm_row));
  {
    ProfScope ps(K_ROW_FWD, st);
    k_row_fwd<CT, TPT, LOGE><<<dim3(row_blocks, channels), rpc * LPT * tpf, sm_row, st>>>(fa);
  }
  AIM_CUDA_TRY(cudaGetLastError());

  // column pass
  const int cols = col_cols_of<CT, TPT, LOGE>(sc, ctx->logH, ctx->logP);
  int log_cols = 0;
  while ((1 << log_cols) < cols) ++log_cols;
  ColArgs ca;
  ca.inter = inter;
  ca.spec = spec;
  ca.live = filtered ? ctx->specA_live : nullptr;
  ca.tw = tw;
  ca.logH = ctx->logH;
  ca.logP = ctx->logP;
  ca.row_lo = ctx->row_lo;
  ca.nrows = ctx->nrows;
  ca.log_cols = log_cols;
  const size_t sm_col = 2 * (size_t)cols * HS * sizeof(T2);
  if (ctx->P / cols > 65535) return fail(AIM_EINVAL, "too many column tiles for one column-pass grid");
  constexpr int kChanX = 8;   // channels from which the column-pass grid runs channels along x
  AIM_TRY(ensure_smem(k_col_conv<CT, TPT, LOGE>, sm_col));
  {
    ProfScope ps(K_COL_CONV, st);
    ca.chan_x = channels >= kChanX;
    const dim3 grid = ca.chan_x ? dim3(channels, ctx->P / cols) : dim3(ctx->P / cols, channels);
    k_col_conv<CT, TPT, LOGE><<<grid, cols * LPT * tpf, sm_col, st>>>(ca);
  }
  AIM_CUDA_TRY(cudaGetLastError());

  // row inverse
  ia.inter = inter;
  ia.tw = tw;
  ia.logH = ctx->logH;
  ia.logP = ctx->logP;
  ia.row_lo = ctx->row_lo;
  ia.nrows = ctx->nrows;
  ia.scale = 1.0 / ((double)ctx->P * (double)ctx->P);
  ia.rows_per_cta = rpc;
  AIM_TRY(ensure_smem(k_row_inv<CT, TPT, LOGE>, sm_row));
  {
    ProfScope ps(K_ROW_INV, st);
    k_row_inv<CT, TPT, LOGE><<<dim3(row_blocks, channels), rpc * LPT * tpf, sm_row, st>>>(ia);
  }
  AIM_CUDA_TRY(cudaGetLastError());
  return AIM_OK;
}

template <typename CT>
static aim_status launch_three_passes(aim_ctx* ctx, int channels, bool filtered, RowFwdArgs fa, RowInvArgs ia,
                                      void* inter, cudaStream_t st) {
  if (channels > 65535) return fail(AIM_EINVAL, "too many channels in one grid pass");
  if (ctx->H < 32) return fail(AIM_EINVAL, "embedding side P must be >= 64");
  const int p = precision_of((CT*)nullptr);
  const Schedule sc = ctx->sched[p];
  if (!feasible_for<CT>(sc, ctx->logH, ctx->logP)) return fail(AIM_EINVAL, "launch schedule not feasible");
  if constexpr (std::is_same<CT, double2>::value) {
    return launch_tpt<CT, 2, 4>(ctx, channels, filtered, fa, ia, inter, sc, st);
  } else {
    if (loge_of(sc) == 3) {
      if (sc.tpt == 1) return launch_tpt<CT, 1, 3>(ctx, channels, filtered, fa, ia, inter, sc, st);
      return launch_tpt<CT, 2, 3>(ctx, channels, filtered, fa, ia, inter, sc, st);
    }
    if (sc.tpt == 1) return launch_tpt<CT, 1, 4>(ctx, channels, filtered, fa, ia, inter, sc, st);
    return launch_tpt<CT, 2, 4>(ctx, channels, filtered, fa, ia, inter, sc, st);
  }
}

template <typename CT>
aim_status grid_pass(aim_ctx* ctx, const PassSpec& spec, int nrhs, const double2* x, double2* y,
                     cudaStream_t st) {
  using VT = typename GridT<CT>::VT;
  const int precision = precision_of((CT*)nullptr);
  const int channels = spec.nproj * nrhs;
  if (inter_bytes_needed(ctx, channels, precision) > ctx->inter_bytes ||
      (size_t)channels * ctx->n_act * sizeof(VT) > ctx->vact_bytes)
    return fail(AIM_ESTATE, "grid workspace not reserved for this many right-hand sides");

  RowFwdArgs fa{};
  fa.x = x;
  fa.dense = 0;
  fa.n = ctx->n;
  fa.m = ctx->m;
  fa.nrhs = nrhs;
  fa.row_ptr = ctx->row_ptr;
  fa.act_ix = ctx->act_ix;
  fa.sc_ptr = ctx->prj.sc_ptr;
  fa.sc_col = ctx->prj.sc_col;
  for (int pj = 0; pj < spec.nproj; ++pj) fa.w[pj] = ctx->prj.sc_w[spec.proj[pj]];
  RowInvArgs ia{};
  ia.vact = ctx->vact;
  ia.dense = 0;
  ia.m = ctx->m;
  ia.n_act = ctx->n_act;
  ia.row_ptr = ctx->row_ptr;
  ia.act_ix = ctx->act_ix;
  AIM_TRY(launch_three_passes<CT>(ctx, channels, spec.filtered, fa, ia, ctx->inter, st));

  GatherArgs ga{};
  ga.vact = ctx->vact;
  ga.n_act = ctx->n_act;
  ga.n = ctx->n;
  ga.nrhs = nrhs;
  ga.nproj = spec.nproj;
  ga.ga_ptr = ctx->prj.ga_ptr;
  ga.ga_act = ctx->prj.ga_act;
  for (int pj = 0; pj < spec.nproj; ++pj) {
    ga.w[pj] = ctx->prj.ga_w[spec.proj[pj]];
    ga.coef[pj] = spec.coef[pj];
  }
  if (spec.near != nullptr && spec.near->nnz > 0) {
    ga.nptr = spec.near->ptr;
    ga.ncol = spec.near->col;
    ga.nval = near_values(spec.near, spec.near_which, (CT*)nullptr);
  }
  ga.x = x;
  ga.out_scale = spec.out_scale;
  ga.y = y;
  ga.accumulate = 0;
  constexpr int kRhsBlock = 8;
  const int rb = nrhs == 1 ? 1 : kRhsBlock;
  const long long groups = (long long)ctx->n * ((nrhs + rb - 1) / rb);
  const int tpb = 256;
  const long long blocks = (groups * kGatherLanes + tpb - 1) / tpb;
  {
    ProfScope ps(K_GATHER, st);
    if (rb == 1)
      k_gather<VT, 1><<<(unsigned)blocks, tpb, 0, st>>>(ga);
    else
      k_gather<VT, kRhsBlock><<<(unsigned)blocks, tpb, 0, st>>>(ga);
  }
  AIM_CUDA_TRY(cudaGetLastError());
  return AIM_OK;
}

// ------------------------------------------------------------------------------------
// several grid passes (contexts of any size) in one persistent launch
// ------------------------------------------------------------------------------------
// One job is a whole grid pass of one context (its channels, its spectrum, its gather). The
// persistent kernel runs four phases over all jobs' work items: forward row pass, column pass,
// inverse row pass, gather. Every CTA takes items c, c + G, c + 2G, ... of the flattened item list
// of a phase (G = CTAs of the launch); each item fills the CTA's threads with lines (rows or
// columns) of its job, so a job with a shorter transform puts more lines into one item. A grid
// barrier separates the phases. The launch is cooperative, so all CTAs are resident and the
// barrier completes; its waits are bounded all the same: after max_spins polls a CTA records the
// failure in *err and every CTA leaves at its next barrier, and the host reports AIM_ETIMEOUT.
constexpr int kMaxMultiJobs = 32;

struct MultiJob {
  RowFwdArgs fa;
  ColArgs ca;
  RowInvArgs ia;
  GatherArgs ga;
  int row_items;       // row blocks per channel
  int col_items;       // column tiles per channel
  int channels;
  int tile_major;      // column items ordered tile by tile (the channels of a tile adjacent)
  int gather_rb;       // right-hand sides per gather group (1 or 8)
};

// The whole job table travels as the kernel's parameter (read-only, in the constant bank: a
// uniform load per field, as for the single-context kernels' arguments).
struct MultiArgs {
  MultiJob jobs[kMaxMultiJobs];
  int njobs;
  long long off[4][kMaxMultiJobs + 1];   // prefix sums of the items of each phase over the jobs
  unsigned* bar;                         // [arrivals, generation], zero at launch
  int* err;                              // 1 when a barrier wait gave up
  long long max_spins;
};

static_assert(sizeof(MultiArgs) <= 32000, "the job table must fit the kernel parameter space (32 KB)");

__device__ __forceinline__ bool multi_grid_barrier(const MultiArgs& m) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* gen = m.bar + 1;
    volatile int* err = m.err;
    const unsigned g0 = *gen;
    __threadfence();
    if (atomicAdd(m.bar, 1u) == gridDim.x - 1) {
      atomicExch(m.bar, 0u);
      __threadfence();
      atomicAdd(m.bar + 1, 1u);
    } else {
      long long spins = 0;
      while (*gen == g0) {
        if (*err != 0) break;
        if (++spins > m.max_spins) {
          atomicExch(m.err, 1);
          break;
        }
        __nanosleep(128);
      }
    }
    __threadfence();
    ok = *err == 0;
  }
  __syncthreads();
  return ok != 0;
}

template <typename CT, int TPT, int LOGE>
__global__ void __launch_bounds__(LaunchMax<CT, TPT, LOGE>::value) k_grid_multi(const __grid_constant__ MultiArgs m) {
  using VT = typename GridT<CT>::VT;
  extern __shared__ __align__(16) unsigned char smraw[];
  for (int phase = 0; phase < 4; ++phase) {
    const long long total = m.off[phase][m.njobs];
    for (long long it = blockIdx.x; it < total; it += gridDim.x) {
      int jb = 0;
      while (it >= m.off[phase][jb + 1]) ++jb;   // the same job in every thread of the CTA
      const MultiJob& J = m.jobs[jb];
      const long long local = it - m.off[phase][jb];
      if (phase == 0) {
        row_fwd_item<CT, TPT, LOGE>(J.fa, (int)(local % J.row_items), (int)(local / J.row_items), smraw);
      } else if (phase == 1) {
        // many channels (right-hand sides): the channels of one column tile run back to back and
        // share its spectrum column through L2, as the single-context launch orders them
        const int tile = J.tile_major ? (int)(local / J.channels) : (int)(local % J.col_items);
        const int ch = J.tile_major ? (int)(local % J.channels) : (int)(local / J.col_items);
        col_conv_item<CT, TPT, LOGE>(J.ca, tile, ch, smraw);
      } else if (phase == 2) {
        row_inv_item<CT, TPT, LOGE>(J.ia, (int)(local % J.row_items), (int)(local / J.row_items), smraw);
      } else if (J.gather_rb == 1) {
        gather_item<VT, 1>(J.ga, local);
      } else {
        gather_item<VT, 8>(J.ga, local);
      }
      __syncthreads();   // the next item reuses the shared memory
    }
    if (phase < 3 && !multi_grid_barrier(m)) return;
  }
}

// Runs the passes (all of element type CT, all contexts on the schedule geometry of jobs[0]: the
// same transforms per thread and elements per thread) in one persistent cooperative launch.
// scratch: 16 device bytes for the barrier and the error flag (zeroed here on the stream);
// err_host: pinned host int that receives the error flag after the launch (read it after a sync).
template <typename CT>
aim_status grid_pass_multi(const MultiPassSpec* passes, int count, unsigned* scratch, int* err_host, cudaStream_t st);

// Threads per CTA of a multi launch whose longest transform has half-length H: two lines of it and
// at least a whole 32-byte column tile of it (W columns), at least a warp, within the launch bound.
template <typename CT, int TPT, int LOGE>
static int multi_cta_threads(int H) {
  constexpr int LPT = 3 - TPT, W = GridT<CT>::W;
  constexpr int Lmax = LaunchMax<CT, TPT, LOGE>::value;
  int B = 32;
  while (B < std::max(2, W) * LPT * (H >> LOGE) && B < Lmax) B *= 2;
  return B;
}

// Whether a context with half-length H can share a launch of B threads per CTA: a CTA takes
// B / (threads per line) of its lines, a power of two of at least one and at most its P columns.
template <typename CT, int TPT, int LOGE>
static bool multi_fits(int B, int H) {
  constexpr int LPT = 3 - TPT;
  const int per_line = LPT * (H >> LOGE);
  return per_line >= 1 && B >= per_line && B / per_line <= 2 * H;
}

template <typename CT, int TPT, int LOGE>
static aim_status launch_multi(const MultiPassSpec* passes, int count, unsigned* scratch, cudaStream_t st) {
  using T2 = CT;
  using VT = typename GridT<CT>::VT;
  constexpr int LPT = 3 - TPT;
  int maxH = 1;
  for (int i = 0; i < count; ++i) maxH = std::max(maxH, passes[i].ctx->H);
  const int B = multi_cta_threads<CT, TPT, LOGE>(maxH);
  if (B < LPT * (maxH >> LOGE)) return fail(AIM_EINVAL, "transform too long for the multi-context launch");
  static thread_local MultiArgs m;   // 17 KB: kept off the stack
  m = MultiArgs{};
  m.njobs = count;
  m.bar = scratch;
  m.err = reinterpret_cast<int*>(scratch + 2);
  m.max_spins = 20000000;   // ~2.5 s of 128 ns polls
  size_t smem = 0;
  for (int i = 0; i < count; ++i) {
    const MultiPassSpec& ps = passes[i];
    aim_ctx* ctx = ps.ctx;
    const PassSpec& spec = ps.spec;
    const int H = ctx->H, P = ctx->P, tpf = H >> LOGE, HS = padded_len<LOGE>(H);
    const int lines = B / (LPT * tpf);
    if (!multi_fits<CT, TPT, LOGE>(B, H) || lines > P || (lines & (lines - 1)))
      return fail(AIM_EINVAL, "contexts of too different sizes for one multi-context launch");
    const int channels = spec.nproj * ps.nrhs;
    const int precision = precision_of((CT*)nullptr);
    if (inter_bytes_needed(ctx, channels, precision) > ctx->inter_bytes ||
        (size_t)channels * ctx->n_act * sizeof(VT) > ctx->vact_bytes)
      return fail(AIM_ESTATE, "grid workspace not reserved for this many right-hand sides");
    smem = std::max(smem, 2 * (size_t)lines * HS * sizeof(T2));
    MultiJob& J = m.jobs[i];
    const void* tw = twiddles(ctx, (CT*)nullptr);
    RowFwdArgs& fa = J.fa;
    fa.x = ps.x;
    fa.dense = 0;
    fa.n = ctx->n;
    fa.m = ctx->m;
    fa.nrhs = ps.nrhs;
    fa.row_ptr = ctx->row_ptr;
    fa.act_ix = ctx->act_ix;
    fa.sc_ptr = ctx->prj.sc_ptr;
    fa.sc_col = ctx->prj.sc_col;
    for (int pj = 0; pj < spec.nproj; ++pj) fa.w[pj] = ctx->prj.sc_w[spec.proj[pj]];
    fa.inter = ctx->inter;
    fa.tw = tw;
    fa.logH = ctx->logH;
    fa.logP = ctx->logP;
    fa.row_lo = ctx->row_lo;
    fa.nrows = ctx->nrows;
    fa.rows_per_cta = lines;
    ColArgs& ca = J.ca;
    ca.inter = ctx->inter;
    ca.spec = spectrum(ctx, spec.filtered, (CT*)nullptr);
    ca.live = spec.filtered ? ctx->specA_live : nullptr;
    ca.tw = tw;
    ca.logH = ctx->logH;
    ca.logP = ctx->logP;
    ca.row_lo = ctx->row_lo;
    ca.nrows = ctx->nrows;
    int lc = 0;
    while ((1 << lc) < lines) ++lc;
    ca.log_cols = lc;
    ca.chan_x = 0;
    RowInvArgs& ia = J.ia;
    ia.inter = ctx->inter;
    ia.tw = tw;
    ia.vact = ctx->vact;
    ia.dense = 0;
    ia.m = ctx->m;
    ia.n_act = ctx->n_act;
    ia.row_ptr = ctx->row_ptr;
    ia.act_ix = ctx->act_ix;
    ia.logH = ctx->logH;
    ia.logP = ctx->logP;
    ia.row_lo = ctx->row_lo;
    ia.nrows = ctx->nrows;
    ia.scale = 1.0 / ((double)P * (double)P);
    ia.rows_per_cta = lines;
    GatherArgs& ga = J.ga;
    ga.vact = ctx->vact;
    ga.n_act = ctx->n_act;
    ga.n = ctx->n;
    ga.nrhs = ps.nrhs;
    ga.nproj = spec.nproj;
    ga.ga_ptr = ctx->prj.ga_ptr;
    ga.ga_act = ctx->prj.ga_act;
    for (int pj = 0; pj < spec.nproj; ++pj) {
      ga.w[pj] = ctx->prj.ga_w[spec.proj[pj]];
      ga.coef[pj] = spec.coef[pj];
    }
    if (spec.near != nullptr && spec.near->nnz > 0) {
      ga.nptr = spec.near->ptr;
      ga.ncol = spec.near->col;
      ga.nval = near_values(spec.near, spec.near_which, (CT*)nullptr);
    }
    ga.x = ps.x;
    ga.out_scale = spec.out_scale;
    ga.y = ps.y;
    ga.accumulate = 0;
    J.gather_rb = ps.nrhs == 1 ? 1 : 8;
    J.row_items = (ctx->nrows + lines - 1) / lines;
    J.col_items = P / lines;
    J.channels = channels;
    J.tile_major = channels >= 8;
    const long long groups = (long long)ctx->n * ((ps.nrhs + J.gather_rb - 1) / J.gather_rb);
    const long long gblocks = (groups * kGatherLanes + B - 1) / B;
    m.off[0][i + 1] = m.off[0][i] + (long long)J.row_items * channels;
    m.off[1][i + 1] = m.off[1][i] + (long long)J.col_items * channels;
    m.off[2][i + 1] = m.off[2][i] + (long long)J.row_items * channels;
    m.off[3][i + 1] = m.off[3][i] + gblocks;
  }
  if (smem > kMaxDynSmem) return fail(AIM_EINVAL, "multi-context launch needs too much shared memory");
  auto kernel = k_grid_multi<CT, TPT, LOGE>;
  AIM_TRY(ensure_smem(kernel, smem));
  int dev = 0, sms = 0, per_sm = 0, coop = 0;
  AIM_CUDA_TRY(cudaGetDevice(&dev));
  AIM_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  AIM_CUDA_TRY(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
  if (!coop) return fail(AIM_ECUDA, "device does not support cooperative launches");
  AIM_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, B, smem));
  if (per_sm < 1) return fail(AIM_EINVAL, "multi-context kernel does not fit an SM");
  long long most = 0;
  for (int ph = 0; ph < 4; ++ph) most = std::max(most, m.off[ph][count]);
  const int grid = (int)std::max(1LL, std::min<long long>((long long)sms * per_sm, most));
  AIM_CUDA_TRY(cudaMemsetAsync(scratch, 0, 2 * sizeof(unsigned), st));   // the barrier words (not the error flag)
  {
    // one launch: the three grid passes and the gathers of every job
    ProfScope ps(K_MULTI, st);
    void* params[] = {&m};
    AIM_CUDA_TRY(cudaLaunchCooperativeKernel((const void*)kernel, dim3(grid), dim3(B), params, smem, st));
  }
  return AIM_OK;
}

// Splits the passes into the fewest launches whose contexts can share one CTA size (longest
// transforms first; a context too short for the CTA size of a longer one goes to a later launch).
template <typename CT, int TPT, int LOGE>
static aim_status launch_multi_groups(const MultiPassSpec* passes, int count, unsigned* scratch, int* err_host,
                                      cudaStream_t st) {
  std::vector<int> left(count);
  for (int i = 0; i < count; ++i) left[i] = i;
  std::stable_sort(left.begin(), left.end(), [&](int a, int b) { return passes[a].ctx->H > passes[b].ctx->H; });
  AIM_CUDA_TRY(cudaMemsetAsync(scratch + 2, 0, sizeof(int), st));   // the stage's error flag
  std::vector<MultiPassSpec> group;
  while (!left.empty()) {
    const int B = multi_cta_threads<CT, TPT, LOGE>(passes[left[0]].ctx->H);
    group.clear();
    std::vector<int> rest;
    for (int i : left) {
      if (multi_fits<CT, TPT, LOGE>(B, passes[i].ctx->H)) group.push_back(passes[i]);
      else rest.push_back(i);
    }
    const aim_status gs = launch_multi<CT, TPT, LOGE>(group.data(), (int)group.size(), scratch, st);
    if (gs != AIM_OK) return gs;
    left.swap(rest);
  }
  AIM_CUDA_TRY(cudaMemcpyAsync(err_host, scratch + 2, sizeof(int), cudaMemcpyDeviceToHost, st));
  return AIM_OK;
}

template <typename CT>
aim_status grid_pass_multi(const MultiPassSpec* passes, int count, unsigned* scratch, int* err_host, cudaStream_t st) {
  if (count < 1 || count > kMaxMultiJobs) return fail(AIM_EINVAL, "1 to 32 passes per multi-context launch");
  const int p = precision_of((CT*)nullptr);
  const Schedule sc = passes[0].ctx->sched[p];
  for (int i = 1; i < count; ++i) {
    const Schedule& o = passes[i].ctx->sched[p];
    if (o.tpt != sc.tpt || loge_of(o) != loge_of(sc))
      return fail(AIM_EINVAL, "contexts of one multi-context launch must share the pass geometry of their schedule");
  }
  if constexpr (std::is_same<CT, double2>::value) {
    return launch_multi_groups<CT, 2, 4>(passes, count, scratch, err_host, st);
  } else {
    if (loge_of(sc) == 3) {
      if (sc.tpt == 1) return launch_multi_groups<CT, 1, 3>(passes, count, scratch, err_host, st);
      return launch_multi_groups<CT, 2, 3>(passes, count, scratch, err_host, st);
    }
    if (sc.tpt == 1) return launch_multi_groups<CT, 1, 4>(passes, count, scratch, err_host, st);
    return launch_multi_groups<CT, 2, 4>(passes, count, scratch, err_host, st);
  }
}


template <typename CT>
aim_status grid_product_dense(aim_ctx* ctx, bool filtered, int nrhs, const double2* u, double2* v, void* inter,
                              size_t inter_bytes, cudaStream_t st) {
  const int precision = precision_of((CT*)nullptr);
  if (inter == nullptr || inter_bytes_needed(ctx, nrhs, precision) > inter_bytes)
    return fail(AIM_ESTATE, "grid workspace not reserved for this many grids");
  AIM_CUDA_TRY(cudaMemsetAsync(v, 0, (size_t)nrhs * ctx->m * ctx->m * sizeof(double2), st));
  RowFwdArgs fa{};
  fa.x = u;
  fa.dense = 1;
  fa.n = ctx->n;
  fa.m = ctx->m;
  fa.nrhs = nrhs;
  RowInvArgs ia{};
  ia.dense = 1;
  ia.dense_out = v;
  ia.m = ctx->m;
  ia.n_act = ctx->n_act;
  return launch_three_passes<CT>(ctx, nrhs, filtered, fa, ia, inter, st);
}

}  // namespace aim
