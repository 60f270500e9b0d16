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
//               grid points the test projection reads (the restriction [.]_restr).
//   k_gather    y_i = sum over projections of coef * (P_t^T v)_i plus the near-field row
//               (C x)_i, one warp per unknown, deterministic.
// The intermediate m x P grid of a channel is stored as column tiles of W entries
// (W * sizeof(complex) = 32 bytes) so that the column pass reads contiguous blocks and the
// row passes touch whole 32-byte sectors. Only grid rows that hold active points are stored.
#include "aim_internal.h"
#include "fft.cuh"

namespace aim {

template <typename T> using C2 = typename Cplx<T>::type;

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
};

template <typename T, int NB>
__global__ void __launch_bounds__(1024) k_row_fwd(RowFwdArgs a) {
  using T2 = C2<T>;
  constexpr int W = TileW<T>::value;
  extern __shared__ __align__(16) unsigned char smraw[];
  T2* sm = reinterpret_cast<T2*>(smraw);
  const int H = 1 << a.logH, P = 1 << a.logP;
  const int rloc = blockIdx.x, iy = a.row_lo + rloc, c = blockIdx.y;
  const T2* tw = static_cast<const T2*>(a.tw);
  for (int i = threadIdx.x; i < 2 * H; i += blockDim.x) sm[i] = T2{0, 0};
  __syncthreads();
  if (a.dense) {
    const double2* u = a.x + (size_t)c * a.m * a.m + (size_t)iy * a.m;
    for (int ix = threadIdx.x; ix < a.m; ix += blockDim.x) {
      const double2 v = u[ix];
      sm[ix] = T2{(T)v.x, (T)v.y};
    }
  } else {
    const int pj = c / a.nrhs, r = c - pj * a.nrhs;
    const double* w = a.w[pj];
    const double2* xv = a.x + (size_t)r * a.n;
    const int a1 = a.row_ptr[iy + 1];
    for (int ap = a.row_ptr[iy] + threadIdx.x; ap < a1; ap += blockDim.x) {
      double re = 0.0, im = 0.0;
      const int e1 = a.sc_ptr[ap + 1];
      for (int e = a.sc_ptr[ap]; e < e1; ++e) {
        const double ww = w[e];
        const double2 xx = xv[a.sc_col[e]];
        re = fma(ww, xx.x, re);
        im = fma(ww, xx.y, im);
      }
      sm[a.act_ix[ap]] = T2{(T)re, (T)im};
    }
  }
  __syncthreads();
  for (int nn = threadIdx.x; nn < H; nn += blockDim.x) sm[H + nn] = cmul(sm[nn], tw[nn]);
  __syncthreads();
  smem_fft<NB, false>(sm, a.logH, 2, tw, a.logP);
  T2* out = static_cast<T2*>(a.inter) + (size_t)c * P * a.nrows;
  for (int q = threadIdx.x; q < P; q += blockDim.x) {
    const T2 val = (q & 1) ? sm[H + (q >> 1)] : sm[q >> 1];
    out[((size_t)(q / W) * a.nrows + rloc) * W + (q % W)] = val;
  }
}

struct ColArgs {
  void* inter;
  const void* spec;
  const void* tw;
  int logH, logP, row_lo, nrows;
};

template <typename T, int NB>
__global__ void __launch_bounds__(1024) k_col_conv(ColArgs a) {
  using T2 = C2<T>;
  constexpr int W = TileW<T>::value;
  extern __shared__ __align__(16) unsigned char smraw[];
  T2* sm = reinterpret_cast<T2*>(smraw);   // [w][half][H]
  const int H = 1 << a.logH, P = 1 << a.logP;
  const int qt = blockIdx.x, c = blockIdx.y;
  const T2* tw = static_cast<const T2*>(a.tw);
  T2* blk = static_cast<T2*>(a.inter) + (size_t)c * P * a.nrows + (size_t)qt * a.nrows * W;
  for (int i = threadIdx.x; i < 2 * W * H; i += blockDim.x) sm[i] = T2{0, 0};
  __syncthreads();
  for (int idx = threadIdx.x; idx < a.nrows * W; idx += blockDim.x) {
    const int row = idx / W, w = idx - row * W;
    sm[(2 * w) * H + a.row_lo + row] = blk[idx];
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < W * a.nrows; idx += blockDim.x) {
    const int w = idx / a.nrows, nn = a.row_lo + (idx - w * a.nrows);
    sm[(2 * w + 1) * H + nn] = cmul(sm[(2 * w) * H + nn], tw[nn]);
  }
  __syncthreads();
  smem_fft<NB, false>(sm, a.logH, 2 * W, tw, a.logP);
  const T2* spec = static_cast<const T2*>(a.spec);
  const int half_h = H >> 1;
  for (int idx = threadIdx.x; idx < 2 * W * H; idx += blockDim.x) {
    const int f = idx >> a.logH, kk = idx & (H - 1);
    const int q = qt * W + (f >> 1);
    const int qq = min(q, P - q);
    const T2* col = spec + (size_t)qq * (H + 1);
    const T2 s = (f & 1) ? col[half_h + 1 + min(kk, H - 1 - kk)] : col[min(kk, H - kk)];
    sm[idx] = cmul(sm[idx], s);
  }
  __syncthreads();
  smem_fft<NB, true>(sm, a.logH, 2 * W, tw, a.logP);
  for (int idx = threadIdx.x; idx < a.nrows * W; idx += blockDim.x) {
    const int row = idx / W, w = idx - row * W;
    const int nn = a.row_lo + row;
    blk[idx] = cadd(sm[(2 * w) * H + nn], cmulc(sm[(2 * w + 1) * H + nn], tw[nn]));
  }
}

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
};

template <typename T, int NB>
__global__ void __launch_bounds__(1024) k_row_inv(RowInvArgs a) {
  using T2 = C2<T>;
  constexpr int W = TileW<T>::value;
  extern __shared__ __align__(16) unsigned char smraw[];
  T2* sm = reinterpret_cast<T2*>(smraw);
  const int H = 1 << a.logH, P = 1 << a.logP;
  const int rloc = blockIdx.x, iy = a.row_lo + rloc, c = blockIdx.y;
  const T2* tw = static_cast<const T2*>(a.tw);
  const T2* blk = static_cast<const T2*>(a.inter) + (size_t)c * P * a.nrows;
  for (int q = threadIdx.x; q < P; q += blockDim.x)
    sm[(q & 1) * H + (q >> 1)] = blk[((size_t)(q / W) * a.nrows + rloc) * W + (q % W)];
  __syncthreads();
  smem_fft<NB, true>(sm, a.logH, 2, tw, a.logP);
  const T sc = (T)a.scale;
  if (a.dense) {
    double2* out = a.dense_out + (size_t)c * a.m * a.m + (size_t)iy * a.m;
    for (int ix = threadIdx.x; ix < a.m; ix += blockDim.x) {
      const T2 v = cadd(sm[ix], cmulc(sm[H + ix], tw[ix]));
      out[ix] = double2{(double)(v.x * sc), (double)(v.y * sc)};
    }
  } else {
    T2* out = static_cast<T2*>(a.vact) + (size_t)c * a.n_act;
    const int a1 = a.row_ptr[iy + 1];
    for (int ap = a.row_ptr[iy] + threadIdx.x; ap < a1; ap += blockDim.x) {
      const int ix = a.act_ix[ap];
      const T2 v = cadd(sm[ix], cmulc(sm[H + ix], tw[ix]));
      out[ap] = T2{v.x * sc, v.y * sc};
    }
  }
}

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

template <typename T>
__global__ void k_gather(GatherArgs a) {
  using T2 = C2<T>;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (gw >= a.n * a.nrhs) return;
  const int r = gw / a.n, i = gw - r * a.n;
  double re = 0.0, im = 0.0;
  const int e0 = a.ga_ptr[i], e1 = a.ga_ptr[i + 1];
  for (int pj = 0; pj < a.nproj; ++pj) {
    const T2* v = static_cast<const T2*>(a.vact) + (size_t)(pj * a.nrhs + r) * a.n_act;
    const double* w = a.w[pj];
    double cr = 0.0, ci = 0.0;
    for (int e = e0 + lane; e < e1; e += 32) {
      const double ww = w[e];
      const T2 val = v[a.ga_act[e]];
      cr = fma(ww, (double)val.x, cr);
      ci = fma(ww, (double)val.y, ci);
    }
    re += a.coef[pj].x * cr - a.coef[pj].y * ci;
    im += a.coef[pj].x * ci + a.coef[pj].y * cr;
  }
  if (a.nptr != nullptr) {
    const T2* val = static_cast<const T2*>(a.nval);
    const double2* xv = a.x + (size_t)r * a.n;
    const int n1 = a.nptr[i + 1];
    for (int e = a.nptr[i] + lane; e < n1; e += 32) {
      const T2 cv = val[e];
      const double2 xx = xv[a.ncol[e]];
      re += (double)cv.x * xx.x - (double)cv.y * xx.y;
      im += (double)cv.x * xx.y + (double)cv.y * xx.x;
    }
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    re += __shfl_xor_sync(0xffffffffu, re, off);
    im += __shfl_xor_sync(0xffffffffu, im, off);
  }
  if (lane == 0) {
    const double2 s = a.out_scale;
    double2 o = double2{s.x * re - s.y * im, s.x * im + s.y * re};
    double2* dst = a.y + (size_t)r * a.n + i;
    if (a.accumulate) {
      const double2 prev = *dst;
      o.x += prev.x;
      o.y += prev.y;
    }
    *dst = o;
  }
}

__global__ void k_gram_inv(const double* __restrict__ gi, int blo, int cnt, int n, int nrhs,
                           const double2* __restrict__ x, double2* __restrict__ y) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * nrhs) return;
  const int r = t / n, i = t - r * n;
  const double* row = gi + (size_t)i * cnt;
  const double2* xv = x + (size_t)r * n;
  double re = 0.0, im = 0.0;
  int j = i - blo;
  if (j < 0) j += n;
  for (int d = 0; d < cnt; ++d) {
    const double g = row[d];
    const double2 xx = xv[j];
    re = fma(g, xx.x, re);
    im = fma(g, xx.y, im);
    if (++j == n) j = 0;
  }
  y[t] = double2{re, im};
}

// ------------------------------------------------------------------------------------
// launch configuration
// ------------------------------------------------------------------------------------
template <typename T> struct Cfg;
template <> struct Cfg<double> { static constexpr int NB_ROW = 4, NB_COL = 4; };
template <> struct Cfg<float> { static constexpr int NB_ROW = 4, NB_COL = 8; };

static int threads_for(int butterflies, int nb) {
  int t = (butterflies + nb - 1) / nb;
  t = (t + 31) / 32 * 32;
  if (t < 64) t = 64;
  if (t > 1024) t = 1024;
  return t;
}

template <typename K>
static aim_status ensure_smem(K kernel, size_t bytes) {
  if (bytes > 48 * 1024) {
    AIM_CUDA_TRY(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
  }
  return AIM_OK;
}

size_t inter_bytes_needed(const aim_ctx* ctx, int channels, int precision) {
  const size_t el = precision == AIM_MIXED ? sizeof(float2) : sizeof(double2);
  return (size_t)channels * ctx->P * ctx->nrows * el;
}

template <typename T>
static aim_status launch_three_passes(aim_ctx* ctx, int channels, bool filtered, RowFwdArgs fa, RowInvArgs ia,
                                      cudaStream_t st) {
  using T2 = C2<T>;
  constexpr int W = TileW<T>::value;
  const int H = ctx->H;
  const T2* tw = std::is_same<T, double>::value ? (const T2*)ctx->tw : (const T2*)ctx->twf;
  const void* spec;
  if (std::is_same<T, double>::value) spec = filtered ? (const void*)ctx->specA : (const void*)ctx->specU;
  else spec = filtered ? (const void*)ctx->specAf : (const void*)ctx->specUf;
  if (channels > 65535) return fail(AIM_EINVAL, "too many channels in one grid pass");

  // row forward
  fa.tw = tw;
  fa.logH = ctx->logH;
  fa.logP = ctx->logP;
  fa.row_lo = ctx->row_lo;
  fa.nrows = ctx->nrows;
  fa.inter = ctx->inter;
  const size_t sm_row = 2 * (size_t)H * sizeof(T2);
  const int th_row = threads_for(H / 2, Cfg<T>::NB_ROW);
  AIM_TRY(ensure_smem(k_row_fwd<T, Cfg<T>::NB_ROW>, sm_row));
  {
    ProfScope ps(K_ROW_FWD, st);
    k_row_fwd<T, Cfg<T>::NB_ROW><<<dim3(ctx->nrows, channels), th_row, sm_row, st>>>(fa);
  }
  AIM_CUDA_TRY(cudaGetLastError());

  // column pass
  ColArgs ca;
  ca.inter = ctx->inter;
  ca.spec = spec;
  ca.tw = tw;
  ca.logH = ctx->logH;
  ca.logP = ctx->logP;
  ca.row_lo = ctx->row_lo;
  ca.nrows = ctx->nrows;
  const size_t sm_col = 2 * (size_t)W * H * sizeof(T2);
  const int th_col = threads_for(W * H / 2, Cfg<T>::NB_COL);
  AIM_TRY(ensure_smem(k_col_conv<T, Cfg<T>::NB_COL>, sm_col));
  {
    ProfScope ps(K_COL_CONV, st);
    k_col_conv<T, Cfg<T>::NB_COL><<<dim3(ctx->P / W, channels), th_col, sm_col, st>>>(ca);
  }
  AIM_CUDA_TRY(cudaGetLastError());

  // row inverse
  ia.inter = ctx->inter;
  ia.tw = tw;
  ia.logH = ctx->logH;
  ia.logP = ctx->logP;
  ia.row_lo = ctx->row_lo;
  ia.nrows = ctx->nrows;
  ia.scale = 1.0 / ((double)ctx->P * (double)ctx->P);
  AIM_TRY(ensure_smem(k_row_inv<T, Cfg<T>::NB_ROW>, sm_row));
  {
    ProfScope ps(K_ROW_INV, st);
    k_row_inv<T, Cfg<T>::NB_ROW><<<dim3(ctx->nrows, channels), th_row, sm_row, st>>>(ia);
  }
  AIM_CUDA_TRY(cudaGetLastError());
  return AIM_OK;
}

template <typename T>
aim_status grid_pass(aim_ctx* ctx, const PassSpec& spec, int nrhs, const double2* x, double2* y,
                     cudaStream_t st) {
  const int precision = std::is_same<T, double>::value ? AIM_FP64 : AIM_MIXED;
  const int channels = spec.nproj * nrhs;
  if (inter_bytes_needed(ctx, channels, precision) > ctx->inter_bytes ||
      (size_t)channels * ctx->n_act * sizeof(C2<T>) > ctx->vact_bytes)
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
  AIM_TRY(launch_three_passes<T>(ctx, channels, spec.filtered, fa, ia, st));

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
    ga.nval = std::is_same<T, double>::value ? (const void*)spec.near->val[spec.near_which]
                                              : (const void*)spec.near->valf[spec.near_which];
  }
  ga.x = x;
  ga.out_scale = spec.out_scale;
  ga.y = y;
  ga.accumulate = 0;
  const long long warps = (long long)ctx->n * nrhs;
  const int tpb = 256;
  const long long blocks = (warps * 32 + tpb - 1) / tpb;
  {
    ProfScope ps(K_GATHER, st);
    k_gather<T><<<(unsigned)blocks, tpb, 0, st>>>(ga);
  }
  AIM_CUDA_TRY(cudaGetLastError());
  return AIM_OK;
}

template <typename T>
aim_status grid_product_dense(aim_ctx* ctx, bool filtered, int nrhs, const double2* u, double2* v,
                              cudaStream_t st) {
  const int precision = std::is_same<T, double>::value ? AIM_FP64 : AIM_MIXED;
  if (inter_bytes_needed(ctx, nrhs, precision) > ctx->inter_bytes)
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
  return launch_three_passes<T>(ctx, nrhs, filtered, fa, ia, st);
}

aim_status gram_inv_apply(aim_ctx* ctx, int nrhs, const double2* x, double2* y, cudaStream_t st) {
  if (ctx->gram_inv == nullptr) return fail(AIM_ESTATE, "no Gram matrix on a TM context");
  const int blo = ctx->gram_band;
  const int cnt = (blo * 2 + 1 <= ctx->n) ? 2 * blo + 1 : ctx->n;
  const int total = ctx->n * nrhs;
  {
    ProfScope ps(K_GRAM, st);
    k_gram_inv<<<(total + 255) / 256, 256, 0, st>>>(ctx->gram_inv, blo, cnt, ctx->n, nrhs, x, y);
  }
  AIM_CUDA_TRY(cudaGetLastError());
  return AIM_OK;
}

template aim_status grid_pass<double>(aim_ctx*, const PassSpec&, int, const double2*, double2*, cudaStream_t);
template aim_status grid_pass<float>(aim_ctx*, const PassSpec&, int, const double2*, double2*, cudaStream_t);
template aim_status grid_product_dense<double>(aim_ctx*, bool, int, const double2*, double2*, cudaStream_t);
template aim_status grid_product_dense<float>(aim_ctx*, bool, int, const double2*, double2*, cudaStream_t);

}  // namespace aim
