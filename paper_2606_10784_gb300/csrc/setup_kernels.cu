// Device-side setup in FP64: grid kernel samples (Sec. III-A, self term zeroed per Sec. III-C),
// the kernel spectrum F(c_grid) and its circular truncation at alpha (Sec. III-B), the exact
// near-field entries (singular quadrature) minus their AIM counterparts, and plane-wave
// right-hand sides (Sec. II).
#include <algorithm>
#include <cmath>
#include <mutex>

#include "aim_internal.h"
#include "fft.cuh"

namespace aim {

// ------------------------------------------------------------------------------------
// Bessel functions of order zero in FP64
//   x < 8      : CUDA's j0 / y0
//   8 <= x < 25: Miller's backward recurrence for J_n normalised by J0 + 2 sum J_2k = 1
//                (DLMF 10.12.4), Y0 from the Neumann series
//                Y0 = (2/pi)(ln(x/2) + gamma) J0 - (4/pi) sum_k (-1)^k J_2k / k (DLMF 10.8.2)
//   x >= 25    : Hankel's asymptotic expansion (DLMF 10.17.3), 12 terms of P and Q,
//                with cos(x - pi/4) = (cos x + sin x)/sqrt 2 to keep the phase exact
// ------------------------------------------------------------------------------------
__device__ void bessel_j0y0(double x, double* J0, double* Y0) {
  if (x < 8.0) {
    *J0 = j0(x);
    *Y0 = y0(x);
    return;
  }
  if (x < 25.0) {
    const int nstart = 2 * (int)((x + 30.0 + 8.0 * cbrt(x)) * 0.5);
    double jp1 = 0.0, jn = 1.0, s_even = 0.0, neu = 0.0;
    for (int nn = nstart; nn > 0; --nn) {
      const double jm1 = (2.0 * nn / x) * jn - jp1;
      jp1 = jn;
      jn = jm1;                       // J_{nn-1}
      const int kk = nn - 1;
      if (kk > 0 && (kk & 1) == 0) {
        s_even += jn;
        const int half = kk >> 1;
        neu += ((half & 1) ? -jn : jn) / (double)half;
      }
      if (fabs(jn) > 1e100) {
        jn *= 1e-100; jp1 *= 1e-100; s_even *= 1e-100; neu *= 1e-100;
      }
    }
    const double norm = jn + 2.0 * s_even;
    const double j0v = jn / norm;
    *J0 = j0v;
    *Y0 = (2.0 / M_PI) * (log(0.5 * x) + 0.57721566490153286061) * j0v - (4.0 / M_PI) * (neu / norm);
    return;
  }
  // a_k(0) = prod_{j<=k} (-(2j-1)^2) / (k! 8^k)
  double a = 1.0, Pv = 1.0, Qv = 0.0, xp = 1.0;
  for (int kk = 1; kk <= 24; ++kk) {
    a *= -(double)((2 * kk - 1) * (2 * kk - 1)) / (8.0 * kk);
    xp *= x;
    const double term = a / xp;
    // P = sum (-1)^k a_2k / x^2k ; Q = sum (-1)^k a_{2k+1} / x^{2k+1}
    if (kk & 1) Qv += ((kk >> 1) & 1 ? -term : term);
    else Pv += ((kk >> 1) & 1 ? -term : term);
  }
  double sx, cx;
  sincos(x, &sx, &cx);
  const double cw = (cx + sx) * 0.70710678118654752440;   // cos(x - pi/4)
  const double sw = (sx - cx) * 0.70710678118654752440;   // sin(x - pi/4)
  const double amp = sqrt(2.0 / (M_PI * x));
  *J0 = amp * (Pv * cw - Qv * sw);
  *Y0 = amp * (Pv * sw + Qv * cw);
}

// J0 alone, by the same three branches (for the filtered kernel's integrand)
__device__ double bessel_j0(double x) {
  if (x < 8.0) return j0(x);
  if (x < 25.0) {
    const int nstart = 2 * (int)((x + 30.0 + 8.0 * cbrt(x)) * 0.5);
    double jp1 = 0.0, jn = 1.0, s_even = 0.0;
    for (int nn = nstart; nn > 0; --nn) {
      const double jm1 = (2.0 * nn / x) * jn - jp1;
      jp1 = jn;
      jn = jm1;
      const int kk = nn - 1;
      if (kk > 0 && (kk & 1) == 0) s_even += jn;
      if (fabs(jn) > 1e100) {
        jn *= 1e-100; jp1 *= 1e-100; s_even *= 1e-100;
      }
    }
    return jn / (jn + 2.0 * s_even);
  }
  double a = 1.0, Pv = 1.0, Qv = 0.0, xp = 1.0;
  for (int kk = 1; kk <= 24; ++kk) {
    a *= -(double)((2 * kk - 1) * (2 * kk - 1)) / (8.0 * kk);
    xp *= x;
    const double term = a / xp;
    if (kk & 1) Qv += ((kk >> 1) & 1 ? -term : term);
    else Pv += ((kk >> 1) & 1 ? -term : term);
  }
  double sx, cx;
  sincos(x, &sx, &cx);
  const double cw = (cx + sx) * 0.70710678118654752440;
  const double sw = (sx - cx) * 0.70710678118654752440;
  return sqrt(2.0 / (M_PI * x)) * (Pv * cw - Qv * sw);
}

// g(r) = -(j/4) H0^(2)(kr) = -(j/4)(J0 - j Y0) = (-Y0/4, -J0/4)
__device__ __forceinline__ double2 green(double k, double r) {
  double J, Y;
  bessel_j0y0(k * r, &J, &Y);
  return double2{-0.25 * Y, -0.25 * J};
}

// ------------------------------------------------------------------------------------
// grid kernel and spectrum
// ------------------------------------------------------------------------------------
__global__ void k_sample_kernel(double2* samp, int H, double eps, double k) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long total = (long long)(H + 1) * (H + 1);
  if (t >= total) return;
  const int i = (int)(t / (H + 1)), j = (int)(t - (long long)i * (H + 1));
  if (i == 0 && j == 0) {
    samp[t] = double2{0.0, 0.0};     // self term set to zero (Sec. III-C)
    return;
  }
  const double r = eps * sqrt((double)i * i + (double)j * j);
  samp[t] = green(k, r);
}

// In-place transform of the even-symmetric P x P array held as its (H+1) x (H+1) quarter:
// along rows (by_rows = 1) or columns. Each CTA expands one line to length P by mirroring,
// runs a P-point DFT in shared memory, and keeps entries 0..H.
template <int NB>
__global__ void k_even_line_dft(double2* a, int H, int logP, const double2* tw, int by_rows) {
  extern __shared__ __align__(16) unsigned char smraw[];
  double2* sm = reinterpret_cast<double2*>(smraw);
  const int P = 1 << logP;
  const int line = blockIdx.x;
  const size_t stride = by_rows ? 1 : (size_t)(H + 1);
  double2* base = by_rows ? a + (size_t)line * (H + 1) : a + line;
  for (int j = threadIdx.x; j < P; j += blockDim.x) {
    const int jj = j <= H ? j : P - j;
    sm[j] = base[(size_t)jj * stride];
  }
  __syncthreads();
  smem_fft<NB, false>(sm, logP, 1, tw, logP);
  for (int q = threadIdx.x; q <= H; q += blockDim.x) base[(size_t)q * stride] = sm[q];
}

__device__ __forceinline__ float4 split_df(double2 v) {
  const float xh = __double2float_rn(v.x), yh = __double2float_rn(v.y);
  // the double-float order (xh, yh, xl, yl)
  return float4{xh, yh, __double2float_rn(v.x - (double)xh), __double2float_rn(v.y - (double)yh)};
}

// The complex64 and double-float copies of FP64 values, rounded as k_pack_spectrum and the
// near-field kernels round them (a context imported from a setup blob derives them here).
__global__ void k_narrow_copies(const double2* src, long long count, float2* f, float4* df) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= count) return;
  const double2 v = src[t];
  f[t] = float2{(float)v.x, (float)v.y};
  if (df != nullptr) df[t] = split_df(v);
}

aim_status derive_narrow_copies(const double2* src, size_t count, float2* f, float4* df, cudaStream_t st) {
  if (count == 0) return AIM_OK;
  const int tpb = 256;
  {
    ProfScope ps(K_SETUP_PACK, st);
    k_narrow_copies<<<(unsigned)((count + tpb - 1) / tpb), tpb, 0, st>>>(src, (long long)count, f, df);
  }
  AIM_CUDA_TRY(cudaGetLastError());
  return AIM_OK;
}

// live[q'] = 0 when the mask zeroes column q' entirely. kappa(p, q') >= kappa(0, q') holds in
// floating point as well (sqrt is exact on the perfect square q'^2 and monotone, and both are
// scaled by the same factor), so the column has a kept entry exactly when its p = 0 entry is kept.
// CA (may be null): the transform of the analytically filtered samples, which then becomes the
// filtered spectrum as it is (no mask; every column live).
__global__ void k_pack_spectrum(const double2* C, const double2* CA, int H, int P, double eps, double alpha,
                                int filter, double2* specU, double2* specA, float2* specUf, float2* specAf,
                                float4* specUdf, float4* specAdf, int* live) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long total = (long long)(H + 1) * (H + 1);
  if (t >= total) return;
  const int qq = (int)(t / (H + 1)), off = (int)(t - (long long)qq * (H + 1));
  const int half = H >> 1;
  const int p = off <= half ? 2 * off : 2 * (off - half - 1) + 1;
  const double2 v = C[(size_t)p * (H + 1) + qq];
  const double kappa = (2.0 * M_PI / ((double)P * eps)) * sqrt((double)p * p + (double)qq * qq);
  const bool keep = !filter || kappa <= alpha;
  specU[t] = v;
  specUf[t] = float2{(float)v.x, (float)v.y};
  const double2 va = CA != nullptr ? CA[(size_t)p * (H + 1) + qq] : keep ? v : double2{0.0, 0.0};
  specA[t] = va;
  specAf[t] = float2{(float)va.x, (float)va.y};
  specUdf[t] = split_df(v);
  specAdf[t] = split_df(va);
  if (off == 0) live[qq] = (CA != nullptr || keep) ? 1 : 0;   // p = 0
}

// ------------------------------------------------------------------------------------
// quadrature tables (Gauss-Legendre on [0,1])
// ------------------------------------------------------------------------------------
struct QuadTables {
  double x10[10], w10[10], x12[12], w12[12], x16[16], w16[16], x20[20], w20[20], x24[24], w24[24];
};
__constant__ QuadTables c_quad;

// The analytically filtered kernel of Eq. 6 on the grid: samp[i (H+1) + j] = g^alpha(eps sqrt(i^2+j^2)).
// With PV int_0^inf J0(sr) s/(s^2-k^2) ds = -(pi/2) Y0(kr), Eq. 6 becomes
//     g^alpha(r) = -(j/4) J0(kr) + (1/2 pi) PV int_0^alpha J0(sr) s/(s^2-k^2) ds,
// regular at r = 0, so the self term keeps its value (Sec. III-C). The pole at s = k is taken out:
//     PV int = int_0^alpha [J0(sr) s - J0(kr) k]/((s-k)(s+k)) ds + (J0(kr)/2) ln((alpha-k)/(alpha+k)),
// and the smooth remainder runs over panels of [0,k] and [k,alpha] no wider than 8/r (about 1.3
// oscillations of J0(sr)), 20 Gauss-Legendre nodes each (no node falls on s = k). One warp per
// sample: lanes take the nodes in turn and a fixed xor-shuffle tree adds them.
constexpr double kFilterPanelPhase = 8.0;

__global__ void k_sample_filtered_kernel(double2* samp, int H, double eps, double k, double alpha) {
  const long long wid = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  const long long total = (long long)(H + 1) * (H + 1);
  if (wid >= total) return;   // whole warps
  const int i = (int)(wid / (H + 1)), j = (int)(wid - (long long)i * (H + 1));
  const double r = eps * sqrt((double)i * i + (double)j * j);
  const double Jk = bessel_j0(k * r);
  const int n1 = max(1, (int)ceil(k * r / kFilterPanelPhase));
  const int n2 = max(1, (int)ceil((alpha - k) * r / kFilterPanelPhase));
  const double w1 = k / n1, w2 = (alpha - k) / n2;
  const int total_nodes = (n1 + n2) * 20;
  double acc = 0.0;
  for (int q = lane; q < total_nodes; q += 32) {
    const int pan = q / 20, node = q - pan * 20;
    const double a0 = pan < n1 ? pan * w1 : k + (pan - n1) * w2;
    const double w = pan < n1 ? w1 : w2;
    const double sv = a0 + w * c_quad.x20[node];
    const double f = (bessel_j0(sv * r) * sv - Jk * k) / ((sv - k) * (sv + k));
    acc = fma(w * c_quad.w20[node], f, acc);
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
  if (lane == 0) {
    const double pv = acc + 0.5 * Jk * log((alpha - k) / (alpha + k));
    samp[wid] = double2{pv / (2.0 * M_PI), -0.25 * Jk};
  }
}


__device__ __forceinline__ double2 cmadd(double2 acc, double s, double2 g) {
  return double2{fma(s, g.x, acc.x), fma(s, g.y, acc.y)};
}

__device__ double dev_pt_seg(double px, double py, double ax, double ay, double bx, double by) {
  const double ex = bx - ax, ey = by - ay;
  double t = ((px - ax) * ex + (py - ay) * ey) / (ex * ex + ey * ey);
  t = fmin(1.0, fmax(0.0, t));
  return hypot(px - (ax + t * ex), py - (ay + t * ey));
}

__device__ __forceinline__ double2 warp_sum(double2 v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    v.x += __shfl_xor_sync(0xffffffffu, v.x, off);
    v.y += __shfl_xor_sync(0xffffffffu, v.y, off);
  }
  return v;
}

// Integrals I_ab = int_e int_f psi_a(sigma) g psi_b(tau) dl dl' for segment pairs (warp per pair).
// psi_0 = 1 - sigma, psi_1 = sigma.
//  self:     I_ab = h^2 int_0^1 g(h t) Q_ab(t) dt with Q_11 = 2/3 - t + t^3/3,
//            Q_00 = 2((1-t)^3/3 + t (1-t)^2/2), Q_01 = Q_10 = (1 - t^3)/3; t = u^6 (24-pt Gauss in u)
//  adjacent: Duffy split at the shared vertex, radial variable X = u^4 (20 points) x 12 points
//  others:   tensor Gauss, 16 x 16 when closer than 3 max(h), else 10 x 10
__global__ void k_te_segment_pairs(const double2* nodes, int n, double k, const int* pe, const int* pf,
                                   int npairs, double2* out) {
  const int wid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (wid >= npairs) return;
  const int e = pe[wid], f = pf[wid];
  const double2 ve0 = nodes[e], ve1 = nodes[(e + 1) % n];
  const double2 vf0 = nodes[f], vf1 = nodes[(f + 1) % n];
  const double dex = ve1.x - ve0.x, dey = ve1.y - ve0.y, dfx = vf1.x - vf0.x, dfy = vf1.y - vf0.y;
  const double he = hypot(dex, dey), hf = hypot(dfx, dfy);
  double2 acc[2][2] = {{{0, 0}, {0, 0}}, {{0, 0}, {0, 0}}};
  bool transpose = false;
  if (e == f) {
    for (int q = lane; q < 24; q += 32) {
      const double u = c_quad.x24[q];
      const double u2 = u * u, u4 = u2 * u2;
      const double t = u4 * u2;
      const double wt = 6.0 * u4 * u * c_quad.w24[q];
      const double2 g = green(k, he * t);
      const double L = 1.0 - t;
      const double q11 = 2.0 / 3.0 - t + t * t * t / 3.0;
      const double q00 = 2.0 * (L * L * L / 3.0 + 0.5 * t * L * L);
      const double q01 = (1.0 - t * t * t) / 3.0;
      acc[0][0] = cmadd(acc[0][0], wt * q00, g);
      acc[0][1] = cmadd(acc[0][1], wt * q01, g);
      acc[1][0] = cmadd(acc[1][0], wt * q01, g);
      acc[1][1] = cmadd(acc[1][1], wt * q11, g);
    }
  } else {
    const bool next = f == (e + 1) % n;
    const bool prev = e == (f + 1) % n;
    if (next || prev) {
      // orient so that the first segment ends where the second begins
      double ax = dex, ay = dey, bx = dfx, by = dfy;
      if (prev) {
        ax = dfx; ay = dfy; bx = dex; by = dey;
        transpose = true;
      }
      for (int q = lane; q < 2 * 20 * 12; q += 32) {
        const int tri = q / 240, rem = q - tri * 240, ix = rem / 12, iyq = rem - ix * 12;
        const double u = c_quad.x20[ix];
        const double X = u * u * u * u;
        const double wX = 4.0 * u * u * u * c_quad.w20[ix];
        const double Y = c_quad.x12[iyq], wY = c_quad.w12[iyq];
        const double xe = tri == 0 ? X : X * Y;     // distance fraction back along the first segment
        const double ta = tri == 0 ? X * Y : X;     // distance fraction along the second segment
        const double r = hypot(xe * ax + ta * bx, xe * ay + ta * by);
        const double2 g = green(k, r);
        const double jw = X * wX * wY;
        const double se = 1.0 - xe;
        const double pa[2] = {1.0 - se, se}, pb[2] = {1.0 - ta, ta};
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
          for (int b = 0; b < 2; ++b) acc[a][b] = cmadd(acc[a][b], jw * pa[a] * pb[b], g);
      }
    } else {
      const double dist = fmin(fmin(dev_pt_seg(ve0.x, ve0.y, vf0.x, vf0.y, vf1.x, vf1.y),
                                    dev_pt_seg(ve1.x, ve1.y, vf0.x, vf0.y, vf1.x, vf1.y)),
                               fmin(dev_pt_seg(vf0.x, vf0.y, ve0.x, ve0.y, ve1.x, ve1.y),
                                    dev_pt_seg(vf1.x, vf1.y, ve0.x, ve0.y, ve1.x, ve1.y)));
      const bool close = dist < 3.0 * fmax(he, hf);
      const int nq = close ? 16 : 10;
      const double* xs = close ? c_quad.x16 : c_quad.x10;
      const double* ws = close ? c_quad.w16 : c_quad.w10;
      for (int q = lane; q < nq * nq; q += 32) {
        const int a1 = q / nq, b1 = q - a1 * nq;
        const double sg = xs[a1], tg = xs[b1];
        const double rx = (ve0.x + sg * dex) - (vf0.x + tg * dfx);
        const double ry = (ve0.y + sg * dey) - (vf0.y + tg * dfy);
        const double2 g = green(k, hypot(rx, ry));
        const double wgt = ws[a1] * ws[b1];
        const double pa[2] = {1.0 - sg, sg}, pb[2] = {1.0 - tg, tg};
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
          for (int b = 0; b < 2; ++b) acc[a][b] = cmadd(acc[a][b], wgt * pa[a] * pb[b], g);
      }
    }
  }
  double2 res[2][2];
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b) res[a][b] = warp_sum(acc[a][b]);
  if (lane == 0) {
    const double s = he * hf;
    for (int a = 0; a < 2; ++a)
      for (int b = 0; b < 2; ++b) {
        const double2 v = transpose ? res[b][a] : res[a][b];
        out[(size_t)wid * 4 + a * 2 + b] = double2{v.x * s, v.y * s};
      }
  }
}

// AIM entry sum_{a in list i} sum_{b in list j} wi_a wj_b c(pos_a - pos_b) for one warp,
// with c read from the (H+1)^2 quarter of the kernel samples (c(0) = 0).
__device__ __forceinline__ double2 aim_pair_sum(const double2* samp, int H, const int* act_ix, const int* act_iy,
                                                const int* ia, const double* wi, int ni,
                                                const int* ib, const double* wj, int nj, int lane) {
  double2 acc{0.0, 0.0};
  for (int a = lane; a < ni; a += 32) {
    const int xa = act_ix[ia[a]], ya = act_iy[ia[a]];
    double2 inner{0.0, 0.0};
    for (int b = 0; b < nj; ++b) {
      const int dx = abs(xa - act_ix[ib[b]]), dy = abs(ya - act_iy[ib[b]]);
      inner = cmadd(inner, wj[b], samp[(size_t)dy * (H + 1) + dx]);
    }
    acc = cmadd(acc, wi[a], inner);
  }
  return warp_sum(acc);
}

struct TENearArgs {
  const double2* nodes;
  int n;
  double k;
  const int* near_ptr;
  const int* near_col;
  const int* pair_seg_idx;
  const double2* I;
  const double2* samp;
  int H;
  const int* act_ix;
  const int* act_iy;
  const int* ga_ptr;
  const int* ga_act;
  const double* ga_w[4];
  double2* cS;
  double2* cN;
  float2* cSf;
  float2* cNf;
};

__global__ void k_te_near_entries(TENearArgs a) {
  const int wid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  const int nnz = a.near_ptr[a.n];
  if (wid >= nnz) return;
  // row of this entry (binary search in near_ptr)
  int lo = 0, hi = a.n;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (a.near_ptr[mid] <= wid) lo = mid; else hi = mid;
  }
  const int i = lo, j = a.near_col[wid];
  const int n = a.n;
  // AIM entries of the four projections
  double2 A[4];
  const int i0 = a.ga_ptr[i], ni = a.ga_ptr[i + 1] - i0;
  const int j0 = a.ga_ptr[j], nj = a.ga_ptr[j + 1] - j0;
#pragma unroll
  for (int pj = 0; pj < 4; ++pj)
    A[pj] = aim_pair_sum(a.samp, a.H, a.act_ix, a.act_iy, a.ga_act + i0, a.ga_w[pj] + i0, ni,
                         a.ga_act + j0, a.ga_w[pj] + j0, nj, lane);
  if (lane != 0) return;
  // exact entries from the four segment pairs (e, a) x (f, b)
  const int es[4] = {i, i, (i + n - 1) % n, (i + n - 1) % n};
  const int fs[4] = {j, (j + n - 1) % n, j, (j + n - 1) % n};
  const int as[4] = {0, 0, 1, 1}, bs[4] = {0, 1, 0, 1};
  double2 S{0, 0}, N{0, 0};
  for (int c = 0; c < 4; ++c) {
    const double2* I = a.I + (size_t)a.pair_seg_idx[(size_t)wid * 4 + c] * 4;
    const int e = es[c], f = fs[c];
    const double2 ve0 = a.nodes[e], ve1 = a.nodes[(e + 1) % n];
    const double2 vf0 = a.nodes[f], vf1 = a.nodes[(f + 1) % n];
    const double dex = ve1.x - ve0.x, dey = ve1.y - ve0.y, dfx = vf1.x - vf0.x, dfy = vf1.y - vf0.y;
    const double he = hypot(dex, dey), hf = hypot(dfx, dfy);
    // n = (t_y, -t_x): n_e . n_f = t_e . t_f
    const double nn = (dex * dfx + dey * dfy) / (he * hf);
    const double2 Iab = I[as[c] * 2 + bs[c]];
    const double2 J = double2{I[0].x + I[1].x + I[2].x + I[3].x, I[0].y + I[1].y + I[2].y + I[3].y};
    const double dd = ((as[c] ? 1.0 : -1.0) / he) * ((bs[c] ? 1.0 : -1.0) / hf);
    S.x += Iab.x;
    S.y += Iab.y;
    N.x += dd * J.x - a.k * a.k * nn * Iab.x;
    N.y += dd * J.y - a.k * a.k * nn * Iab.y;
  }
  const double k2 = a.k * a.k;
  const double2 cs = double2{S.x - A[0].x, S.y - A[0].y};
  const double2 cn = double2{N.x - (A[1].x - k2 * (A[2].x + A[3].x)), N.y - (A[1].y - k2 * (A[2].y + A[3].y))};
  a.cS[wid] = cs;
  a.cN[wid] = cn;
  a.cSf[wid] = float2{(float)cs.x, (float)cs.y};
  a.cNf[wid] = float2{(float)cn.x, (float)cn.y};
}

struct TMNearArgs {
  const double2* nodes;
  int n;
  double k;
  const int* near_ptr;
  const int* near_col;
  const double2* samp;
  int H;
  const int* act_ix;
  const int* act_iy;
  const int* ga_ptr;
  const int* ga_act;
  const double* ga_w;
  const int* sr_ptr;
  const int* sr_act;
  const double* sr_w;
  double2* cS;
  float2* cSf;
};

// Collocation entry int_{seg j} g(|mid_i - r'|) dl' minus its AIM value (warp per entry).
__global__ void k_tm_near_entries(TMNearArgs a) {
  const int wid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  const int nnz = a.near_ptr[a.n];
  if (wid >= nnz) return;
  int lo = 0, hi = a.n;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (a.near_ptr[mid] <= wid) lo = mid; else hi = mid;
  }
  const int i = lo, j = a.near_col[wid], n = a.n;
  const int i0 = a.ga_ptr[i], ni = a.ga_ptr[i + 1] - i0;
  const int j0 = a.sr_ptr[j], nj = a.sr_ptr[j + 1] - j0;
  const double2 A = aim_pair_sum(a.samp, a.H, a.act_ix, a.act_iy, a.ga_act + i0, a.ga_w + i0, ni,
                                 a.sr_act + j0, a.sr_w + j0, nj, lane);
  const double2 vi0 = a.nodes[i], vi1 = a.nodes[(i + 1) % n];
  const double mx = 0.5 * (vi0.x + vi1.x), my = 0.5 * (vi0.y + vi1.y);
  const double2 vj0 = a.nodes[j], vj1 = a.nodes[(j + 1) % n];
  const double djx = vj1.x - vj0.x, djy = vj1.y - vj0.y, hj = hypot(djx, djy);
  double2 acc{0.0, 0.0};
  if (i == j) {
    // midpoint singularity: two halves of length h/2, t = u^6 toward the midpoint
    for (int q = lane; q < 24; q += 32) {
      const double u = c_quad.x24[q];
      const double u2 = u * u, u4 = u2 * u2;
      const double t = u4 * u2;
      const double wt = 6.0 * u4 * u * c_quad.w24[q];
      acc = cmadd(acc, wt * hj, green(a.k, 0.5 * hj * t));   // 2 halves x (h/2)
    }
  } else {
    const double dist = dev_pt_seg(mx, my, vj0.x, vj0.y, vj1.x, vj1.y);
    const bool close = dist < 3.0 * hj;
    const int nq = close ? 16 : 10;
    const double* xs = close ? c_quad.x16 : c_quad.x10;
    const double* ws = close ? c_quad.w16 : c_quad.w10;
    for (int q = lane; q < nq; q += 32) {
      const double rx = mx - (vj0.x + xs[q] * djx), ry = my - (vj0.y + xs[q] * djy);
      acc = cmadd(acc, ws[q] * hj, green(a.k, hypot(rx, ry)));
    }
  }
  acc = warp_sum(acc);
  if (lane == 0) {
    const double2 cs = double2{acc.x - A.x, acc.y - A.y};
    a.cS[wid] = cs;
    a.cSf[wid] = float2{(float)cs.x, (float)cs.y};
  }
}

// ------------------------------------------------------------------------------------
// plane-wave right-hand sides
// ------------------------------------------------------------------------------------
__global__ void k_rhs(const double2* nodes, int n, int te, double k, const double* angles, int nrhs, double2* out) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * nrhs) return;
  const int r = t / n, i = t - r * n;
  double sa, ca;
  sincos(angles[r], &sa, &ca);
  if (!te) {
    const double2 v0 = nodes[i], v1 = nodes[(i + 1) % n];
    const double ph = k * (ca * 0.5 * (v0.x + v1.x) + sa * 0.5 * (v0.y + v1.y));
    double s, c;
    sincos(ph, &s, &c);
    out[t] = double2{c, -s};
    return;
  }
  // E_i = jk sum_pieces h_e sum_u w_u psi(xi_u) exp(-jk khat.r_u) (khat_x t_y - khat_y t_x)
  double re = 0.0, im = 0.0;
  for (int pc = 0; pc < 2; ++pc) {
    const int e = pc == 0 ? i : (i + n - 1) % n;
    const double2 v0 = nodes[e], v1 = nodes[(e + 1) % n];
    const double dx = v1.x - v0.x, dy = v1.y - v0.y, h = hypot(dx, dy);
    const double proj = (ca * dy - sa * dx) / h;
    for (int u = 0; u < 10; ++u) {
      const double xi = c_quad.x10[u];
      const double psi = pc == 0 ? 1.0 - xi : xi;
      const double ph = k * (ca * (v0.x + xi * dx) + sa * (v0.y + xi * dy));
      double s, c;
      sincos(ph, &s, &c);
      const double wgt = c_quad.w10[u] * psi * h * proj;
      re += wgt * c;
      im -= wgt * s;
    }
  }
  // multiply by jk
  out[t] = double2{-k * im, k * re};
}

// ------------------------------------------------------------------------------------
// host orchestration
// ------------------------------------------------------------------------------------
// The quadrature tables live in constant memory, one copy per device: uploaded on the first
// setup on each device (guarded, so concurrent setups on several threads do it once).
static aim_status upload_quad_tables() {
  static std::mutex mu;
  static bool done[64] = {};
  int dev = 0;
  AIM_CUDA_TRY(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(mu);
  if (dev >= 0 && dev < 64 && done[dev]) return AIM_OK;
  QuadTables qt;
  std::vector<double> x, w;
  auto fill = [&](int nq, double* xs, double* ws) {
    gauss_legendre01(nq, &x, &w);
    for (int i = 0; i < nq; ++i) { xs[i] = x[i]; ws[i] = w[i]; }
  };
  fill(10, qt.x10, qt.w10);
  fill(12, qt.x12, qt.w12);
  fill(16, qt.x16, qt.w16);
  fill(20, qt.x20, qt.w20);
  fill(24, qt.x24, qt.w24);
  AIM_CUDA_TRY(cudaMemcpyToSymbol(c_quad, &qt, sizeof(qt)));
  if (dev >= 0 && dev < 64) done[dev] = true;
  return AIM_OK;
}

struct DeviceTemp {
  std::vector<void*> ptrs;
  ~DeviceTemp() {
    for (void* p : ptrs) cudaFree(p);
  }
  template <typename T>
  aim_status alloc(T** p, size_t count) {
    void* q = nullptr;
    cudaError_t e = cudaMalloc(&q, std::max<size_t>(count, 1) * sizeof(T));
    if (e != cudaSuccess) return fail(AIM_ENOMEM, std::string("setup temporary: ") + cudaGetErrorString(e));
    ptrs.push_back(q);
    *p = static_cast<T*>(q);
    return AIM_OK;
  }
  template <typename T>
  aim_status up(T** p, const std::vector<T>& h, cudaStream_t st) {
    AIM_TRY(alloc(p, h.size()));
    if (!h.empty()) AIM_CUDA_TRY(cudaMemcpyAsync(*p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, st));
    return AIM_OK;
  }
};

// In-place 2-D DFT of an even-symmetric P x P array held as its (H+1) x (H+1) quarter.
static aim_status even_dft_2d(aim_ctx* ctx, double2* a, cudaStream_t st) {
  const int H = ctx->H, P = ctx->P;
  const size_t sm = (size_t)P * sizeof(double2);
  constexpr int NB = 4;
  const int th = std::max(64, std::min(1024, (P / 4 + NB - 1) / NB));
  if (sm > 48 * 1024)
    AIM_CUDA_TRY(cudaFuncSetAttribute(k_even_line_dft<NB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
  for (int by_rows = 1; by_rows >= 0; --by_rows) {
    {
      ProfScope ps(K_SETUP_DFT, st);
      k_even_line_dft<NB><<<H + 1, th, sm, st>>>(a, H, ctx->logP, ctx->tw, by_rows);
    }
    AIM_CUDA_TRY(cudaGetLastError());
  }
  return AIM_OK;
}

// g^alpha of Eq. 6 at the grid offsets (i, j), i, j = 0..H, into `out` ((H+1)^2, device).
aim_status analytic_samples(aim_ctx* ctx, double2* out, cudaStream_t st) {
  if (!(ctx->alpha > ctx->k)) return fail(AIM_ESTATE, "the analytic filter needs alpha > k (set up with a filter)");
  AIM_TRY(upload_quad_tables());
  const long long total = (long long)(ctx->H + 1) * (ctx->H + 1);
  const int tpb = 256;
  const long long blocks = (total * 32 + tpb - 1) / tpb;
  {
    ProfScope ps(K_SETUP_SAMPLE, st);
    k_sample_filtered_kernel<<<(unsigned)blocks, tpb, 0, st>>>(out, ctx->H, ctx->eps, ctx->k, ctx->alpha);
  }
  AIM_CUDA_TRY(cudaGetLastError());
  return AIM_OK;
}

// Natural-order quarter F[p][q], p, q = 0..H, of a packed spectrum (per column q: even rows, then odd rows).
__global__ void k_unpack_spectrum(const double2* packed, int H, double2* out) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long total = (long long)(H + 1) * (H + 1);
  if (t >= total) return;
  const int p = (int)(t / (H + 1)), q = (int)(t - (long long)p * (H + 1));
  const int half = H >> 1;
  const int off = (p & 1) ? half + 1 + (p >> 1) : (p >> 1);
  out[t] = packed[(size_t)q * (H + 1) + off];
}

aim_status kernel_table(aim_ctx* ctx, int which, double2* out, cudaStream_t st) {
  const int H = ctx->H;
  const long long total = (long long)(H + 1) * (H + 1);
  const int tpb = 256;
  switch (which) {
    case AIM_TABLE_SPECTRUM:
    case AIM_TABLE_SPECTRUM_FILTERED: {
      const double2* src = which == AIM_TABLE_SPECTRUM ? ctx->specU : ctx->specA;
      {
        ProfScope ps(K_SETUP_PACK, st);
        k_unpack_spectrum<<<(unsigned)((total + tpb - 1) / tpb), tpb, 0, st>>>(src, H, out);
      }
      AIM_CUDA_TRY(cudaGetLastError());
      return AIM_OK;
    }
    case AIM_TABLE_ANALYTIC_SAMPLES:
      return analytic_samples(ctx, out, st);
    case AIM_TABLE_ANALYTIC_SPECTRUM:
      AIM_TRY(analytic_samples(ctx, out, st));
      return even_dft_2d(ctx, out, st);
    default:
      return fail(AIM_EINVAL, "unknown kernel table");
  }
}

// Builds spectra and the near field. The kernel samples are needed by both: the near-field
// AIM entries read them first, then the spectrum transform overwrites them in place.
aim_status device_spectra_and_near(aim_ctx* ctx, const HostSetup& hs, cudaStream_t st) {
  AIM_TRY(upload_quad_tables());
  DeviceTemp tmp;
  const int H = ctx->H, P = ctx->P;
  const size_t nq = (size_t)(H + 1) * (H + 1);
  double2* samp = nullptr;
  AIM_TRY(tmp.alloc(&samp, nq));
  {
    const int tpb = 256;
    ProfScope ps(K_SETUP_SAMPLE, st);
    k_sample_kernel<<<(unsigned)((nq + tpb - 1) / tpb), tpb, 0, st>>>(samp, H, ctx->eps, ctx->k);
    AIM_CUDA_TRY(cudaGetLastError());
  }

  // ---- near field
  const long long nnz = hs.near_ptr.empty() ? 0 : hs.near_ptr.back();
  ctx->near.nnz = nnz;
  ctx->nnz_near = nnz;
  if (nnz > 0) {
    AIM_TRY(upload(ctx, &ctx->near.ptr, hs.near_ptr, st));
    AIM_TRY(upload(ctx, &ctx->near.col, hs.near_col, st));
    int* act_iy = nullptr;
    AIM_TRY(tmp.up(&act_iy, hs.act_iy, st));
    const int nvals = ctx->form == AIM_TE_P1_GALERKIN ? 2 : 1;
    for (int v = 0; v < nvals; ++v) {
      AIM_TRY(dev_alloc_t(ctx, &ctx->near.val[v], (size_t)nnz));
      AIM_TRY(dev_alloc_t(ctx, &ctx->near.valf[v], (size_t)nnz));
    }
    const int tpb = 256, wpb = tpb / 32;
    if (ctx->form == AIM_TE_P1_GALERKIN) {
      int *pe = nullptr, *pf = nullptr, *psi = nullptr;
      double2* I = nullptr;
      AIM_TRY(tmp.up(&pe, hs.seg_e, st));
      AIM_TRY(tmp.up(&pf, hs.seg_f, st));
      AIM_TRY(tmp.up(&psi, hs.pair_seg_idx, st));
      const int npairs = (int)hs.seg_e.size();
      AIM_TRY(tmp.alloc(&I, (size_t)npairs * 4));
      {
        ProfScope ps(K_SETUP_SEGPAIRS, st);
        k_te_segment_pairs<<<(npairs + wpb - 1) / wpb, tpb, 0, st>>>(ctx->nodes, ctx->n, ctx->k, pe, pf, npairs, I);
      }
      AIM_CUDA_TRY(cudaGetLastError());
      TENearArgs a{};
      a.nodes = ctx->nodes;
      a.n = ctx->n;
      a.k = ctx->k;
      a.near_ptr = ctx->near.ptr;
      a.near_col = ctx->near.col;
      a.pair_seg_idx = psi;
      a.I = I;
      a.samp = samp;
      a.H = H;
      a.act_ix = ctx->act_ix;
      a.act_iy = act_iy;
      a.ga_ptr = ctx->prj.ga_ptr;
      a.ga_act = ctx->prj.ga_act;
      for (int q = 0; q < 4; ++q) a.ga_w[q] = ctx->prj.ga_w[q];
      a.cS = ctx->near.val[0];
      a.cN = ctx->near.val[1];
      a.cSf = ctx->near.valf[0];
      a.cNf = ctx->near.valf[1];
      ProfScope ps(K_SETUP_NEAR, st);
      k_te_near_entries<<<(unsigned)((nnz + wpb - 1) / wpb), tpb, 0, st>>>(a);
      AIM_CUDA_TRY(cudaGetLastError());
    } else {
      int *sr_ptr = nullptr, *sr_act = nullptr;
      double* sr_w = nullptr;
      AIM_TRY(tmp.up(&sr_ptr, hs.sr_ptr, st));
      AIM_TRY(tmp.up(&sr_act, hs.sr_act, st));
      AIM_TRY(tmp.up(&sr_w, hs.sr_w, st));
      TMNearArgs a{};
      a.nodes = ctx->nodes;
      a.n = ctx->n;
      a.k = ctx->k;
      a.near_ptr = ctx->near.ptr;
      a.near_col = ctx->near.col;
      a.samp = samp;
      a.H = H;
      a.act_ix = ctx->act_ix;
      a.act_iy = act_iy;
      a.ga_ptr = ctx->prj.ga_ptr;
      a.ga_act = ctx->prj.ga_act;
      a.ga_w = ctx->prj.ga_w[0];
      a.sr_ptr = sr_ptr;
      a.sr_act = sr_act;
      a.sr_w = sr_w;
      a.cS = ctx->near.val[0];
      a.cSf = ctx->near.valf[0];
      ProfScope ps(K_SETUP_NEAR, st);
      k_tm_near_entries<<<(unsigned)((nnz + wpb - 1) / wpb), tpb, 0, st>>>(a);
      AIM_CUDA_TRY(cudaGetLastError());
    }
  }

  // ---- spectrum: even-symmetric 2-D DFT of the samples, in place, then pack + mask
  AIM_TRY(even_dft_2d(ctx, samp, st));
  // the analytically filtered kernel (Eq. 6) sampled on the grid and transformed, when asked for
  double2* sampA = nullptr;
  if (ctx->filter_enabled == AIM_FILTER_ANALYTIC) {
    AIM_TRY(tmp.alloc(&sampA, nq));
    AIM_TRY(analytic_samples(ctx, sampA, st));
    AIM_TRY(even_dft_2d(ctx, sampA, st));
  }
  AIM_TRY(dev_alloc_t(ctx, &ctx->specU, nq));
  AIM_TRY(dev_alloc_t(ctx, &ctx->specA, nq));
  AIM_TRY(dev_alloc_t(ctx, &ctx->specUf, nq));
  AIM_TRY(dev_alloc_t(ctx, &ctx->specAf, nq));
  AIM_TRY(dev_alloc_t(ctx, &ctx->specUdf, nq));
  AIM_TRY(dev_alloc_t(ctx, &ctx->specAdf, nq));
  AIM_TRY(dev_alloc_t(ctx, &ctx->specA_live, (size_t)H + 1));
  {
    const int tpb = 256;
    ProfScope ps(K_SETUP_PACK, st);
    k_pack_spectrum<<<(unsigned)((nq + tpb - 1) / tpb), tpb, 0, st>>>(samp, sampA, H, P, ctx->eps, ctx->alpha,
                                                                      ctx->filter_enabled, ctx->specU, ctx->specA,
                                                                      ctx->specUf, ctx->specAf, ctx->specUdf,
                                                                      ctx->specAdf, ctx->specA_live);
    AIM_CUDA_TRY(cudaGetLastError());
  }
  // temporaries are freed when `tmp` goes out of scope: wait for the kernels first
  AIM_CUDA_TRY(cudaStreamSynchronize(st));
  return AIM_OK;
}

aim_status device_rhs_planewave(aim_ctx* ctx, int nrhs, const double* angles_dev, double2* out, cudaStream_t st) {
  const int total = ctx->n * nrhs;
  ProfScope ps(K_RHS, st);
  k_rhs<<<(total + 255) / 256, 256, 0, st>>>(ctx->nodes, ctx->n, ctx->form == AIM_TE_P1_GALERKIN, ctx->k,
                                             angles_dev, nrhs, out);
  AIM_CUDA_TRY(cudaGetLastError());
  return AIM_OK;
}

}  // namespace aim
