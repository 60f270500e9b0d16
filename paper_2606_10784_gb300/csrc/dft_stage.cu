// Radix-16 DFT stage on CUDA cores and on tensor cores: a measurement beside the product.
//
// The grid product's transforms (Eq. 8 / Eq. 10) run as register-resident radix-16/8 passes on
// the FP32 pipe. A batch of DFT-16s can instead be written as a dense contraction: with each
// complex input split into its real and imaginary parts, the DFT-16 of a column is the 32 x 32
// real matrix
//     A = [  C  S ]     C[k][i] = cos(2 pi k i/16),  S[k][i] = sin(2 pi k i/16)
//         [ -S  C ]
// times the column's 32 reals, so a batch of n columns is one (32 x 32) x (32 x n) product that
// tensor cores execute. These kernels run one pass of the transforms -- twiddle, DFT-16, exchange
// through shared memory -- in four variants, on data that stays in shared memory for many passes,
// so that the stage's own throughput is measured, not HBM:
//   variant 0: the product's register butterfly (dft_reg<16>) with paired FP32 complex products;
//   variant 1: mma.sync m16n8k8 with TF32 operands, one product per term: the FP32 data go in as
//              they are and the tensor core reads their top 19 bits (about 2^-10 relative error
//              per operand: far from the complex64 grid's accuracy);
//   variant 2: the same with the data split in two parts, hi = the top 19 bits (a mask) and
//              lo = x - hi (exact), and the products a_hi b_hi + a_hi b_lo + a_lo b_hi (three
//              products, close to FP32 accuracy); the DFT matrix is split once, with rounding;
//   variant 3: variant 2's data path without the products: the loads, twiddles and split of the
//              data and the stores, with hi + lo written back in place of the DFT (output =
//              t(c, i) x_i(c) at value c + 256 i). Its rate bounds any tensor-core pass that
//              feeds the products from registers.
// The pass (the same linear map in every variant; 4096 complex values per CTA):
//   element i of column c is value c + 256 i; output k of column c is value 16 c + k;
//   X_k(c) = sum_i x_i(c) t(c, i) exp(-2 pi j k i/16),  t(c, i) = exp(-2 pi j (c mod 16) i/256)/4.
// The factor 1/4 keeps repeated passes at the inputs' scale. Each thread's twiddles do not change
// from pass to pass, so every variant holds them in registers; the product reads them from the
// twiddle table instead, at the same cost for any butterfly.
#include <cuda_runtime.h>

#include "aim_internal.h"
#include "fft_reg.cuh"

namespace aim {
namespace {

constexpr int kStageThreads = 256;
constexpr int kStageGroup = 4096;          // complex values per CTA (256 columns of 16)
constexpr int kStageBuf = 4096 + 256;      // padded length of one buffer (largest layout)

// Shared-memory placement of value L. Variant 0: one pad element every 16 (the product's
// padding), so a thread's stride-256 reads and its 16 consecutive writes both fall in distinct
// banks. Tensor-core variants: bits 2-3 of L flipped by bits 8-9 xor bits 5-6, so that both the
// fragment-ordered reads (lanes differ in bits 0-1 and 8-9) and writes (bits 0-1 and 5-6) of a
// half-warp's 64-bit accesses fall in 16 distinct bank pairs.
template <int V>
__device__ __forceinline__ int stage_phys(int L) {
  if constexpr (V == 0) return L + (L >> 4);
  else return L ^ ((((L >> 8) ^ (L >> 5)) & 3) << 2);
}

// FP32 to TF32, rounded to nearest (used once per thread for the DFT matrix)
__device__ __forceinline__ unsigned to_tf32(float x) {
  unsigned r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

// The split of a data value: hi keeps the sign, exponent and top 10 mantissa bits (what the
// tensor core reads of an FP32 register), lo = x - hi is exact in FP32.
__device__ __forceinline__ void split_tf32(float x, unsigned& hi, unsigned& lo) {
  hi = __float_as_uint(x) & 0xffffe000u;
  lo = __float_as_uint(x - __uint_as_float(hi));
}

// D += A B, m16n8k8, TF32 inputs, FP32 accumulation (A row-major 16 x 8, B column-major 8 x 8)
__device__ __forceinline__ void mma_tf32(float (&d)[4], const unsigned (&a)[4], unsigned b0, unsigned b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// exp(-2 pi j e/256) for e < 256, one entry per thread, rounded once from FP64 (shared memory)
__device__ __forceinline__ void fill_unit_roots(float2* tab) {
  double s, c;
  sincospi((double)threadIdx.x / 128.0, &s, &c);
  tab[threadIdx.x] = make_float2((float)c, (float)-s);
}

// Entry (row rho, column kappa) of the 32 x 32 real DFT-16 matrix A above, from the table of
// roots: cos and sin of 2 pi k i/16 are the real part and minus the imaginary part of entry
// 16 ((k i) mod 16).
__device__ __forceinline__ float dft16_real_entry(const float2* tab, int rho, int kappa) {
  const float2 w = tab[16 * (((rho & 15) * (kappa & 15)) & 15)];
  if ((rho >> 4) == (kappa >> 4)) return w.x;
  return (rho >> 4) == 0 ? -w.y : w.y;
}

// t(c, i) = exp(-2 pi j (c mod 16) i/256)/4 (the scaling by 4 is exact)
__device__ __forceinline__ float2 stage_twiddle(const float2* tab, int e) {
  const float2 w = tab[e];
  return make_float2(0.25f * w.x, 0.25f * w.y);
}

// One pass, variant 0: thread c transforms column c in registers.
__device__ __forceinline__ void stage_cuda_cores(const float2* __restrict__ in, float2* __restrict__ out,
                                                 const float2 (&tw)[16]) {
  const int c = threadIdx.x;
  float2 v[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = cmul(in[stage_phys<0>(c + 256 * i)], tw[i]);
  dft_reg<16, false>(v);
#pragma unroll
  for (int k = 0; k < 16; ++k) out[stage_phys<0>(16 * c + k)] = v[k];
}

// One pass, tensor-core variants: warp w transforms the groups of 8 columns g = w, w + 8, w + 16,
// w + 24. In a group, MMA column n (lane / 4 for the B operand) is DFT column 8 g + n; the B
// operand's row kappa is Re x_kappa (kappa < 16) or Im x_(kappa - 16), so lane (r = lane / 4,
// q = lane % 4) supplies x_i for i = q, q + 4, q + 8, q + 12 of column 8 g + r. The accumulator
// rows are Re X_k (m-tile 0) and Im X_k (m-tile 1): lane (r, q) receives X_r and X_(r + 8) of
// columns 8 g + 2 q and 8 g + 2 q + 1.
template <int V>
__device__ __forceinline__ void stage_tensor_cores(const float2* __restrict__ in, float2* __restrict__ out,
                                                   const float2 (&tw)[4], const unsigned (&ahi)[2][4][4],
                                                   const unsigned (&alo)[2][4][4]) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, q = lane & 3, r = lane >> 2;
#pragma unroll 2
  for (int gi = 0; gi < 4; ++gi) {
    const int g = w + 8 * gi;
    const int c = 8 * g + r;
    float2 xv[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) xv[j] = cmul(in[stage_phys<V>(c + 256 * (q + 4 * j))], tw[j]);
    // B operand of k-tile kt: rows 8 kt + q and 8 kt + q + 4
    const float bsrc[4][2] = {{xv[0].x, xv[1].x}, {xv[2].x, xv[3].x}, {xv[0].y, xv[1].y}, {xv[2].y, xv[3].y}};
    float d[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
    if constexpr (V == 3) {
      // the split of variant 2, recombined and stored where the operands came from
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        unsigned hx, lx, hy, ly;
        split_tf32(xv[j].x, hx, lx);
        split_tf32(xv[j].y, hy, ly);
        out[stage_phys<V>(c + 256 * (q + 4 * j))] =
            make_float2(__uint_as_float(hx) + __uint_as_float(lx), __uint_as_float(hy) + __uint_as_float(ly));
      }
      continue;
    }
    if constexpr (V == 1) {
#pragma unroll
      for (int kt = 0; kt < 4; ++kt) {
        const unsigned b0 = __float_as_uint(bsrc[kt][0]), b1 = __float_as_uint(bsrc[kt][1]);
#pragma unroll
        for (int mt = 0; mt < 2; ++mt) mma_tf32(d[mt], ahi[mt][kt], b0, b1);
      }
    } else {
      unsigned bh[4][2], bl[4][2];
#pragma unroll
      for (int kt = 0; kt < 4; ++kt)
#pragma unroll
        for (int e = 0; e < 2; ++e) split_tf32(bsrc[kt][e], bh[kt][e], bl[kt][e]);
      // the small cross terms first, then the leading products
#pragma unroll
      for (int kt = 0; kt < 4; ++kt)
#pragma unroll
        for (int mt = 0; mt < 2; ++mt) {
          mma_tf32(d[mt], alo[mt][kt], bh[kt][0], bh[kt][1]);
          mma_tf32(d[mt], ahi[mt][kt], bl[kt][0], bl[kt][1]);
        }
#pragma unroll
      for (int kt = 0; kt < 4; ++kt)
#pragma unroll
        for (int mt = 0; mt < 2; ++mt) mma_tf32(d[mt], ahi[mt][kt], bh[kt][0], bh[kt][1]);
    }
    const int c0 = 8 * g + 2 * q;
    out[stage_phys<V>(16 * c0 + r)] = make_float2(d[0][0], d[1][0]);
    out[stage_phys<V>(16 * (c0 + 1) + r)] = make_float2(d[0][1], d[1][1]);
    out[stage_phys<V>(16 * c0 + r + 8)] = make_float2(d[0][2], d[1][2]);
    out[stage_phys<V>(16 * (c0 + 1) + r + 8)] = make_float2(d[0][3], d[1][3]);
  }
}

template <int V>
__global__ void __launch_bounds__(kStageThreads) k_dft_stage(const float2* x, float2* y, int passes) {
  extern __shared__ __align__(16) unsigned char smraw[];
  float2* b0 = reinterpret_cast<float2*>(smraw);
  float2* b1 = b0 + kStageBuf;
  float2* roots = b1 + kStageBuf;
  const float2* xg = x + (size_t)blockIdx.x * kStageGroup;
  fill_unit_roots(roots);
  for (int L = threadIdx.x; L < kStageGroup; L += kStageThreads) b0[stage_phys<V>(L)] = xg[L];
  __syncthreads();
  if constexpr (V == 0) {
    float2 tw[16];
    const int cm = threadIdx.x & 15;
#pragma unroll
    for (int i = 0; i < 16; ++i) tw[i] = stage_twiddle(roots, cm * i);
    for (int p = 0; p < passes; ++p) {
      stage_cuda_cores(b0, b1, tw);
      __syncthreads();
      float2* t = b0; b0 = b1; b1 = t;
    }
  } else {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, q = lane & 3, r = lane >> 2;
    // every group of this warp has columns 8 g + r with g = w (mod 8), so c mod 16 = 8 (w & 1) + r
    const int cm = 8 * (w & 1) + r;
    float2 tw[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) tw[j] = stage_twiddle(roots, cm * (q + 4 * j));
    // A fragments (m16n8k8 TF32: a0 (row r, col q), a1 (row r + 8, col q), a2 (row r, col q + 4),
    // a3 (row r + 8, col q + 4) of each 16 x 8 tile), split into TF32 high and low parts
    unsigned ahi[2][4][4], alo[2][4][4];
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
      for (int kt = 0; kt < 4; ++kt)
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int rho = 16 * mt + r + ((e & 1) ? 8 : 0), kappa = 8 * kt + q + ((e & 2) ? 4 : 0);
          const float a = dft16_real_entry(roots, rho, kappa);
          ahi[mt][kt][e] = to_tf32(a);
          alo[mt][kt][e] = to_tf32(a - __uint_as_float(ahi[mt][kt][e]));
        }
    for (int p = 0; p < passes; ++p) {
      stage_tensor_cores<V>(b0, b1, tw, ahi, alo);
      __syncthreads();
      float2* t = b0; b0 = b1; b1 = t;
    }
  }
  float2* yg = y + (size_t)blockIdx.x * kStageGroup;
  for (int L = threadIdx.x; L < kStageGroup; L += kStageThreads) yg[L] = b0[stage_phys<V>(L)];
}

template <int V>
aim_status launch_dft_stage(int groups, int passes, const float2* x, float2* y, cudaStream_t st) {
  const size_t smem = (2 * (size_t)kStageBuf + kStageThreads) * sizeof(float2);
  AIM_CUDA_TRY(cudaFuncSetAttribute(k_dft_stage<V>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  ProfScope ps(K_DFT_STAGE, st);
  k_dft_stage<V><<<groups, kStageThreads, smem, st>>>(x, y, passes);
  AIM_CUDA_TRY(cudaGetLastError());
  return AIM_OK;
}

}  // namespace
}  // namespace aim

using namespace aim;

extern "C" aim_status aim_dft_stage(int variant, int groups, int passes, const void* x, void* y, void* stream) {
  if (variant < AIM_DFT_STAGE_CUDA_CORES || variant > AIM_DFT_STAGE_SPLIT_ONLY)
    return fail(AIM_EINVAL, "variant must be 0 (CUDA cores), 1 (TF32 tensor cores), 2 (split TF32 tensor cores) or "
                            "3 (split data path without products)");
  if (groups < 1 || groups > (1 << 20) || passes < 0 || passes > (1 << 20))
    return fail(AIM_EINVAL, "groups must be in [1, 2^20] and passes in [0, 2^20]");
  if (!x || !y) return fail(AIM_EINVAL, "x and y must not be NULL");
  if ((reinterpret_cast<size_t>(x) | reinterpret_cast<size_t>(y)) & 7)
    return fail(AIM_EINVAL, "x and y must be 8-byte aligned (complex64)");
  cudaPointerAttributes ax, ay;
  if (cudaPointerGetAttributes(&ax, x) != cudaSuccess || cudaPointerGetAttributes(&ay, y) != cudaSuccess) {
    cudaGetLastError();
    return fail(AIM_EINVAL, "x and y must be device pointers");
  }
  if ((ax.type != cudaMemoryTypeDevice && ax.type != cudaMemoryTypeManaged) ||
      (ay.type != cudaMemoryTypeDevice && ay.type != cudaMemoryTypeManaged))
    return fail(AIM_EINVAL, "x and y must be device pointers");
  int dev = -1;
  AIM_CUDA_TRY(cudaGetDevice(&dev));
  if (ax.device != dev || ay.device != dev) return fail(AIM_EINVAL, "x and y must be on the current device");
  const float2* xin = static_cast<const float2*>(x);
  float2* yout = static_cast<float2*>(y);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (variant == AIM_DFT_STAGE_CUDA_CORES) return launch_dft_stage<0>(groups, passes, xin, yout, st);
  if (variant == AIM_DFT_STAGE_MMA_TF32) return launch_dft_stage<1>(groups, passes, xin, yout, st);
  if (variant == AIM_DFT_STAGE_MMA_TF32X3) return launch_dft_stage<2>(groups, passes, xin, yout, st);
  return launch_dft_stage<3>(groups, passes, xin, yout, st);
}
