// Grid-product helpers shared by every element type: the banded Gram inverse (G^-1 of Eq. 3),
// workspace sizing, and the feasibility of a launch schedule.
#include "matvec_kernels.cuh"

namespace aim {

// y = G^-1 x from the stored band (or the dense inverse for small n). Each output (i, r) belongs
// to a group of kGramLanes adjacent lanes: lane g of the group sums the entries d = g, g + 8, ...
// in order, and the group then adds its partial sums by xor shuffles, so the order of every sum
// is fixed whatever the number of right-hand sides. FP64 throughput sets the cost of this kernel
// on this GPU: a whole warp per output spent twice as many FP64 operations on its shuffle tree
// as on the band itself, and a thread per output left the GPU idle for one vector (n threads,
// each a chain of cnt dependent loads and FMAs).
constexpr int kGramLanes = 8;

__global__ void k_gram_inv(const double* __restrict__ gi, int blo, int cnt, int n, int nrhs,
                           const double2* __restrict__ x, double2* __restrict__ y) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long o = t / kGramLanes;
  const int g = threadIdx.x & (kGramLanes - 1);
  const bool valid = o < (long long)n * nrhs;
  double re = 0.0, im = 0.0;
  if (valid) {
    const int r = (int)(o / n), i = (int)(o - (long long)r * n);
    const double* row = gi + (size_t)i * cnt;
    const double2* xv = x + (size_t)r * n;
#pragma unroll 4
    for (int d = g; d < cnt; d += kGramLanes) {
      int j = i - blo + d;
      if (j < 0) j += n;
      if (j >= n) j -= n;
      const double gv = row[d];
      const double2 xx = xv[j];
      re = fma(gv, xx.x, re);
      im = fma(gv, xx.y, im);
    }
  }
  // every lane of the warp takes part in the shuffles (groups past the end carry zeros)
#pragma unroll
  for (int off = kGramLanes / 2; off > 0; off >>= 1) {
    re += __shfl_xor_sync(0xffffffffu, re, off);
    im += __shfl_xor_sync(0xffffffffu, im, off);
  }
  if (valid && g == 0) y[o] = double2{re, im};
}

size_t inter_bytes_needed(const aim_ctx* ctx, int channels, int precision) {
  const size_t el = precision == AIM_MIXED ? sizeof(float2) : sizeof(double2);   // dfc is 16 bytes too
  return (size_t)channels * ctx->P * ctx->nrows * el;
}

bool schedule_feasible(int precision, int logH, int logP, const Schedule& s) {
  switch (precision) {
    case AIM_MIXED: return feasible_for<float2>(s, logH, logP);
    case AIM_FP64: return feasible_for<dfc>(s, logH, logP);
    case AIM_FP64_NATIVE: return feasible_for<double2>(s, logH, logP);
    default: return false;
  }
}

aim_status gram_inv_apply(aim_ctx* ctx, int nrhs, const double2* x, double2* y, cudaStream_t st) {
  if (ctx->gram_inv == nullptr) return fail(AIM_ESTATE, "no Gram matrix on a TM context");
  const int blo = ctx->gram_band;
  const int cnt = (blo * 2 + 1 <= ctx->n) ? 2 * blo + 1 : ctx->n;
  const int total = ctx->n * nrhs;
  {
    ProfScope ps(K_GRAM, st);
    k_gram_inv<<<(unsigned)(((long long)total * kGramLanes + 255) / 256), 256, 0, st>>>(ctx->gram_inv, blo, cnt,
                                                                                        ctx->n, nrhs, x, y);
  }
  AIM_CUDA_TRY(cudaGetLastError());
  return AIM_OK;
}

}  // namespace aim
