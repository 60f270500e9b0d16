// Grid-product helpers shared by every element type: the banded Gram inverse (G^-1 of Eq. 3),
// workspace sizing, and the feasibility of a launch schedule.
#include "matvec_kernels.cuh"

namespace aim {

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
    k_gram_inv<<<(total + 255) / 256, 256, 0, st>>>(ctx->gram_inv, blo, cnt, ctx->n, nrhs, x, y);
  }
  AIM_CUDA_TRY(cudaGetLastError());
  return AIM_OK;
}

}  // namespace aim
