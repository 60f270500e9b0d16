// Golub-Kahan-Lanczos bidiagonalisation of an AIM operator, for the singular-value studies of
// Sec. IV (Figs. 2-3): the operator A (S, S^alpha, N, N^alpha, G^-1 or a Calderon product, all
// applied through the grid product) is reduced to an upper bidiagonal B with
//     A v_j = alpha_j u_j + beta_{j-1} u_{j-1},   A^H u_j = alpha_j v_j + beta_j v_{j+1},
// whose singular values approximate those of A (all of them when k = n). Both Lanczos bases are
// reorthogonalised in full against every earlier vector, classical Gram-Schmidt applied twice, in
// FP64 with fixed-order sums (deterministic). The norms and the normalisations stay on the device,
// so the loop never waits for the host.
//
// The adjoint: the TE Galerkin operators are complex symmetric (the same projections on both sides,
// an even grid kernel, a symmetric near field), so A^H x = conj(A conj(x)); for the Calderon
// products G^-1 S G^-1 N the transpose is N G^-1 S G^-1, the same factors in reverse order.
#include <algorithm>
#include <cmath>

#include "aim_internal.h"

namespace aim {

namespace {

constexpr int kLzChunk = 1024;   // elements per partial inner product

// part[z * J + j] = sum over chunk z of conj(B_j[i]) w[i], j < J (basis rows of length n)
__global__ void k_lz_dots_partial(const double2* __restrict__ B, const double2* __restrict__ w, int n, int J,
                                  double2* __restrict__ part) {
  const int j = blockIdx.x, z = blockIdx.y;
  const int i0 = z * kLzChunk, i1 = min(n, i0 + kLzChunk);
  const double2* b = B + (size_t)j * n;
  double re = 0.0, im = 0.0;
  for (int i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
    const double2 a = b[i], x = w[i];
    re = fma(a.x, x.x, fma(a.y, x.y, re));
    im = fma(a.x, x.y, fma(-a.y, x.x, im));
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
    if (lane == 0) part[(size_t)z * J + j] = double2{re, im};
  }
}

// c[j] = sum over chunks (in order) of the partials
__global__ void k_lz_dots_finish(const double2* __restrict__ part, int nz, int J, double2* __restrict__ c) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= J) return;
  double re = 0.0, im = 0.0;
  for (int z = 0; z < nz; ++z) {
    const double2 p = part[(size_t)z * J + j];
    re += p.x;
    im += p.y;
  }
  c[j] = double2{re, im};
}

// w[i] -= sum_j c[j] B_j[i], j < J, in order of j
__global__ void k_lz_subtract(const double2* __restrict__ B, const double2* __restrict__ c, int n, int J,
                              double2* __restrict__ w) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double re = 0.0, im = 0.0;
  for (int j = 0; j < J; ++j) {
    const double2 b = B[(size_t)j * n + i], cj = c[j];
    re = fma(cj.x, b.x, fma(-cj.y, b.y, re));
    im = fma(cj.x, b.y, fma(cj.y, b.x, im));
  }
  const double2 x = w[i];
  w[i] = double2{x.x - re, x.y - im};
}

// w -= s * prev, s = coef[idx] (a real Lanczos coefficient kept on the device); idx < 0: nothing
__global__ void k_lz_axpy(double2* __restrict__ w, const double2* __restrict__ prev, const double* __restrict__ coef,
                          int idx, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n || idx < 0) return;
  const double s = coef[idx];
  const double2 p = prev[i], x = w[i];
  w[i] = double2{x.x - s * p.x, x.y - s * p.y};
}

// out = w / ||w|| with ||w||^2 = Re sum of the (finished) self inner products nrm[0]; the norm goes to
// coef[idx]. A zero vector (breakdown: the Krylov space is exhausted) stays zero.
__global__ void k_lz_normalise(const double2* __restrict__ w, const double2* __restrict__ nrm, double* __restrict__ coef,
                               int idx, int n, double2* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const double nn = sqrt(fmax(nrm[0].x, 0.0));
  if (i == 0) coef[idx] = nn;
  if (i >= n) return;
  const double s = nn > 1e-300 ? 1.0 / nn : 0.0;
  const double2 x = w[i];
  out[i] = double2{x.x * s, x.y * s};
}

__global__ void k_lz_conj(const double2* __restrict__ x, int n, double2* __restrict__ y) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = double2{x[i].x, -x[i].y};
}

struct LzWork {
  double2* part;    // partial inner products
  double2* c;       // finished inner products
  int nz;
};

inline unsigned blocks(long long n, int tpb) { return (unsigned)((n + tpb - 1) / tpb); }

// c = B[0..J)^H w (J >= 1), then w -= B c: one classical Gram-Schmidt pass
aim_status cgs_pass(const double2* B, int J, int n, double2* w, const LzWork& ws, cudaStream_t st) {
  count_launches(K_GMRES, 3);
  k_lz_dots_partial<<<dim3(J, ws.nz), 256, 0, st>>>(B, w, n, J, ws.part);
  k_lz_dots_finish<<<blocks(J, 128), 128, 0, st>>>(ws.part, ws.nz, J, ws.c);
  k_lz_subtract<<<blocks(n, 256), 256, 0, st>>>(B, ws.c, n, J, w);
  AIM_CUDA_TRY(cudaGetLastError());
  return AIM_OK;
}

// ||w||^2 into ws.c[0], then out = w/||w|| and coef[idx] = ||w||
aim_status normalise(const double2* w, int n, double* coef, int idx, double2* out, const LzWork& ws, cudaStream_t st) {
  count_launches(K_GMRES, 3);
  k_lz_dots_partial<<<dim3(1, ws.nz), 256, 0, st>>>(w, w, n, 1, ws.part);
  k_lz_dots_finish<<<1, 32, 0, st>>>(ws.part, ws.nz, 1, ws.c);
  k_lz_normalise<<<blocks(n, 256), 256, 0, st>>>(w, ws.c, coef, idx, n, out);
  AIM_CUDA_TRY(cudaGetLastError());
  return AIM_OK;
}

bool is_calderon(aim_op op) {
  return op == AIM_OP_CALDERON || op == AIM_OP_CALDERON_ALPHA || op == AIM_OP_CALDERON_ALPHA2;
}

// y = A^T x: A itself for the complex-symmetric operators, the reversed chain for the Calderon products
aim_status apply_transpose(aim_ctx* ctx, aim_op op, const double2* x, double2* y, double2* t1, double2* t2,
                           int precision, cudaStream_t st) {
  if (!is_calderon(op)) return apply_op(ctx, op, 1, x, y, precision, st);
  // (G^-1 S' G^-1 N')^T = N' G^-1 S' G^-1
  const aim_op s_op = op == AIM_OP_CALDERON ? AIM_OP_S : AIM_OP_S_ALPHA;
  const aim_op n_op = op == AIM_OP_CALDERON_ALPHA2 ? AIM_OP_N_ALPHA : AIM_OP_N;
  AIM_TRY(gram_inv_apply(ctx, 1, x, t1, st));
  AIM_TRY(apply_op(ctx, s_op, 1, t1, t2, precision, st));
  AIM_TRY(gram_inv_apply(ctx, 1, t2, t1, st));
  return apply_op(ctx, n_op, 1, t1, y, precision, st);
}

}  // namespace

aim_status lanczos_bidiag(aim_ctx* ctx, aim_op op, int k, int precision, const double2* v0, double* alpha_h,
                          double* beta_h, double2* U_out, double2* V_out, cudaStream_t st) {
  const int n = ctx->n;
  const size_t vec = (size_t)n * sizeof(double2);
  // device workspace: the two bases (unless the caller's), four vectors, the coefficients, partials
  const int nz = (n + kLzChunk - 1) / kLzChunk;
  const size_t own_u = U_out ? 0 : (size_t)k * n, own_v = V_out ? 0 : (size_t)(k + 1) * n;
  const size_t total = (own_u + own_v + 4 * (size_t)n + (size_t)nz * (k + 1) + (k + 1)) * sizeof(double2) +
                       2 * (size_t)(k + 1) * sizeof(double);
  void* mem = nullptr;
  AIM_CUDA_TRY(cudaMallocAsync(&mem, total, st));
  double2* base = static_cast<double2*>(mem);
  double2* U = U_out ? U_out : base;
  base += own_u;
  double2* V = V_out ? V_out : base;
  base += own_v;
  double2* w = base;
  double2* t0 = w + n;
  double2* t1 = t0 + n;
  double2* t2 = t1 + n;
  LzWork ws{t2 + n, t2 + n + (size_t)nz * (k + 1), nz};
  double* coef = reinterpret_cast<double*>(ws.c + (k + 1));   // alpha[0..k), then beta[0..k)
  double* alpha = coef;
  double* beta = coef + (k + 1);
  aim_status s = AIM_OK;
  // v_0 = v0 / ||v0|| (the norm lands in beta[k], a spare slot)
  if (cudaMemcpyAsync(w, v0, vec, cudaMemcpyDefault, st) != cudaSuccess) s = fail(AIM_ECUDA, "start vector copy");
  if (s == AIM_OK) s = normalise(w, n, beta, k, V, ws, st);
  for (int j = 0; j < k && s == AIM_OK; ++j) {
    const double2* vj = V + (size_t)j * n;
    double2* uj = U + (size_t)j * n;
    // u = A v_j - beta_{j-1} u_{j-1}, reorthogonalised against u_0..u_{j-1}
    s = apply_op(ctx, op, 1, vj, w, precision, st);
    if (s != AIM_OK) break;
    if (j > 0) {
      count_launches(K_GMRES, 1);
      k_lz_axpy<<<blocks(n, 256), 256, 0, st>>>(w, U + (size_t)(j - 1) * n, beta, j - 1, n);
      for (int pass = 0; pass < 2 && s == AIM_OK; ++pass) s = cgs_pass(U, j, n, w, ws, st);
      if (s != AIM_OK) break;
    }
    s = normalise(w, n, alpha, j, uj, ws, st);
    if (s != AIM_OK) break;
    // v = A^H u_j - alpha_j v_j = conj(A^T conj(u_j)) - alpha_j v_j, reorthogonalised against v_0..v_j
    count_launches(K_GMRES, 1);
    k_lz_conj<<<blocks(n, 256), 256, 0, st>>>(uj, n, t0);
    s = apply_transpose(ctx, op, t0, w, t1, t2, precision, st);
    if (s != AIM_OK) break;
    count_launches(K_GMRES, 2);
    k_lz_conj<<<blocks(n, 256), 256, 0, st>>>(w, n, w);
    k_lz_axpy<<<blocks(n, 256), 256, 0, st>>>(w, vj, alpha, j, n);
    for (int pass = 0; pass < 2 && s == AIM_OK; ++pass) s = cgs_pass(V, j + 1, n, w, ws, st);
    if (s != AIM_OK) break;
    s = normalise(w, n, beta, j, V + (size_t)(j + 1) * n, ws, st);
  }
  if (s == AIM_OK) {
    cudaError_t e = cudaMemcpyAsync(alpha_h, alpha, k * sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(beta_h, beta, k * sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) s = fail(AIM_ECUDA, std::string("Lanczos coefficients: ") + cudaGetErrorString(e));
  }
  cudaFreeAsync(mem, st);
  const cudaError_t es = cudaStreamSynchronize(st);
  if (s == AIM_OK && es != cudaSuccess) s = fail(AIM_ECUDA, std::string("Lanczos: ") + cudaGetErrorString(es));
  if (s == AIM_OK) {
    for (int j = 0; j < k; ++j)
      if (!std::isfinite(alpha_h[j]) || !std::isfinite(beta_h[j])) return fail(AIM_ENUMERIC, "non-finite Lanczos coefficient");
  }
  return s;
}

}  // namespace aim

using namespace aim;

extern "C" aim_status aim_lanczos_bidiag(aim_ctx* ctx, aim_op op, int k, int precision, const void* v0, double* alpha,
                                         double* beta, void* U, void* V, void* stream) {
  if (!ctx || !v0 || !alpha || !beta || k < 1) return fail(AIM_EINVAL, "bad argument");
  if (k > ctx->n) return fail(AIM_EINVAL, "k must not exceed the number of unknowns");
  if (precision < AIM_FP64 || precision > AIM_FP64_NATIVE) return fail(AIM_EINVAL, "precision must be 0, 1 or 2");
  if (ctx->form != AIM_TE_P1_GALERKIN)
    return fail(AIM_ESTATE, "the adjoint product needs the complex-symmetric TE operators (TM collocation is not)");
  switch (op) {
    case AIM_OP_S: case AIM_OP_S_ALPHA: case AIM_OP_N: case AIM_OP_N_ALPHA: case AIM_OP_GRAM_INV:
    case AIM_OP_CALDERON: case AIM_OP_CALDERON_ALPHA: case AIM_OP_CALDERON_ALPHA2: case AIM_OP_EFIE:
      break;
    default:
      return fail(AIM_EINVAL, "operator has no adjoint here");
  }
  AIM_TRY(check_device(ctx));
  cudaPointerAttributes a;
  for (const void* p : {static_cast<const void*>(U), static_cast<const void*>(V)}) {
    if (p == nullptr) continue;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess || a.type != cudaMemoryTypeDevice) {
      cudaGetLastError();
      return fail(AIM_EINVAL, "U and V must be device pointers (or NULL)");
    }
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  AIM_TRY(reserve(ctx, 1, precision));
  return lanczos_bidiag(ctx, op, k, precision, static_cast<const double2*>(v0), alpha, beta,
                        static_cast<double2*>(U), static_cast<double2*>(V), st);
}
