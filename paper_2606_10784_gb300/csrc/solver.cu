// Restarted GMRES for the AIM systems (the iterative solver of Sec. I; the Calderon system of
// Eq. 3). Arnoldi runs in FP64 on the device with classical Gram-Schmidt applied twice; the
// small Hessenberg least-squares problem (Givens rotations) is solved on the host, one
// device-to-host copy of the new Hessenberg column per iteration. Several right-hand sides
// run in lock step, each with its own Krylov basis.
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

// Double-float form of k_multidot_partial: part[(z J + j) nrhs + r] = sum over chunk z of
// conj(V[j][r][i]) w[r][i], products, per-thread and block sums in double-float.
__global__ void k_multidot_partial_df(const dfc* __restrict__ V, const dfc* __restrict__ w, int n, int nrhs, int J,
                                      double2* __restrict__ part) {
  const int j = blockIdx.x, r = blockIdx.y, z = blockIdx.z;
  const int i0 = z * kDotChunk, i1 = min(n, i0 + kDotChunk);
  const dfc* v = V + ((size_t)j * nrhs + r) * n;
  const dfc* x = w + (size_t)r * n;
  float rh = 0.f, rl = 0.f, ih = 0.f, il = 0.f;
  for (int i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
    const dfc a = v[i], b = x[i];
    float ph, pl;
    df_dot2<+1>(a.xh, a.xl, b.xh, b.xl, a.yh, a.yl, b.yh, b.yl, ph, pl);   // ax bx + ay by
    df_add(rh, rl, ph, pl, rh, rl);
    df_dot2<-1>(a.xh, a.xl, b.yh, b.yl, a.yh, a.yl, b.xh, b.xl, ph, pl);   // ax by - ay bx
    df_add(ih, il, ph, pl, ih, il);
  }
  // warp and block sums in double-float as well: on this part FP64 runs at 1/64 of the FP32
  // rate, and an FP64 shuffle tree per block cost about as much time as reading the basis
  __shared__ float s4[32][4];
  warp_sum_df(rh, rl, ih, il);
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) {
    s4[wid][0] = rh;
    s4[wid][1] = rl;
    s4[wid][2] = ih;
    s4[wid][3] = il;
  }
  __syncthreads();
  if (wid == 0) {
    const int nw = blockDim.x >> 5;
    rh = lane < nw ? s4[lane][0] : 0.f;
    rl = lane < nw ? s4[lane][1] : 0.f;
    ih = lane < nw ? s4[lane][2] : 0.f;
    il = lane < nw ? s4[lane][3] : 0.f;
    warp_sum_df(rh, rl, ih, il);
    if (lane == 0) part[((size_t)z * J + j) * nrhs + r] = to_d2(rh, rl, ih, il);
  }
}

// out[t] = sum of the chunk partials (FP64, in chunk order), and its double-float copy
__global__ void k_multidot_finish_df(const double2* __restrict__ part, int nz, int count, double2* __restrict__ out,
                                     dfc* __restrict__ out_df) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= count) return;
  double re = 0.0, im = 0.0;
  for (int z = 0; z < nz; ++z) {
    const double2 p = part[(size_t)z * count + t];
    re += p.x;
    im += p.y;
  }
  out[t] = double2{re, im};
  out_df[t] = to_dfc(double2{re, im});
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

__global__ void k_add_small(double2* a, const double2* b, int count) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < count) { a[t].x += b[t].x; a[t].y += b[t].y; }
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

// out[j*nrhs + r] = <V[j][r], w[r]> for j < J over the double-float basis (two launches)
static aim_status multidot_df(const dfc* V, const dfc* w, int J, int n, int nrhs, double2* out, dfc* out_df,
                              double2* part, cudaStream_t st) {
  const int nz = (n + kDotChunk - 1) / kDotChunk;
  count_launches(K_GMRES, 2);
  k_multidot_partial_df<<<dim3(J, nrhs, nz), 256, 0, st>>>(V, w, n, nrhs, J, part);
  k_multidot_finish_df<<<blocks_for((long long)J * nrhs, 256), 256, 0, st>>>(part, nz, J * nrhs, out, out_df);
  AIM_CUDA_TRY(cudaGetLastError());
  return AIM_OK;
}

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
  // partial sums of the basis updates (chunks of kCgsChunk vectors) or of the inner products
  // (chunks of kDotChunk elements), whichever needs more
  const size_t nz = (n + kDotChunk - 1) / kDotChunk;
  const size_t part_vecs = std::max((size_t)(restart + kCgsChunk) / kCgsChunk, (nz * (restart + 1) + n - 1) / n);
  // basis (restart + 1, double-float), w, r, the current vector, w in double-float, partial sums
  const size_t nvec = (size_t)(restart + 1) + 4 + part_vecs;
  return nvec * nrhs * n * sizeof(double2);
}

size_t reduction_bytes(int nrhs, int restart) {
  // dots, dots2, norms, their double-float copies, and the active flags
  return ((size_t)(restart + 2) * 5 + 1) * nrhs * sizeof(double2) + nrhs * sizeof(int);
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
  ws.active = reinterpret_cast<int*>(red + ((size_t)(restart + 2) * 5 + 1) * nrhs);
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
    // Arnoldi step j: w = A v_j, CGS2 against v_0..v_j, v_{j+1} = w / ||w||, and the D2H copy
    // of Hessenberg column j into host slot j % 2. A step needs nothing from the host, so step
    // j + 1 is queued before the host waits for column j: the Givens updates on the host overlap
    // the next matvec on the device (one step of lookahead; the step queued after the last
    // useful one is discarded).
    auto arnoldi_step = [&](int j) -> aim_status {
      double2* slot = hred + (size_t)(j & 1) * (restart + 2) * nrhs;
      // w = A v_j (cur = v_j)
      if (!op_graph.tried) op_graph.capture(ctx, op, nrhs, ws.cur, ws.w, precision, st);
      if (op_graph.exec != nullptr) {
        AIM_TRY(op_graph.replay(st));
      } else {
        AIM_TRY(solver_apply(ctx, op, nrhs, ws.cur, ws.w, precision, st));
      }
      // CGS2 (3 launches here + 2 x 2 in multidot_df + 2 x 2 in vcombine_df + 2 in dot_norms),
      // timed as one group when profiling
      ProfScope group(K_GMRES, st, /*count_launch=*/false);
      count_launches(K_GMRES, 3);
      k_to_dfc<<<nb, tpb, 0, st>>>(ws.w, (int)vsz, ws.wdf);
      AIM_TRY(multidot_df(ws.V, ws.wdf, j + 1, n, nrhs, ws.dots, ws.dots_df, ws.tmp, st));
      vcombine_df(ws.V, ws.dots_df, j + 1, n, nrhs, -1.0, ws.w, ws.wdf, ws.tmp, st);
      AIM_TRY(multidot_df(ws.V, ws.wdf, j + 1, n, nrhs, ws.dots2, ws.dots2_df, ws.tmp, st));
      vcombine_df(ws.V, ws.dots2_df, j + 1, n, nrhs, -1.0, ws.w, nullptr, ws.tmp, st);
      k_add_small<<<blocks_for((j + 1) * nrhs, tpb), tpb, 0, st>>>(ws.dots, ws.dots2, (j + 1) * nrhs);
      AIM_TRY(dot_norms(ws.w, n, nrhs, ws.nrm, ws.tmp, st));
      k_normalize<<<nb, tpb, 0, st>>>(ws.w, ws.nrm, ws.active, n, nrhs, ws.V + (size_t)(j + 1) * vsz, ws.cur);
      AIM_CUDA_TRY(cudaGetLastError());
      AIM_CUDA_TRY(cudaMemcpyAsync(slot, ws.dots, (size_t)(j + 1) * nrhs * sizeof(double2), cudaMemcpyDeviceToHost, st));
      AIM_CUDA_TRY(cudaMemcpyAsync(slot + (size_t)(j + 1) * nrhs, ws.nrm, nrhs * sizeof(double2), cudaMemcpyDeviceToHost, st));
      AIM_CUDA_TRY(cudaEventRecord(col_ready.e[j & 1], st));
      return AIM_OK;
    };
    int jdone = 0;
    AIM_TRY(arnoldi_step(0));
    for (int j = 0; j < restart; ++j) {
      if (j + 1 < restart) AIM_TRY(arnoldi_step(j + 1));
      AIM_CUDA_TRY(cudaEventSynchronize(col_ready.e[j & 1]));
      const double2* hcol = hred + (size_t)(j & 1) * (restart + 2) * nrhs;
      jdone = j + 1;
      bool all_done = true;
      if ((int)Hcol.size() <= j) Hcol.resize(j + 1);
      Hcol[j].assign((size_t)(j + 2) * nrhs, Zc{0.0, 0.0});
      Zc* col = Hcol[j].data();   // column j, rows 0..j+1
      for (int r = 0; r < nrhs; ++r) {
        if (!active[r] || jconv[r]) continue;
        for (int i = 0; i <= j; ++i) col[(size_t)i * nrhs + r] = {hcol[(size_t)i * nrhs + r].x, hcol[(size_t)i * nrhs + r].y};
        const double hn = std::sqrt(std::fmax(hcol[(size_t)(j + 1) * nrhs + r].x, 0.0));
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
