// C ABI of the AIM library (declared in include/aim.h): context lifecycle, setup
// orchestration, operator composition (Eq. 3), host/device pointer staging and the solve.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <new>

#include "aim_internal.h"

namespace aim {

static thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }

aim_status fail(aim_status st, const std::string& msg) {
  g_last_error = msg;
  return st;
}

aim_status dev_alloc(aim_ctx* ctx, void** p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) return AIM_OK;
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(AIM_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  }
  ctx->allocations.push_back(*p);
  ctx->device_bytes += bytes;
  return AIM_OK;
}

static bool is_pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }
static int ilog2(int v) {
  int l = 0;
  while ((1 << l) < v) ++l;
  return l;
}

static bool device_pointer(const void* p) {
  if (p == nullptr) return false;
  cudaPointerAttributes attr;
  if (cudaPointerGetAttributes(&attr, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged;
}

aim_status check_device(const aim_ctx* ctx) {
  int dev = -1;
  const cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(AIM_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  }
  if (dev != ctx->device)
    return fail(AIM_EINVAL, "the current CUDA device (" + std::to_string(dev) + ") is not the context's device (" +
                                std::to_string(ctx->device) + "); make it current before the call");
  return AIM_OK;
}

static aim_status grow(void** buf, size_t* have, size_t need) {
  if (*have >= need) return AIM_OK;
  if (*buf) cudaFree(*buf);
  *buf = nullptr;
  *have = 0;
  cudaError_t e = cudaMalloc(buf, need);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(AIM_ENOMEM, std::string("workspace cudaMalloc: ") + cudaGetErrorString(e));
  }
  *have = need;
  return AIM_OK;
}

aim_status reserve(aim_ctx* ctx, int nrhs, int precision) {
  if (nrhs < 1) return fail(AIM_EINVAL, "nrhs must be >= 1");
  const int pidx = precision;
  const int chan = (ctx->form == AIM_TE_P1_GALERKIN ? 3 : 1) * nrhs;
  const size_t el = precision == AIM_MIXED ? sizeof(float2) : sizeof(double2);
  AIM_TRY(grow(&ctx->inter, &ctx->inter_bytes, inter_bytes_needed(ctx, chan, precision)));
  AIM_TRY(grow(&ctx->vact, &ctx->vact_bytes, (size_t)chan * ctx->n_act * el));
  void* vw = ctx->vec_ws;
  AIM_TRY(grow(&vw, &ctx->vec_ws_bytes, 2 * (size_t)nrhs * ctx->n * sizeof(double2)));
  ctx->vec_ws = static_cast<double2*>(vw);
  ctx->reserved_rhs[pidx] = std::max(ctx->reserved_rhs[pidx], nrhs);
  return AIM_OK;
}

static aim_status stage(aim_ctx* ctx, size_t in_bytes, size_t out_bytes) {
  const size_t need = std::max(in_bytes, out_bytes);
  if (ctx->stage_bytes < need) {
    if (ctx->stage_in) cudaFree(ctx->stage_in);
    if (ctx->stage_out) cudaFree(ctx->stage_out);
    ctx->stage_in = ctx->stage_out = nullptr;
    ctx->stage_bytes = 0;
    void* a = nullptr;
    void* b = nullptr;
    AIM_CUDA_TRY(cudaMalloc(&a, need));
    cudaError_t e = cudaMalloc(&b, need);
    if (e != cudaSuccess) {
      cudaFree(a);
      return fail(AIM_ENOMEM, "staging buffer");
    }
    ctx->stage_in = static_cast<double2*>(a);
    ctx->stage_out = static_cast<double2*>(b);
    ctx->stage_bytes = need;
  }
  return AIM_OK;
}

static PassSpec make_spec(const aim_ctx* ctx, aim_op op) {
  PassSpec s{};
  s.out_scale = double2{1.0, 0.0};
  const double k2 = ctx->k * ctx->k;
  switch (op) {
    case AIM_OP_N:
      s.nproj = 3;
      s.proj[0] = 1; s.proj[1] = 2; s.proj[2] = 3;
      s.coef[0] = double2{1.0, 0.0};
      s.coef[1] = double2{-k2, 0.0};
      s.coef[2] = double2{-k2, 0.0};
      s.filtered = false;
      s.near = &ctx->near;
      s.near_which = 1;
      break;
    case AIM_OP_N_ALPHA:
      s.nproj = 3;
      s.proj[0] = 1; s.proj[1] = 2; s.proj[2] = 3;
      s.coef[0] = double2{1.0, 0.0};
      s.coef[1] = double2{-k2, 0.0};
      s.coef[2] = double2{-k2, 0.0};
      s.filtered = true;
      s.near = nullptr;
      break;
    case AIM_OP_S_ALPHA:
    case AIM_OP_EFIE_ALPHA:
      s.nproj = 1;
      s.proj[0] = 0;
      s.coef[0] = double2{1.0, 0.0};
      s.filtered = true;
      s.near = nullptr;
      break;
    default:   // S and the TM EFIE
      s.nproj = 1;
      s.proj[0] = 0;
      s.coef[0] = double2{1.0, 0.0};
      s.filtered = false;
      s.near = &ctx->near;
      s.near_which = 0;
      break;
  }
  if (ctx->form == AIM_TM_PULSE_COLLOC && (op == AIM_OP_EFIE || op == AIM_OP_EFIE_ALPHA))
    s.out_scale = double2{0.0, ctx->k};   // j k eta, eta = 1
  return s;
}

static aim_status pass(aim_ctx* ctx, aim_op op, int nrhs, const double2* x, double2* y, int precision, cudaStream_t st) {
  const PassSpec spec = make_spec(ctx, op);
  if (precision == AIM_MIXED) return grid_pass<float2>(ctx, spec, nrhs, x, y, st);
  if (precision == AIM_FP64_NATIVE) return grid_pass<double2>(ctx, spec, nrhs, x, y, st);
  return grid_pass<dfc>(ctx, spec, nrhs, x, y, st);
}

aim_status apply_op(aim_ctx* ctx, aim_op op, int nrhs, const double2* x, double2* y, int precision, cudaStream_t st) {
  const bool te = ctx->form == AIM_TE_P1_GALERKIN;
  if (ctx->reserved_rhs[precision] < nrhs) AIM_TRY(reserve(ctx, nrhs, precision));
  switch (op) {
    case AIM_OP_S:
    case AIM_OP_S_ALPHA:
      return pass(ctx, op, nrhs, x, y, precision, st);
    case AIM_OP_N:
    case AIM_OP_N_ALPHA:
      if (!te) return fail(AIM_ESTATE, "N is a TE operator");
      return pass(ctx, op, nrhs, x, y, precision, st);
    case AIM_OP_EFIE:
      return pass(ctx, te ? AIM_OP_N : AIM_OP_EFIE, nrhs, x, y, precision, st);
    case AIM_OP_EFIE_ALPHA:
      if (te) return fail(AIM_ESTATE, "the filtered EFIE system is defined for TM contexts");
      return pass(ctx, op, nrhs, x, y, precision, st);
    case AIM_OP_GRAM_INV:
      if (!te) return fail(AIM_ESTATE, "G is a TE operator");
      return gram_inv_apply(ctx, nrhs, x, y, st);
    case AIM_OP_CALDERON:
    case AIM_OP_CALDERON_ALPHA:
    case AIM_OP_CALDERON_ALPHA2: {
      if (!te) return fail(AIM_ESTATE, "the Calderon product is a TE operator");
      // y = G^-1 S G^-1 N x  (Eq. 3), S^alpha of Eq. 10 for the filtered variants, N^alpha too
      // for the doubly filtered one
      double2* t1 = ctx->vec_ws;
      double2* t2 = ctx->vec_ws + (size_t)nrhs * ctx->n;
      AIM_TRY(pass(ctx, op == AIM_OP_CALDERON_ALPHA2 ? AIM_OP_N_ALPHA : AIM_OP_N, nrhs, x, t1, precision, st));
      AIM_TRY(gram_inv_apply(ctx, nrhs, t1, t2, st));
      AIM_TRY(pass(ctx, op == AIM_OP_CALDERON ? AIM_OP_S : AIM_OP_S_ALPHA, nrhs, t2, t1, precision, st));
      return gram_inv_apply(ctx, nrhs, t1, y, st);
    }
    default:
      return fail(AIM_EINVAL, "unknown operator");
  }
}

aim_status device_spectra_and_near(aim_ctx* ctx, const HostSetup& hs, cudaStream_t st);

// ------------------------------------------------------------------------------------
// several contexts per launch
// ------------------------------------------------------------------------------------
constexpr int kMultiStages = 2;

aim_status MultiLauncher::init() {
  if (scratch != nullptr) return AIM_OK;
  void* p = nullptr;
  AIM_CUDA_TRY(cudaMalloc(&p, kMultiStages * 4 * sizeof(unsigned)));
  scratch = static_cast<unsigned*>(p);
  AIM_CUDA_TRY(cudaMallocHost(&p, kMultiStages * sizeof(int)));
  err_host = static_cast<int*>(p);
  for (int i = 0; i < kMultiStages; ++i) err_host[i] = 0;
  return AIM_OK;
}

aim_status MultiLauncher::check() {
  for (int i = 0; i < kMultiStages; ++i)
    if (err_host != nullptr && err_host[i] != 0) {
      err_host[i] = 0;
      return fail(AIM_ETIMEOUT, "a grid barrier of the multi-context launch gave up waiting");
    }
  return AIM_OK;
}

MultiLauncher::~MultiLauncher() {
  if (scratch) cudaFree(scratch);
  if (err_host) cudaFreeHost(err_host);
}

static aim_status multi_stage(MultiLauncher& ml, int stage, const std::vector<MultiPassSpec>& passes, int precision,
                              cudaStream_t st) {
  if (passes.empty()) return AIM_OK;
  unsigned* sc = ml.scratch + 4 * stage;
  int* eh = ml.err_host + stage;
  if (precision == AIM_MIXED) return grid_pass_multi<float2>(passes.data(), (int)passes.size(), sc, eh, st);
  if (precision == AIM_FP64_NATIVE) return grid_pass_multi<double2>(passes.data(), (int)passes.size(), sc, eh, st);
  return grid_pass_multi<dfc>(passes.data(), (int)passes.size(), sc, eh, st);
}

aim_status apply_op_multi(MultiLauncher& ml, int count, aim_ctx* const* ctxs, const aim_op* ops, const int* nrhs,
                          const double2* const* x, double2* const* y, int precision, cudaStream_t st) {
  AIM_TRY(ml.init());
  std::vector<MultiPassSpec> first, second;
  for (int i = 0; i < count; ++i) {
    aim_ctx* ctx = ctxs[i];
    const bool te = ctx->form == AIM_TE_P1_GALERKIN;
    if (ctx->reserved_rhs[precision] < nrhs[i]) AIM_TRY(reserve(ctx, nrhs[i], precision));
    const aim_op op = ops[i];
    switch (op) {
      case AIM_OP_S: case AIM_OP_S_ALPHA:
        first.push_back({ctx, make_spec(ctx, op), nrhs[i], x[i], y[i]});
        break;
      case AIM_OP_N: case AIM_OP_N_ALPHA:
        if (!te) return fail(AIM_ESTATE, "N is a TE operator");
        first.push_back({ctx, make_spec(ctx, op), nrhs[i], x[i], y[i]});
        break;
      case AIM_OP_EFIE:
        first.push_back({ctx, make_spec(ctx, te ? AIM_OP_N : AIM_OP_EFIE), nrhs[i], x[i], y[i]});
        break;
      case AIM_OP_EFIE_ALPHA:
        if (te) return fail(AIM_ESTATE, "the filtered EFIE system is defined for TM contexts");
        first.push_back({ctx, make_spec(ctx, op), nrhs[i], x[i], y[i]});
        break;
      case AIM_OP_GRAM_INV:
        if (!te) return fail(AIM_ESTATE, "G is a TE operator");
        break;
      case AIM_OP_CALDERON: case AIM_OP_CALDERON_ALPHA: case AIM_OP_CALDERON_ALPHA2: {
        if (!te) return fail(AIM_ESTATE, "the Calderon product is a TE operator");
        double2* t1 = ctx->vec_ws;
        double2* t2 = ctx->vec_ws + (size_t)nrhs[i] * ctx->n;
        first.push_back({ctx, make_spec(ctx, op == AIM_OP_CALDERON_ALPHA2 ? AIM_OP_N_ALPHA : AIM_OP_N), nrhs[i], x[i], t1});
        second.push_back({ctx, make_spec(ctx, op == AIM_OP_CALDERON ? AIM_OP_S : AIM_OP_S_ALPHA), nrhs[i], t2, t1});
        break;
      }
      default:
        return fail(AIM_EINVAL, "unknown operator");
    }
  }
  // stage 1: every context's first grid pass, then the Gram inverses between the Calderon factors
  AIM_TRY(multi_stage(ml, 0, first, precision, st));
  for (int i = 0; i < count; ++i) {
    aim_ctx* ctx = ctxs[i];
    const aim_op op = ops[i];
    if (op == AIM_OP_GRAM_INV) AIM_TRY(gram_inv_apply(ctx, nrhs[i], x[i], y[i], st));
    if (op == AIM_OP_CALDERON || op == AIM_OP_CALDERON_ALPHA || op == AIM_OP_CALDERON_ALPHA2)
      AIM_TRY(gram_inv_apply(ctx, nrhs[i], ctx->vec_ws, ctx->vec_ws + (size_t)nrhs[i] * ctx->n, st));
  }
  // stage 2: the single-layer factors of the Calderon products, then their last Gram inverse
  AIM_TRY(multi_stage(ml, 1, second, precision, st));
  for (int i = 0; i < count; ++i) {
    const aim_op op = ops[i];
    if (op == AIM_OP_CALDERON || op == AIM_OP_CALDERON_ALPHA || op == AIM_OP_CALDERON_ALPHA2)
      AIM_TRY(gram_inv_apply(ctxs[i], nrhs[i], ctxs[i]->vec_ws, y[i], st));
  }
  return AIM_OK;
}

// e^{-2 pi i t / P}, t < P, from its FP64 (re, im) pairs: the FP64, complex64 and double-float
// (hi, lo) copies the three grid precisions read.
aim_status upload_twiddles(aim_ctx* ctx, const double* tw2, cudaStream_t st) {
  const int P = ctx->P;
  std::vector<double2> tw(P);
  std::vector<float2> twf(P);
  std::vector<float4> twdf(P);
  for (int t = 0; t < P; ++t) {
    const double c = tw2[2 * t], s = tw2[2 * t + 1];
    const float ch = (float)c, sh = (float)s;
    tw[t] = double2{c, s};
    twf[t] = float2{ch, sh};
    twdf[t] = float4{ch, sh, (float)(c - (double)ch), (float)(s - (double)sh)};   // (xh, yh, xl, yl)
  }
  AIM_TRY(upload(ctx, &ctx->tw, tw, st));
  AIM_TRY(upload(ctx, &ctx->twf, twf, st));
  AIM_TRY(upload(ctx, &ctx->twdf, twdf, st));
  return AIM_OK;
}

aim_status validate_setup(const aim_geometry* g, double k, const aim_grid* grid, const aim_stencil* st,
                           const aim_filter* f) {
  if (!g || !grid || !st || !g->xy) return fail(AIM_EINVAL, "null argument");
  if (g->n_seg < 3) return fail(AIM_EINVAL, "n_seg must be >= 3");
  if (g->form != AIM_TM_PULSE_COLLOC && g->form != AIM_TE_P1_GALERKIN) return fail(AIM_EINVAL, "unknown form");
  if (g->quad_p < 1 || g->quad_p > 16) return fail(AIM_EINVAL, "quad_p must be in 1..16");
  if (!(k > 0.0) || !std::isfinite(k)) return fail(AIM_EINVAL, "k must be positive and finite");
  if (grid->m < 8) return fail(AIM_EINVAL, "m must be >= 8");
  if (st->s < 2 || st->s > 12) return fail(AIM_EINVAL, "stencil s must be in 2..12");
  if (grid->fft_P != 0 && (!is_pow2(grid->fft_P) || grid->fft_P < 2 * grid->m - 1))
    return fail(AIM_EINVAL, "fft_P must be a power of two >= 2m-1");
  if (f && (f->enabled < AIM_FILTER_NONE || f->enabled > AIM_FILTER_ANALYTIC))
    return fail(AIM_EINVAL, "filter kind must be AIM_FILTER_NONE, AIM_FILTER_NUMERICAL or AIM_FILTER_ANALYTIC");
  if (f && f->enabled && !(f->alpha > k) && std::isfinite(f->alpha)) return fail(AIM_EINVAL, "filter radius alpha must exceed k");
  if (f && f->enabled && !std::isfinite(f->alpha)) return fail(AIM_EINVAL, "filter radius alpha must be finite");
  for (int i = 0; i < 2 * g->n_seg; ++i)
    if (!std::isfinite(g->xy[i])) return fail(AIM_EINVAL, "non-finite vertex coordinate");
  return AIM_OK;
}

// The sizes and grid parameters of a context from the caller's description (no device work).
aim_status derive_params(aim_ctx* ctx, const aim_geometry* geometry, double k, const aim_grid* grid,
                                const aim_stencil* stencil, const aim_filter* filter) {
  ctx->form = geometry->form;
  ctx->n = geometry->n_seg;
  ctx->m = grid->m;
  ctx->s = stencil->s;
  ctx->p = geometry->quad_p;
  ctx->k = k;
  ctx->xy.assign(geometry->xy, geometry->xy + 2 * (size_t)geometry->n_seg);
  int P = grid->fft_P;
  if (P == 0) {
    P = kMinP;
    while (P < 2 * grid->m - 1) P *= 2;
  }
  if (P > kMaxP) return fail(AIM_EINVAL, "embedding side P exceeds 4096 (m too large)");
  if (P < kMinP) return fail(AIM_EINVAL, "embedding side P must be >= 64");
  ctx->P = P;
  ctx->logP = ilog2(P);
  ctx->H = P / 2;
  ctx->logH = ctx->logP - 1;
  ctx->L = grid->half_side_L > 0.0 ? grid->half_side_L : host_grid_half_side(geometry->xy, ctx->n, ctx->m, ctx->s);
  ctx->eps = 2.0 * ctx->L / (ctx->m - 1);
  ctx->near_radius = stencil->near_radius > 0.0 ? stencil->near_radius : ctx->s * ctx->eps;
  ctx->filter_enabled = filter ? filter->enabled : AIM_FILTER_NONE;
  ctx->alpha = ctx->filter_enabled ? filter->alpha : 0.0;
  return AIM_OK;
}

}  // namespace aim

using namespace aim;

extern "C" {

const char* aim_status_str(aim_status s) {
  switch (s) {
    case AIM_OK: return "ok";
    case AIM_EINVAL: return "invalid argument";
    case AIM_ENOMEM: return "out of memory";
    case AIM_ECUDA: return "CUDA error";
    case AIM_ENOCONV: return "not converged";
    case AIM_ENUMERIC: return "non-finite value";
    case AIM_ETIMEOUT: return "timeout";
    case AIM_ESTATE: return "operation not valid for this context";
  }
  return "unknown status";
}

const char* aim_last_error(void) { return g_last_error.c_str(); }

void aim_destroy(aim_ctx* ctx) {
  if (!ctx) return;
  for (void* p : ctx->allocations) cudaFree(p);
  if (ctx->inter) cudaFree(ctx->inter);
  if (ctx->vact) cudaFree(ctx->vact);
  if (ctx->vec_ws) cudaFree(ctx->vec_ws);
  if (ctx->stage_in) cudaFree(ctx->stage_in);
  if (ctx->stage_out) cudaFree(ctx->stage_out);
  if (ctx->kry) cudaFree(ctx->kry);
  if (ctx->red) cudaFree(ctx->red);
  if (ctx->red_host) cudaFreeHost(ctx->red_host);
  delete ctx;
}

aim_status aim_setup(const aim_geometry* geometry, double k, const aim_grid* grid, const aim_stencil* stencil,
                     const aim_filter* filter, void* stream, aim_ctx** out) {
  if (!out) return fail(AIM_EINVAL, "out is null");
  *out = nullptr;
  AIM_TRY(validate_setup(geometry, k, grid, stencil, filter));
  const auto t0 = std::chrono::steady_clock::now();
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  aim_ctx* ctx = new (std::nothrow) aim_ctx();
  if (!ctx) return fail(AIM_ENOMEM, "context allocation");
  struct Guard {
    aim_ctx* c;
    ~Guard() { if (c) aim_destroy(c); }
  } guard{ctx};

  cudaGetDevice(&ctx->device);
  AIM_TRY(derive_params(ctx, geometry, k, grid, stencil, filter));

  HostSetup hs;
  AIM_TRY(host_setup(ctx, &hs));
  ctx->n_act = hs.n_act;
  ctx->row_lo = hs.row_lo;
  ctx->row_hi = hs.row_hi;
  ctx->nrows = hs.row_hi - hs.row_lo + 1;

  // upload
  std::vector<double2> nodes(ctx->n);
  for (int i = 0; i < ctx->n; ++i) nodes[i] = double2{ctx->xy[2 * i], ctx->xy[2 * i + 1]};
  AIM_TRY(upload(ctx, &ctx->nodes, nodes, st));
  AIM_TRY(upload(ctx, &ctx->row_ptr, hs.row_ptr, st));
  AIM_TRY(upload(ctx, &ctx->act_ix, hs.act_ix, st));
  AIM_TRY(upload(ctx, &ctx->prj.sc_ptr, hs.sc_ptr, st));
  AIM_TRY(upload(ctx, &ctx->prj.sc_col, hs.sc_col, st));
  AIM_TRY(upload(ctx, &ctx->prj.ga_ptr, hs.ga_ptr, st));
  AIM_TRY(upload(ctx, &ctx->prj.ga_act, hs.ga_act, st));
  ctx->prj.nproj = hs.nproj;
  for (int q = 0; q < hs.nproj; ++q) {
    AIM_TRY(upload(ctx, &ctx->prj.sc_w[q], hs.sc_w[q], st));
    AIM_TRY(upload(ctx, &ctx->prj.ga_w[q], hs.ga_w[q], st));
  }
  AIM_TRY(upload_twiddles(ctx, hs.tw.data(), st));
  if (!hs.gram_inv.empty()) {
    AIM_TRY(upload(ctx, &ctx->gram_inv, hs.gram_inv, st));
    ctx->gram_band = hs.gram_band;
  }
  ctx->n_sc = hs.sc_col.size();
  ctx->n_ga = hs.ga_act.size();
  ctx->n_gram = hs.gram_inv.size();
  AIM_TRY(device_spectra_and_near(ctx, hs, st));
  AIM_CUDA_TRY(cudaStreamSynchronize(st));
  ctx->setup_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  guard.c = nullptr;
  *out = ctx;
  return AIM_OK;
}

aim_status aim_get_info(const aim_ctx* ctx, aim_info* info) {
  if (!ctx || !info) return fail(AIM_EINVAL, "null argument");
  info->n = ctx->n;
  info->m = ctx->m;
  info->fft_P = ctx->P;
  info->s = ctx->s;
  info->quad_p = ctx->p;
  info->k = ctx->k;
  info->L = ctx->L;
  info->eps = ctx->eps;
  info->alpha = ctx->alpha;
  info->n_active = ctx->n_act;
  info->row_lo = ctx->row_lo;
  info->row_hi = ctx->row_hi;
  info->nnz_near = ctx->nnz_near;
  info->device_bytes = ctx->device_bytes + ctx->inter_bytes + ctx->vact_bytes + ctx->vec_ws_bytes +
                       2 * ctx->stage_bytes + ctx->kry_bytes + ctx->red_bytes;
  info->setup_seconds = ctx->setup_seconds;
  info->filter_kind = ctx->filter_enabled;
  return AIM_OK;
}

aim_status aim_kernel_table(aim_ctx* ctx, int which, void* out, void* stream) {
  if (!ctx || !out) return fail(AIM_EINVAL, "bad argument");
  if (which < AIM_TABLE_SPECTRUM || which > AIM_TABLE_ANALYTIC_SPECTRUM) return fail(AIM_EINVAL, "unknown kernel table");
  AIM_TRY(check_device(ctx));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t bytes = (size_t)(ctx->H + 1) * (ctx->H + 1) * sizeof(double2);
  const bool dev = device_pointer(out);
  double2* buf = static_cast<double2*>(out);
  if (!dev) {
    void* p = nullptr;
    AIM_CUDA_TRY(cudaMalloc(&p, bytes));
    buf = static_cast<double2*>(p);
  }
  aim_status s = kernel_table(ctx, which, buf, st);
  if (s == AIM_OK && !dev) {
    const cudaError_t e = cudaMemcpyAsync(out, buf, bytes, cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) s = fail(AIM_ECUDA, std::string("kernel table copy: ") + cudaGetErrorString(e));
  }
  const cudaError_t es = cudaStreamSynchronize(st);
  if (s == AIM_OK && es != cudaSuccess) s = fail(AIM_ECUDA, std::string("kernel table: ") + cudaGetErrorString(es));
  if (!dev) cudaFree(buf);
  return s;
}

aim_status aim_reserve(aim_ctx* ctx, int nrhs, int precision) {
  if (!ctx) return fail(AIM_EINVAL, "null context");
  if (precision < AIM_FP64 || precision > AIM_FP64_NATIVE) return fail(AIM_EINVAL, "precision must be 0, 1 or 2");
  AIM_TRY(check_device(ctx));
  return reserve(ctx, nrhs, precision);
}

aim_status aim_set_schedule(aim_ctx* ctx, int precision, const aim_schedule* schedule) {
  if (!ctx || !schedule) return fail(AIM_EINVAL, "bad argument");
  if (precision < AIM_FP64 || precision > AIM_FP64_NATIVE) return fail(AIM_EINVAL, "precision must be 0, 1 or 2");
  const Schedule sc{schedule->transforms_per_thread, schedule->row_threads, schedule->col_cols,
                    schedule->elems_per_thread};
  if (!schedule_feasible(precision, ctx->logH, ctx->logP, sc))
    return fail(AIM_EINVAL, "schedule cannot be launched for this transform length");
  ctx->sched[precision] = sc;
  return AIM_OK;
}

aim_status aim_get_schedule(const aim_ctx* ctx, int precision, aim_schedule* schedule) {
  if (!ctx || !schedule) return fail(AIM_EINVAL, "bad argument");
  if (precision < AIM_FP64 || precision > AIM_FP64_NATIVE) return fail(AIM_EINVAL, "precision must be 0, 1 or 2");
  const Schedule& sc = ctx->sched[precision];
  *schedule = aim_schedule{sc.tpt, sc.min_row_threads, sc.col_cols, sc.elems == 0 ? 16 : sc.elems};
  return AIM_OK;
}

aim_status aim_autotune(aim_ctx* ctx, int nrhs, int precision, void* stream, aim_schedule* chosen) {
  if (!ctx || nrhs < 1) return fail(AIM_EINVAL, "bad argument");
  if (precision < AIM_FP64 || precision > AIM_FP64_NATIVE) return fail(AIM_EINVAL, "precision must be 0, 1 or 2");
  AIM_TRY(check_device(ctx));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  AIM_TRY(reserve(ctx, nrhs, precision));
  const size_t bytes = (size_t)ctx->n * nrhs * sizeof(double2);
  AIM_TRY(stage(ctx, bytes, bytes));
  AIM_CUDA_TRY(cudaMemsetAsync(ctx->stage_in, 0, bytes, st));
  cudaEvent_t e0, e1;
  AIM_CUDA_TRY(cudaEventCreate(&e0));
  AIM_CUDA_TRY(cudaEventCreate(&e1));
  const Schedule saved = ctx->sched[precision];
  Schedule best = saved;
  float best_ms = 1e30f;
  const int tpts[2] = {1, 2};
  const int rows[3] = {128, 256, 1024};
  const int cols[5] = {0, 1, 2, 4, 8};
  const int elems[2] = {16, 8};
  aim_status s = AIM_OK;
  for (int e = 0; e < 2 && s == AIM_OK; ++e)
  for (int a = 0; a < 2 && s == AIM_OK; ++a)
    for (int b = 0; b < 3 && s == AIM_OK; ++b)
      for (int cc = 0; cc < 5 && s == AIM_OK; ++cc) {
        const Schedule cand{tpts[a], rows[b], cols[cc], elems[e]};
        if (!schedule_feasible(precision, ctx->logH, ctx->logP, cand)) continue;
        ctx->sched[precision] = cand;
        s = apply_op(ctx, AIM_OP_S_ALPHA, nrhs, ctx->stage_in, ctx->stage_out, precision, st);   // warm
        if (s != AIM_OK) break;
        cudaEventRecord(e0, st);
        for (int it = 0; it < 3 && s == AIM_OK; ++it)
          s = apply_op(ctx, AIM_OP_S_ALPHA, nrhs, ctx->stage_in, ctx->stage_out, precision, st);
        cudaEventRecord(e1, st);
        if (cudaEventSynchronize(e1) != cudaSuccess) { s = fail(AIM_ECUDA, "autotune event"); break; }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best_ms) {
          best_ms = ms;
          best = cand;
        }
      }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  ctx->sched[precision] = s == AIM_OK ? best : saved;
  if (chosen) {
    const Schedule& w = ctx->sched[precision];
    *chosen = aim_schedule{w.tpt, w.min_row_threads, w.col_cols, w.elems == 0 ? 16 : w.elems};
  }
  return s;
}

aim_status aim_rhs_planewave(aim_ctx* ctx, int nrhs, const double* angles, void* rhs, void* stream) {
  if (!ctx || !angles || !rhs || nrhs < 1) return fail(AIM_EINVAL, "bad argument");
  AIM_TRY(check_device(ctx));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t bytes = (size_t)ctx->n * nrhs * sizeof(double2);
  AIM_TRY(stage(ctx, std::max(bytes, nrhs * sizeof(double)), bytes));
  double* ang = reinterpret_cast<double*>(ctx->stage_in);
  AIM_CUDA_TRY(cudaMemcpyAsync(ang, angles, nrhs * sizeof(double), cudaMemcpyHostToDevice, st));
  const bool dev = device_pointer(rhs);
  double2* out = dev ? static_cast<double2*>(rhs) : ctx->stage_out;
  AIM_TRY(device_rhs_planewave(ctx, nrhs, ang, out, st));
  if (!dev) {
    AIM_CUDA_TRY(cudaMemcpyAsync(rhs, out, bytes, cudaMemcpyDeviceToHost, st));
    AIM_CUDA_TRY(cudaStreamSynchronize(st));
  } else {
    // the angle upload comes from pageable memory: keep the call synchronous w.r.t. `angles`
    AIM_CUDA_TRY(cudaStreamSynchronize(st));
  }
  return AIM_OK;
}

aim_status aim_matvec(aim_ctx* ctx, aim_op op, int nrhs, const void* x, void* y, int precision, void* stream) {
  if (!ctx || !x || !y || nrhs < 1) return fail(AIM_EINVAL, "bad argument");
  if (precision < AIM_FP64 || precision > AIM_FP64_NATIVE) return fail(AIM_EINVAL, "precision must be 0, 1 or 2");
  if (x == y) return fail(AIM_EINVAL, "x and y must not overlap");
  AIM_TRY(check_device(ctx));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t bytes = (size_t)ctx->n * nrhs * sizeof(double2);
  const bool dx = device_pointer(x), dy = device_pointer(y);
  if (!dx || !dy) AIM_TRY(stage(ctx, bytes, bytes));
  const double2* xin = static_cast<const double2*>(x);
  if (!dx) {
    AIM_CUDA_TRY(cudaMemcpyAsync(ctx->stage_in, x, bytes, cudaMemcpyHostToDevice, st));
    xin = ctx->stage_in;
  }
  double2* yout = dy ? static_cast<double2*>(y) : ctx->stage_out;
  AIM_TRY(apply_op(ctx, op, nrhs, xin, yout, precision, st));
  if (!dy) {
    AIM_CUDA_TRY(cudaMemcpyAsync(y, yout, bytes, cudaMemcpyDeviceToHost, st));
    AIM_CUDA_TRY(cudaStreamSynchronize(st));
  }
  return AIM_OK;
}

aim_status aim_matvec_multi(int count, aim_ctx* const* ctxs, const aim_op* ops, const int* nrhs, const void* const* x,
                            void* const* y, int precision, void* stream) {
  if (count < 1 || count > 32 || !ctxs || !ops || !nrhs || !x || !y) return fail(AIM_EINVAL, "bad argument");
  if (precision < AIM_FP64 || precision > AIM_FP64_NATIVE) return fail(AIM_EINVAL, "precision must be 0, 1 or 2");
  for (int i = 0; i < count; ++i) {
    if (!ctxs[i] || nrhs[i] < 1 || !x[i] || !y[i]) return fail(AIM_EINVAL, "bad argument");
    for (int j = 0; j < i; ++j)
      if (ctxs[j] == ctxs[i]) return fail(AIM_EINVAL, "a context may appear once per multi-context call");
    if (x[i] == y[i]) return fail(AIM_EINVAL, "x and y must not overlap");
    if (!device_pointer(x[i]) || !device_pointer(y[i])) return fail(AIM_EINVAL, "x and y must be device pointers");
    AIM_TRY(check_device(ctxs[i]));
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  MultiLauncher ml;
  aim_status s = apply_op_multi(ml, count, ctxs, ops, nrhs, reinterpret_cast<const double2* const*>(x),
                                reinterpret_cast<double2* const*>(y), precision, st);
  const cudaError_t e = cudaStreamSynchronize(st);
  if (s == AIM_OK && e != cudaSuccess) s = fail(AIM_ECUDA, std::string("multi-context product: ") + cudaGetErrorString(e));
  if (s == AIM_OK) s = ml.check();
  return s;
}

aim_status aim_grid_product(aim_ctx* ctx, int filtered, int nrhs, const void* u, void* v, int precision, void* stream) {
  if (!ctx || !u || !v || nrhs < 1) return fail(AIM_EINVAL, "bad argument");
  if (precision < AIM_FP64 || precision > AIM_FP64_NATIVE) return fail(AIM_EINVAL, "precision must be 0, 1 or 2");
  AIM_TRY(check_device(ctx));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t bytes = (size_t)ctx->m * ctx->m * nrhs * sizeof(double2);
  const bool du = device_pointer(u), dv = device_pointer(v);
  if (!du || !dv) AIM_TRY(stage(ctx, bytes, bytes));
  // workspace for nrhs channels
  const int chan_needed = nrhs;
  AIM_TRY(grow(&ctx->inter, &ctx->inter_bytes, inter_bytes_needed(ctx, chan_needed, precision)));
  const double2* uin = static_cast<const double2*>(u);
  if (!du) {
    AIM_CUDA_TRY(cudaMemcpyAsync(ctx->stage_in, u, bytes, cudaMemcpyHostToDevice, st));
    uin = ctx->stage_in;
  }
  double2* vout = dv ? static_cast<double2*>(v) : ctx->stage_out;
  void* in = ctx->inter;
  const size_t ib = ctx->inter_bytes;
  if (precision == AIM_MIXED) AIM_TRY(grid_product_dense<float2>(ctx, filtered != 0, nrhs, uin, vout, in, ib, st));
  else if (precision == AIM_FP64_NATIVE) AIM_TRY(grid_product_dense<double2>(ctx, filtered != 0, nrhs, uin, vout, in, ib, st));
  else AIM_TRY(grid_product_dense<dfc>(ctx, filtered != 0, nrhs, uin, vout, in, ib, st));
  if (!dv) {
    AIM_CUDA_TRY(cudaMemcpyAsync(v, vout, bytes, cudaMemcpyDeviceToHost, st));
    AIM_CUDA_TRY(cudaStreamSynchronize(st));
  }
  return AIM_OK;
}

aim_status aim_solve(aim_ctx* ctx, aim_op system, int nrhs, const void* rhs, void* x, int x0_given,
                     const aim_solve_opts* opts, aim_solve_info* info, void* stream) {
  if (!ctx || !rhs || !x || !opts || nrhs < 1) return fail(AIM_EINVAL, "bad argument");
  if (!(opts->tol > 0.0) || opts->restart < 1 || opts->restart > 10000 || opts->max_iter < 1)
    return fail(AIM_EINVAL, "bad solver options");
  if (opts->precision < AIM_FP64 || opts->precision > AIM_FP64_NATIVE) return fail(AIM_EINVAL, "bad precision");
  const bool te = ctx->form == AIM_TE_P1_GALERKIN;
  const bool calderon =
      system == AIM_OP_CALDERON || system == AIM_OP_CALDERON_ALPHA || system == AIM_OP_CALDERON_ALPHA2;
  if (system != AIM_OP_EFIE && system != AIM_OP_EFIE_ALPHA && !calderon)
    return fail(AIM_EINVAL, "system must be EFIE, EFIE_ALPHA, CALDERON, CALDERON_ALPHA or CALDERON_ALPHA2");
  if (!te && calderon)
    return fail(AIM_ESTATE, "Calderon systems need a TE context");
  if (te && system == AIM_OP_EFIE_ALPHA) return fail(AIM_ESTATE, "filtered EFIE system is TM only");
  AIM_TRY(check_device(ctx));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t bytes = (size_t)ctx->n * nrhs * sizeof(double2);
  const bool dr = device_pointer(rhs), dx = device_pointer(x);
  AIM_TRY(reserve(ctx, nrhs, AIM_FP64));
  if (opts->precision != AIM_FP64) AIM_TRY(reserve(ctx, nrhs, opts->precision));
  AIM_TRY(stage(ctx, bytes, bytes));
  // b lives in stage_in (for Calderon systems: G^-1 S G^-1 E); x in place or staged
  double2* b = ctx->stage_in;
  double2* xd = dx ? static_cast<double2*>(x) : ctx->stage_out;
  if (dr) AIM_CUDA_TRY(cudaMemcpyAsync(b, rhs, bytes, cudaMemcpyDeviceToDevice, st));
  else AIM_CUDA_TRY(cudaMemcpyAsync(b, rhs, bytes, cudaMemcpyHostToDevice, st));
  if (x0_given) {
    if (!dx) AIM_CUDA_TRY(cudaMemcpyAsync(xd, x, bytes, cudaMemcpyHostToDevice, st));
  } else {
    AIM_CUDA_TRY(cudaMemsetAsync(xd, 0, bytes, st));
  }
  if (calderon) {
    // b <- G^-1 S G^-1 E, with S^alpha for the filtered systems (Eq. 3)
    double2* t1 = ctx->vec_ws;
    double2* t2 = ctx->vec_ws + (size_t)nrhs * ctx->n;
    AIM_TRY(gram_inv_apply(ctx, nrhs, b, t1, st));
    AIM_TRY(apply_op(ctx, system == AIM_OP_CALDERON ? AIM_OP_S : AIM_OP_S_ALPHA, nrhs, t1, t2, AIM_FP64, st));
    AIM_TRY(gram_inv_apply(ctx, nrhs, t2, b, st));
  }
  aim_status s = gmres_solve(ctx, system, nrhs, b, xd, opts, info, st);
  if (!dx) {
    AIM_CUDA_TRY(cudaMemcpyAsync(x, xd, bytes, cudaMemcpyDeviceToHost, st));
  }
  AIM_CUDA_TRY(cudaStreamSynchronize(st));
  return s;
}

// Device bytes of one cudaMalloc of `b` bytes as the allocator commits them (2 MiB pages).
static size_t committed(size_t b) {
  constexpr size_t kPage = (size_t)2 << 20;
  return b == 0 ? 0 : (b + kPage - 1) / kPage * kPage;
}

// Exact sizes of what aim_setup and aim_reserve(nrhs, precision) allocate, from the host-side
// setup (active grid points, projection lists, near-field pattern, Gram band), each allocation
// counted in whole allocator pages, plus the largest set of setup temporaries alive at once.
static aim_status query_context_bytes(const aim_geometry* geometry, const aim_grid* grid, const aim_stencil* stencil,
                                      int nrhs, int precision, size_t* bytes) {
  if (!geometry || !grid || !stencil || !bytes || nrhs < 1) return fail(AIM_EINVAL, "bad argument");
  if (precision < AIM_FP64 || precision > AIM_FP64_NATIVE) return fail(AIM_EINVAL, "precision must be 0, 1 or 2");
  // k and the filter do not change any size: validate with placeholders
  AIM_TRY(validate_setup(geometry, 1.0, grid, stencil, nullptr));
  aim_ctx tmp;
  AIM_TRY(derive_params(&tmp, geometry, 1.0, grid, stencil, nullptr));
  HostSetup hs;
  AIM_TRY(host_setup(&tmp, &hs));
  const bool te = tmp.form == AIM_TE_P1_GALERKIN;
  const size_t n = tmp.n, m = tmp.m, P = tmp.P, H = tmp.H, nact = hs.n_act;
  const size_t nrows = (size_t)(hs.row_hi - hs.row_lo + 1);
  const size_t nsc = hs.sc_col.size(), nga = hs.ga_act.size();
  const size_t nnz = hs.near_col.size(), nq = (H + 1) * (H + 1);
  size_t b = 0;
  // persistent arrays of the context
  b += committed(n * 16);                                        // vertices
  b += committed((m + 1) * 4) + committed(nact * 4);             // row_ptr, act_ix
  b += committed((nact + 1) * 4) + committed(nsc * 4);           // scatter CSR
  b += committed((n + 1) * 4) + committed(nga * 4);              // gather CSR
  b += hs.nproj * (committed(nsc * 8) + committed(nga * 8));     // projection weights
  b += committed(P * 16) + committed(P * 8) + committed(P * 16); // twiddles
  b += committed(hs.gram_inv.size() * 8);
  const size_t nvals = te ? 2 : 1;
  if (nnz > 0) b += committed((n + 1) * 4) + committed(nnz * 4) + nvals * (committed(nnz * 16) + committed(nnz * 8));
  b += 2 * (committed(nq * 16) + committed(nq * 8) + committed(nq * 16)) + committed((H + 1) * 4);   // spectra
  // setup temporaries (freed before aim_setup returns)
  size_t t = committed(nq * 16);                                 // kernel samples
  if (nnz > 0) {
    t += committed(nact * 4);
    if (te) {
      const size_t npairs = hs.seg_e.size();
      t += 2 * committed(npairs * 4) + committed(nnz * 4 * 4) + committed(npairs * 4 * 16);
    } else {
      t += committed((n + 1) * 4) + committed(hs.sr_act.size() * 4) + committed(hs.sr_w.size() * 8);
    }
  }
  b += t;
  // grid workspaces of aim_reserve(nrhs, precision)
  const size_t chan = (size_t)(te ? 3 : 1) * nrhs;
  const size_t el = precision == AIM_MIXED ? 8 : 16;
  b += committed(chan * P * nrows * el) + committed(chan * nact * el) + committed(2 * (size_t)nrhs * n * 16);
  *bytes = b;
  return AIM_OK;
}

aim_status aim_query_bytes(const aim_geometry* geometry, const aim_grid* grid, const aim_stencil* stencil, int nrhs,
                           int precision, size_t* bytes) {
  return query_context_bytes(geometry, grid, stencil, nrhs, precision, bytes);
}

aim_status aim_query_solve_bytes(const aim_geometry* geometry, const aim_grid* grid, const aim_stencil* stencil,
                                 int nrhs, const aim_solve_opts* opts, size_t* bytes) {
  if (!opts || !bytes || nrhs < 1) return fail(AIM_EINVAL, "bad argument");
  if (opts->restart < 1 || opts->restart > 10000) return fail(AIM_EINVAL, "restart must be in 1..10000");
  if (opts->precision < AIM_FP64 || opts->precision > AIM_FP64_NATIVE) return fail(AIM_EINVAL, "bad precision");
  // every solve reserves the FP64 grid workspaces (the largest), the mixed one as well
  size_t b = 0;
  AIM_TRY(query_context_bytes(geometry, grid, stencil, nrhs, AIM_FP64, &b));
  const size_t n = geometry->n_seg;
  b += 2 * committed(n * nrhs * 16);                                  // staging of b and x
  b += committed(krylov_bytes(n, nrhs, opts->restart)) + committed(reduction_bytes(nrhs, opts->restart));
  if (opts->precision == AIM_MIXED) b += committed(2 * n * nrhs * 16);   // residual and correction
  *bytes = b;
  return AIM_OK;
}

}  // extern "C"
