// Internal declarations shared by the translation units of the AIM library.
#pragma once

#include <cuda_runtime.h>
#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/aim.h"

namespace aim {

struct dfc;   // double-float complex (dfloat.cuh)

// ------------------------------------------------------------------------------------
// error plumbing
// ------------------------------------------------------------------------------------
void set_error(const std::string& msg);
aim_status fail(aim_status st, const std::string& msg);
}  // namespace aim
struct aim_ctx;
namespace aim {
// AIM_EINVAL unless the calling thread's current CUDA device is the one the context was set up on
// (every array of a context lives on that device)
aim_status check_device(const aim_ctx* ctx);

#define AIM_CUDA_TRY(expr)                                                              \
  do {                                                                                  \
    cudaError_t e__ = (expr);                                                           \
    if (e__ != cudaSuccess) {                                                           \
      return ::aim::fail(e__ == cudaErrorMemoryAllocation ? AIM_ENOMEM : AIM_ECUDA,     \
                         std::string(#expr) + ": " + cudaGetErrorString(e__));          \
    }                                                                                   \
  } while (0)

#define AIM_TRY(expr)                      \
  do {                                     \
    aim_status s__ = (expr);               \
    if (s__ != AIM_OK) return s__;         \
  } while (0)

// ------------------------------------------------------------------------------------
// launch accounting (prof.cu): construct a ProfScope around every kernel launch
// ------------------------------------------------------------------------------------
enum KernelId {
  K_ROW_FWD = 0, K_COL_CONV, K_ROW_INV, K_GATHER, K_GRAM,
  K_SETUP_SAMPLE, K_SETUP_DFT, K_SETUP_PACK, K_SETUP_SEGPAIRS, K_SETUP_NEAR,
  K_RHS, K_GMRES, K_MULTI, K_DFT_STAGE, K_COUNT
};
void count_launches(int id, int n);   // counted, not timed
void thread_launch_counts(long long* out);   // this host thread's counts, K_COUNT entries
bool profiling_active();
struct ProfScope {
  // count_launch = false: a timing-only scope around a group of launches counted elsewhere
  ProfScope(int id, cudaStream_t st, bool count_launch = true);
  ~ProfScope();
  int id;
  cudaStream_t st;
  int slot;
};

// ------------------------------------------------------------------------------------
// sizes
// ------------------------------------------------------------------------------------
constexpr int kMaxP = 4096;          // largest embedding side (FFT length)
constexpr int kMinP = 64;            // smallest: every half-length transform has >= 2 passes
constexpr int kMaxProj = 4;          // TE: phi, phi', n_x phi, n_y phi
constexpr int kGramBand = 40;        // half bandwidth of the banded G^-1 for large N
constexpr int kGramDenseMax = 512;   // N at or below which G^-1 is stored dense

// column-tile width of the intermediate layout (32-byte chunks)
template <typename T> struct TileW;
template <> struct TileW<double> { static constexpr int value = 2; };
template <> struct TileW<float> { static constexpr int value = 4; };

template <typename T> struct Cplx;
template <> struct Cplx<double> { using type = double2; };
template <> struct Cplx<float> { using type = float2; };

// ------------------------------------------------------------------------------------
// device-side arrays of one context
// ------------------------------------------------------------------------------------
struct Projections {
  // scatter side, grid-point-major CSR over the active points: u[a] = sum w * x[col]
  int* sc_ptr = nullptr;   // n_act + 1
  int* sc_col = nullptr;   // hat / segment index
  double* sc_w[kMaxProj] = {};
  // gather side, unknown-major CSR: y[i] = sum w * v[act]
  int* ga_ptr = nullptr;   // n + 1
  int* ga_act = nullptr;   // active point index
  double* ga_w[kMaxProj] = {};
  int nproj = 0;
};

struct NearField {
  int* ptr = nullptr;      // n + 1
  int* col = nullptr;
  double2* val[2] = {};    // TE: [0] correction of S, [1] correction of N ; TM: [0] of S
  float2* valf[2] = {};
  long long nnz = 0;
};

// Launch schedule of the grid kernels for one precision: transforms per thread (1: even/odd
// halves in adjacent lanes, 2: both in one thread), the minimum threads of a row-pass CTA, the
// columns of a column-pass CTA (0: the fewest whole tiles that give 128 threads), and the
// elements each thread owns per transform (16 or 8; 0 means 16).
struct Schedule {
  int tpt;
  int min_row_threads;
  int col_cols;
  int elems;
};

// Whether a schedule can be launched for a context whose transforms have length H = 2^logH
// (checks the launch bounds and the shared-memory limit; precision selects the element type).
bool schedule_feasible(int precision, int logH, int logP, const Schedule& s);

// operator selection for one batched grid pass
struct PassSpec {
  int nproj;                       // projections applied to each rhs (N: 3, S: 1)
  int proj[kMaxProj];              // which projection weights
  double2 coef[kMaxProj];          // gather coefficient per projection
  bool filtered;                   // spectrum choice
  const NearField* near;           // near-field correction (nullptr: none)
  int near_which;                  // which near value array
  double2 out_scale;               // overall factor on the gathered result
};

}  // namespace aim

struct aim_ctx {
  // problem
  int form = 0;
  int n = 0, m = 0, P = 0, H = 0, logH = 0, logP = 0, s = 0, p = 0;
  double k = 0, L = 0, eps = 0, alpha = 0, near_radius = 0;
  int filter_enabled = 0;
  int device = 0;
  // active grid set
  int n_act = 0, row_lo = 0, row_hi = -1, nrows = 0;
  int* row_ptr = nullptr;   // m + 1 : active points of grid row iy are [row_ptr[iy], row_ptr[iy+1])
  int* act_ix = nullptr;    // n_act : column index of each active point
  aim::Projections prj;
  aim::NearField near;
  // spectra, (H+1) x (H+1) each, per column q' = 0..H: [even part (H/2+1) | odd part (H/2)]
  double2* specU = nullptr;
  double2* specA = nullptr;
  float2* specUf = nullptr;
  float2* specAf = nullptr;
  float4* specUdf = nullptr;   // double-float copies (re hi, re lo, im hi, im lo)
  float4* specAdf = nullptr;
  // per column q' = 0..H of the filtered spectrum: 0 when the mask zeroes the whole column
  int* specA_live = nullptr;
  double2* tw = nullptr;    // e^{-2 pi i t / P}, t < P
  float2* twf = nullptr;
  float4* twdf = nullptr;
  // Gram inverse, row i: entries for columns (i + d) mod n, d = -band..band
  double* gram_inv = nullptr;
  int gram_band = 0;
  // entry counts of the scatter and gather lists and of gram_inv (for aim_export_setup)
  size_t n_sc = 0, n_ga = 0, n_gram = 0;
  // geometry: host copy and device vertices
  std::vector<double> xy;
  double2* nodes = nullptr;
  // workspaces (grown by reserve)
  void* inter = nullptr; size_t inter_bytes = 0;
  void* vact = nullptr; size_t vact_bytes = 0;
  double2* vec_ws = nullptr; size_t vec_ws_bytes = 0;  // temporaries for composite operators
  double2* stage_in = nullptr; double2* stage_out = nullptr; size_t stage_bytes = 0;
  double2* kry = nullptr; size_t kry_bytes = 0;        // GMRES workspace
  double* red = nullptr; size_t red_bytes = 0;          // reduction scratch (dot products)
  double* red_host = nullptr; size_t red_host_bytes = 0;
  int reserved_rhs[3] = {0, 0, 0};   // per precision (AIM_FP64, AIM_MIXED, AIM_FP64_NATIVE)
  // launch schedule per precision; defaults measured on GB300, aim_autotune re-measures
  // defaults: measured at the single-solve scale (2048^2 grid, P = 4096), feasible at every P
  aim::Schedule sched[3] = {{2, 128, 0, 8}, {2, 128, 0, 16}, {2, 128, 0, 16}};
  // bookkeeping
  std::vector<void*> allocations;
  size_t device_bytes = 0;
  double setup_seconds = 0;
  long long nnz_near = 0;
};

namespace aim {

// allocation helpers (tracked by the context)
aim_status dev_alloc(aim_ctx* ctx, void** p, size_t bytes);
template <typename T>
aim_status dev_alloc_t(aim_ctx* ctx, T** p, size_t count) {
  return dev_alloc(ctx, reinterpret_cast<void**>(p), count * sizeof(T));
}
template <typename T>
aim_status upload(aim_ctx* ctx, T** p, const std::vector<T>& h, cudaStream_t st) {
  if (h.empty()) { *p = nullptr; return AIM_OK; }
  AIM_TRY(dev_alloc_t(ctx, p, h.size()));
  AIM_CUDA_TRY(cudaMemcpyAsync(*p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, st));
  return AIM_OK;
}

// ------------------------------------------------------------------------------------
// host-side setup products (setup_host.cpp)
// ------------------------------------------------------------------------------------
struct HostSetup {
  // segments
  std::vector<double> dx, dy, h, tx, ty, nx, ny;
  // Gauss rule on [0,1]
  std::vector<double> gx, gw;
  // active points
  int n_act = 0, row_lo = 0, row_hi = -1;
  std::vector<int> row_ptr, act_ix, act_iy;
  // scatter / gather CSR
  std::vector<int> sc_ptr, sc_col, ga_ptr, ga_act;
  std::vector<double> sc_w[kMaxProj], ga_w[kMaxProj];
  int nproj = 0;
  // TM only: source projection per segment (the TE source list is the gather list)
  std::vector<int> sr_ptr, sr_act;
  std::vector<double> sr_w;
  // near field: unknown pairs (CSR rows) and the segment pairs they need
  std::vector<int> near_ptr, near_col;
  std::vector<int> seg_e, seg_f;          // unique segment pairs (TE) or point-segment pairs (TM)
  std::vector<int> pair_seg_idx;          // TE: 4 per near entry (e=i,f=j),(i,j-1),(i-1,j),(i-1,j-1); TM: 1
  // Gram inverse
  std::vector<double> gram_inv;
  int gram_band = 0;
  // twiddles
  std::vector<double> tw;                 // 2*P
};

aim_status host_setup(aim_ctx* ctx, HostSetup* hs);
// argument checks of aim_setup, and the context's sizes and grid parameters from them (host only)
aim_status validate_setup(const aim_geometry* g, double k, const aim_grid* grid, const aim_stencil* st,
                          const aim_filter* f);
aim_status derive_params(aim_ctx* ctx, const aim_geometry* geometry, double k, const aim_grid* grid,
                         const aim_stencil* stencil, const aim_filter* filter);
// FP64, complex64 and double-float twiddle tables of ctx->P from 2P doubles (re, im)
aim_status upload_twiddles(aim_ctx* ctx, const double* tw2, cudaStream_t st);
double host_grid_half_side(const double* xy, int n, int m, int s);
void gauss_legendre01(int n, std::vector<double>* x, std::vector<double>* w);

// ------------------------------------------------------------------------------------
// device setup (setup_kernels.cu)
// ------------------------------------------------------------------------------------
// kernel samples -> near-field entries -> spectrum F(c) and its truncation (in that order)
aim_status device_spectra_and_near(aim_ctx* ctx, const HostSetup& hs, cudaStream_t st);
// the grid kernel tables of aim_kernel_table (natural order, (H+1)^2 complex128, device `out`)
aim_status kernel_table(aim_ctx* ctx, int which, double2* out, cudaStream_t st);
// f[i] = complex64 rounding of src[i]; df[i] = its double-float split (hi, lo per part), when
// df is not null: the derived copies aim_setup makes of each FP64 spectrum and near-field value
aim_status derive_narrow_copies(const double2* src, size_t count, float2* f, float4* df, cudaStream_t st);
aim_status device_rhs_planewave(aim_ctx* ctx, int nrhs, const double* angles_dev, double2* out, cudaStream_t st);

// ------------------------------------------------------------------------------------
// matvec pipeline (matvec_kernels.cu)
// ------------------------------------------------------------------------------------
// y[r] (+)= op(x[r]) for r < nrhs, FP64 vectors; T selects the grid arithmetic
template <typename T>
aim_status grid_pass(aim_ctx* ctx, const PassSpec& spec, int nrhs, const double2* x, double2* y,
                     cudaStream_t st);
// the grid product on full m x m grids with an explicit intermediate buffer (inter, inter_bytes)
template <typename T>
aim_status grid_product_dense(aim_ctx* ctx, bool filtered, int nrhs, const double2* u, double2* v, void* inter,
                              size_t inter_bytes, cudaStream_t st);
aim_status gram_inv_apply(aim_ctx* ctx, int nrhs, const double2* x, double2* y, cudaStream_t st);
size_t inter_bytes_needed(const aim_ctx* ctx, int channels, int precision);

// several grid passes of several contexts in one persistent launch (matvec_kernels.cuh)
struct MultiPassSpec {   // one pass of a multi launch, as the caller describes it
  aim_ctx* ctx;
  PassSpec spec;
  int nrhs;
  const double2* x;
  double2* y;
};
template <typename T>
aim_status grid_pass_multi(const MultiPassSpec* passes, int count, unsigned* scratch, int* err_host, cudaStream_t st);

// full operator application with composition (capi.cu)
aim_status apply_op(aim_ctx* ctx, aim_op op, int nrhs, const double2* x, double2* y, int precision,
                    cudaStream_t st);
aim_status reserve(aim_ctx* ctx, int nrhs, int precision);

// Buffers of a multi-context launch: the barrier words and the error flags of its stages
// (pinned). Owned by one caller at a time.
struct MultiLauncher {
  unsigned* scratch = nullptr;   // 4 words per stage
  int* err_host = nullptr;       // one flag per stage (pinned)
  aim_status init();
  aim_status check();            // after a synchronisation: AIM_ETIMEOUT if a launch gave up
  ~MultiLauncher();
};
// y_i = A_i x_i for `count` contexts (device vectors), every grid pass stage of all of them in one
// persistent launch; composite operators run stage by stage (Eq. 3). Asynchronous on `st`.
aim_status apply_op_multi(MultiLauncher& ml, int count, aim_ctx* const* ctxs, const aim_op* ops, const int* nrhs,
                          const double2* const* x, double2* const* y, int precision, cudaStream_t st);

// ------------------------------------------------------------------------------------
// batched products of concurrent solves (batcher.cu)
// ------------------------------------------------------------------------------------
}  // namespace aim
struct aim_batcher;
namespace aim {
// the batcher attached to the calling thread by aim_solve_batched (nullptr outside it)
aim_batcher* current_batcher();
// y = A x for one solve, fused with the products that other solves of the batcher submit at about
// the same time; asynchronous: `st` waits for the result on the device
aim_status batcher_product(aim_batcher* b, aim_ctx* ctx, aim_op op, int nrhs, const double2* x, double2* y,
                           int precision, cudaStream_t st);

// ------------------------------------------------------------------------------------
// GMRES (solver.cu)
// ------------------------------------------------------------------------------------
aim_status gmres_solve(aim_ctx* ctx, aim_op system, int nrhs, const double2* b, double2* x,
                       const aim_solve_opts* opts, aim_solve_info* info, cudaStream_t st);
// device bytes of the GMRES workspaces for n unknowns, nrhs vectors and a restart length
size_t krylov_bytes(size_t n, int nrhs, int restart);
size_t reduction_bytes(int nrhs, int restart);

}  // namespace aim
