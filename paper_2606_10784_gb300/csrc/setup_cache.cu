// Setup blobs: what aim_setup computes (projections of Eq. 7, G^-1 of Eq. 3, the near-field
// correction, the kernel spectrum and its truncation of Eq. 10) saved to host memory and
// reloaded, so that a restarted process skips the setup. The key and the checksum are
// FNV-1a (Fowler, Noll, Vo), the checksum taken over 64-bit words in four interleaved lanes.
#include <chrono>
#include <cstdint>
#include <cstring>
#include <new>
#include <vector>

#include "aim_internal.h"

namespace aim {
namespace {

constexpr char kMagic[8] = {'A', 'I', 'M', 'S', 'E', 'T', 'U', 'P'};
constexpr uint32_t kVersion = 1;
constexpr uint64_t kFnvBasis = 14695981039346656037ull;
constexpr uint64_t kFnvPrime = 1099511628211ull;

struct BlobHeader {
  char magic[8];
  uint32_t version;
  uint32_t header_bytes;
  uint64_t key;
  uint64_t payload_bytes;
  uint64_t checksum;
  // the problem (compared bit for bit with the importer's derived parameters)
  int32_t form, n, m, P, s, p, filter_kind, nproj;
  double k, L, eps, alpha, near_radius;
  // the setup's sizes
  int32_t n_act, row_lo, row_hi, gram_band;
  int64_t n_sc, n_ga, n_gram, nnz;
};
static_assert(sizeof(BlobHeader) == 160, "setup blob header layout");

struct Fnv {
  uint64_t h = kFnvBasis;
  void bytes(const void* p, size_t n) {
    const unsigned char* b = static_cast<const unsigned char*>(p);
    for (size_t i = 0; i < n; ++i) h = (h ^ b[i]) * kFnvPrime;
  }
  template <typename T>
  void val(T v) { bytes(&v, sizeof(T)); }
};

uint64_t problem_key(const aim_ctx& c) {
  Fnv f;
  f.bytes("aim-setup-key", 13);
  f.val<uint32_t>(kVersion);
  for (int32_t v : {c.form, c.n, c.m, c.P, c.s, c.p, c.filter_enabled}) f.val(v);
  for (double v : {c.k, c.L, c.eps, c.alpha, c.near_radius}) f.val(v);
  f.bytes(c.xy.data(), c.xy.size() * sizeof(double));
  return f.h;
}

// payload_bytes is a multiple of 16 by construction
uint64_t payload_checksum(const unsigned char* p, size_t bytes) {
  uint64_t lane[4] = {kFnvBasis, kFnvBasis ^ 1, kFnvBasis ^ 2, kFnvBasis ^ 3};
  const size_t words = bytes / 8;
  size_t i = 0;
  for (; i + 4 <= words; i += 4) {
    uint64_t w[4];
    std::memcpy(w, p + 8 * i, 32);
    for (int l = 0; l < 4; ++l) lane[l] = (lane[l] ^ w[l]) * kFnvPrime;
  }
  for (; i < words; ++i) {
    uint64_t w;
    std::memcpy(&w, p + 8 * i, 8);
    lane[i & 3] = (lane[i & 3] ^ w) * kFnvPrime;
  }
  Fnv f;
  for (uint64_t l : lane) f.val(l);
  f.val<uint64_t>(bytes);
  return f.h;
}

// One array of the payload: the context field it belongs to, its element size and count.
struct Section {
  void** slot;
  size_t elem;
  size_t count;
  size_t offset = 0;   // from the payload's start, a multiple of 16
};

enum SectionId { SEC_NODES = 0, SEC_ROW_PTR, SEC_ACT_IX, SEC_SC_PTR, SEC_SC_COL, SEC_GA_PTR, SEC_GA_ACT };

// The payload's arrays in order, for a context whose counts are set. Returns the payload size.
size_t layout(aim_ctx* c, int nproj, long long nnz, std::vector<Section>* out) {
  auto& v = *out;
  v.clear();
  const size_t n = c->n, nq = (size_t)(c->H + 1) * (c->H + 1);
  v.push_back({reinterpret_cast<void**>(&c->nodes), sizeof(double2), n});
  v.push_back({reinterpret_cast<void**>(&c->row_ptr), sizeof(int), (size_t)c->m + 1});
  v.push_back({reinterpret_cast<void**>(&c->act_ix), sizeof(int), (size_t)c->n_act});
  v.push_back({reinterpret_cast<void**>(&c->prj.sc_ptr), sizeof(int), (size_t)c->n_act + 1});
  v.push_back({reinterpret_cast<void**>(&c->prj.sc_col), sizeof(int), c->n_sc});
  v.push_back({reinterpret_cast<void**>(&c->prj.ga_ptr), sizeof(int), n + 1});
  v.push_back({reinterpret_cast<void**>(&c->prj.ga_act), sizeof(int), c->n_ga});
  for (int q = 0; q < nproj; ++q) {
    v.push_back({reinterpret_cast<void**>(&c->prj.sc_w[q]), sizeof(double), c->n_sc});
    v.push_back({reinterpret_cast<void**>(&c->prj.ga_w[q]), sizeof(double), c->n_ga});
  }
  v.push_back({reinterpret_cast<void**>(&c->tw), sizeof(double2), (size_t)c->P});
  v.push_back({reinterpret_cast<void**>(&c->gram_inv), sizeof(double), c->n_gram});
  if (nnz > 0) {
    v.push_back({reinterpret_cast<void**>(&c->near.ptr), sizeof(int), n + 1});
    v.push_back({reinterpret_cast<void**>(&c->near.col), sizeof(int), (size_t)nnz});
    const int nvals = c->form == AIM_TE_P1_GALERKIN ? 2 : 1;
    for (int k = 0; k < nvals; ++k)
      v.push_back({reinterpret_cast<void**>(&c->near.val[k]), sizeof(double2), (size_t)nnz});
  }
  v.push_back({reinterpret_cast<void**>(&c->specU), sizeof(double2), nq});
  v.push_back({reinterpret_cast<void**>(&c->specA), sizeof(double2), nq});
  v.push_back({reinterpret_cast<void**>(&c->specA_live), sizeof(int), (size_t)c->H + 1});
  size_t off = 0;
  for (Section& sct : v) {
    sct.offset = off;
    off += (sct.elem * sct.count + 15) & ~size_t(15);
  }
  return off;
}

// A CSR row pointer: starts at 0, never decreases, ends at `total`.
bool csr_ok(const int* ptr, size_t rows, long long total) {
  if (ptr[0] != 0) return false;
  for (size_t i = 0; i < rows; ++i)
    if (ptr[i + 1] < ptr[i]) return false;
  return ptr[rows] == total;
}

bool all_below(const int* idx, size_t count, int bound) {
  for (size_t i = 0; i < count; ++i)
    if (idx[i] < 0 || idx[i] >= bound) return false;
  return true;
}

template <typename T>
bool same_bits(T a, T b) { return std::memcmp(&a, &b, sizeof(T)) == 0; }

}  // namespace
}  // namespace aim

using namespace aim;

extern "C" {

aim_status aim_setup_key(const aim_geometry* geometry, double k, const aim_grid* grid, const aim_stencil* stencil,
                         const aim_filter* filter, unsigned long long* key) {
  if (!key) return fail(AIM_EINVAL, "key is null");
  AIM_TRY(validate_setup(geometry, k, grid, stencil, filter));
  aim_ctx c;
  AIM_TRY(derive_params(&c, geometry, k, grid, stencil, filter));
  *key = problem_key(c);
  return AIM_OK;
}

aim_status aim_export_setup(const aim_ctx* ctx_in, void* buf, size_t* bytes, void* stream) {
  if (!ctx_in || !bytes) return fail(AIM_EINVAL, "null argument");
  aim_ctx* ctx = const_cast<aim_ctx*>(ctx_in);   // layout() only reads the fields it names
  std::vector<Section> secs;
  const size_t payload = layout(ctx, ctx->prj.nproj, ctx->near.nnz, &secs);
  const size_t total = sizeof(BlobHeader) + payload;
  if (buf == nullptr) {
    *bytes = total;
    return AIM_OK;
  }
  if (*bytes < total) return fail(AIM_EINVAL, "buffer smaller than the setup blob (" + std::to_string(total) + " bytes)");
  AIM_TRY(check_device(ctx));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  unsigned char* out = static_cast<unsigned char*>(buf);
  unsigned char* pay = out + sizeof(BlobHeader);
  for (const Section& s : secs) {
    const size_t len = s.elem * s.count, padded = (len + 15) & ~size_t(15);
    if (len > 0) AIM_CUDA_TRY(cudaMemcpyAsync(pay + s.offset, *s.slot, len, cudaMemcpyDeviceToHost, st));
    if (padded > len) std::memset(pay + s.offset + len, 0, padded - len);
  }
  AIM_CUDA_TRY(cudaStreamSynchronize(st));
  BlobHeader h;
  std::memset(&h, 0, sizeof(h));
  std::memcpy(h.magic, kMagic, sizeof(kMagic));
  h.version = kVersion;
  h.header_bytes = sizeof(BlobHeader);
  h.key = problem_key(*ctx);
  h.payload_bytes = payload;
  h.checksum = payload_checksum(pay, payload);
  h.form = ctx->form; h.n = ctx->n; h.m = ctx->m; h.P = ctx->P; h.s = ctx->s; h.p = ctx->p;
  h.filter_kind = ctx->filter_enabled; h.nproj = ctx->prj.nproj;
  h.k = ctx->k; h.L = ctx->L; h.eps = ctx->eps; h.alpha = ctx->alpha; h.near_radius = ctx->near_radius;
  h.n_act = ctx->n_act; h.row_lo = ctx->row_lo; h.row_hi = ctx->row_hi; h.gram_band = ctx->gram_band;
  h.n_sc = (int64_t)ctx->n_sc; h.n_ga = (int64_t)ctx->n_ga; h.n_gram = (int64_t)ctx->n_gram; h.nnz = ctx->near.nnz;
  std::memcpy(out, &h, sizeof(h));
  *bytes = total;
  return AIM_OK;
}

aim_status aim_import_setup(const aim_geometry* geometry, double k, const aim_grid* grid, const aim_stencil* stencil,
                            const aim_filter* filter, const void* blob, size_t bytes, void* stream, aim_ctx** out) {
  if (!out) return fail(AIM_EINVAL, "out is null");
  *out = nullptr;
  if (!blob) return fail(AIM_EINVAL, "blob is null");
  AIM_TRY(validate_setup(geometry, k, grid, stencil, filter));
  const auto t0 = std::chrono::steady_clock::now();
  if (bytes < sizeof(BlobHeader)) return fail(AIM_EINVAL, "too short to be a setup blob");
  BlobHeader h;
  std::memcpy(&h, blob, sizeof(h));
  if (std::memcmp(h.magic, kMagic, sizeof(kMagic)) != 0) return fail(AIM_EINVAL, "not a setup blob (bad magic)");
  if (h.version != kVersion || h.header_bytes != sizeof(BlobHeader))
    return fail(AIM_EINVAL, "setup blob of another format version (" + std::to_string(h.version) + ")");
  if (h.payload_bytes != bytes - sizeof(BlobHeader)) return fail(AIM_EINVAL, "setup blob truncated or padded");

  aim_ctx* ctx = new (std::nothrow) aim_ctx();
  if (!ctx) return fail(AIM_ENOMEM, "context allocation");
  struct Guard {
    aim_ctx* c;
    ~Guard() { if (c) aim_destroy(c); }
  } guard{ctx};
  AIM_TRY(derive_params(ctx, geometry, k, grid, stencil, filter));

  // the problem: every parameter the setup depends on, bit for bit
  const bool te = ctx->form == AIM_TE_P1_GALERKIN;
  const char* differs = nullptr;
  if (h.form != ctx->form) differs = "form";
  else if (h.n != ctx->n) differs = "n_seg";
  else if (h.m != ctx->m) differs = "m";
  else if (h.P != ctx->P) differs = "fft_P";
  else if (h.s != ctx->s) differs = "stencil s";
  else if (h.p != ctx->p) differs = "quad_p";
  else if (h.filter_kind != ctx->filter_enabled) differs = "filter kind";
  else if (!same_bits(h.k, ctx->k)) differs = "k";
  else if (!same_bits(h.L, ctx->L)) differs = "grid half side L";
  else if (!same_bits(h.eps, ctx->eps)) differs = "grid spacing";
  else if (!same_bits(h.alpha, ctx->alpha)) differs = "filter radius alpha";
  else if (!same_bits(h.near_radius, ctx->near_radius)) differs = "near radius";
  if (differs) return fail(AIM_EINVAL, std::string("setup blob made for another problem: ") + differs + " differs");
  // the setup's sizes: consistent with the problem and with the blob's length
  const int n = ctx->n, m = ctx->m;
  const long long gram_expect = !te ? 0 : n <= kGramDenseMax ? (long long)n * n : (long long)n * (2 * kGramBand + 1);
  const int band_expect = !te ? 0 : n <= kGramDenseMax ? n / 2 : kGramBand;
  if (h.nproj != (te ? 4 : 1) || h.n_act < 1 || (long long)h.n_act > (long long)m * m || h.row_lo < 0 ||
      h.row_hi < h.row_lo || h.row_hi >= m || h.n_sc < 0 || h.n_ga < 0 || h.nnz < 0 || h.n_gram != gram_expect ||
      h.gram_band != band_expect || h.n_sc > (long long)bytes || h.n_ga > (long long)bytes || h.nnz > (long long)bytes)
    return fail(AIM_EINVAL, "setup blob holds inconsistent sizes");
  ctx->n_act = h.n_act;
  ctx->row_lo = h.row_lo;
  ctx->row_hi = h.row_hi;
  ctx->nrows = h.row_hi - h.row_lo + 1;
  ctx->n_sc = (size_t)h.n_sc;
  ctx->n_ga = (size_t)h.n_ga;
  ctx->n_gram = (size_t)h.n_gram;
  ctx->gram_band = h.gram_band;
  std::vector<Section> secs;
  const size_t payload = layout(ctx, h.nproj, h.nnz, &secs);
  if (payload != h.payload_bytes) return fail(AIM_EINVAL, "setup blob holds inconsistent sizes");
  const unsigned char* pay = static_cast<const unsigned char*>(blob) + sizeof(BlobHeader);
  if (payload_checksum(pay, payload) != h.checksum) return fail(AIM_EINVAL, "setup blob checksum mismatch (corrupted)");
  if (std::memcmp(pay + secs[SEC_NODES].offset, ctx->xy.data(), ctx->xy.size() * sizeof(double)) != 0)
    return fail(AIM_EINVAL, "setup blob made for another problem: vertices differ");
  if (h.key != problem_key(*ctx)) return fail(AIM_EINVAL, "setup blob key does not match its problem");
  // every stored index within its range, so that no kernel reads out of bounds
  auto ints = [&](int id) { return reinterpret_cast<const int*>(pay + secs[id].offset); };
  bool ok = csr_ok(ints(SEC_ROW_PTR), m, h.n_act) && all_below(ints(SEC_ACT_IX), h.n_act, m) &&
            csr_ok(ints(SEC_SC_PTR), h.n_act, h.n_sc) && all_below(ints(SEC_SC_COL), h.n_sc, n) &&
            csr_ok(ints(SEC_GA_PTR), n, h.n_ga) && all_below(ints(SEC_GA_ACT), h.n_ga, h.n_act);
  for (int iy = 0; ok && iy < m; ++iy)   // active points only on rows row_lo..row_hi
    if ((iy < h.row_lo || iy > h.row_hi) && ints(SEC_ROW_PTR)[iy + 1] != ints(SEC_ROW_PTR)[iy]) ok = false;
  int near_sec = -1;
  for (size_t i = 0; i < secs.size(); ++i)
    if (secs[i].slot == reinterpret_cast<void**>(&ctx->near.ptr)) near_sec = (int)i;
  if (ok && near_sec >= 0)
    ok = csr_ok(ints(near_sec), n, h.nnz) && all_below(ints(near_sec + 1), (size_t)h.nnz, n);
  if (!ok) return fail(AIM_EINVAL, "setup blob holds an index out of range");

  // device state: the stored arrays, then the copies derived from them
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaGetDevice(&ctx->device);
  ctx->prj.nproj = h.nproj;
  ctx->near.nnz = h.nnz;
  ctx->nnz_near = h.nnz;
  for (const Section& s : secs) {
    if (s.slot == reinterpret_cast<void**>(&ctx->tw)) {
      AIM_TRY(upload_twiddles(ctx, reinterpret_cast<const double*>(pay + s.offset), st));
      continue;
    }
    if (s.count == 0) continue;
    AIM_TRY(dev_alloc(ctx, s.slot, s.elem * s.count));
    AIM_CUDA_TRY(cudaMemcpyAsync(*s.slot, pay + s.offset, s.elem * s.count, cudaMemcpyHostToDevice, st));
  }
  const size_t nq = (size_t)(ctx->H + 1) * (ctx->H + 1);
  AIM_TRY(dev_alloc_t(ctx, &ctx->specUf, nq));
  AIM_TRY(dev_alloc_t(ctx, &ctx->specAf, nq));
  AIM_TRY(dev_alloc_t(ctx, &ctx->specUdf, nq));
  AIM_TRY(dev_alloc_t(ctx, &ctx->specAdf, nq));
  AIM_TRY(derive_narrow_copies(ctx->specU, nq, ctx->specUf, ctx->specUdf, st));
  AIM_TRY(derive_narrow_copies(ctx->specA, nq, ctx->specAf, ctx->specAdf, st));
  if (h.nnz > 0) {
    for (int v = 0; v < (te ? 2 : 1); ++v) {
      AIM_TRY(dev_alloc_t(ctx, &ctx->near.valf[v], (size_t)h.nnz));
      AIM_TRY(derive_narrow_copies(ctx->near.val[v], (size_t)h.nnz, ctx->near.valf[v], nullptr, st));
    }
  }
  // the host copies are read until the copies above complete
  AIM_CUDA_TRY(cudaStreamSynchronize(st));
  ctx->setup_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  guard.c = nullptr;
  *out = ctx;
  return AIM_OK;
}

}  // extern "C"
