// Fused operator products of concurrent solves: the batching side of serving.
//
// Several solves run at once, each on its own host thread and CUDA stream (a serving slot each).
// With a batcher attached (aim_solve_batched), every operator product of a solve becomes a request
// to the batcher instead of its own launches. Requests that arrive together are fused: their grid
// passes run as ONE persistent multi-context launch (grid_pass_multi), so many small problems share
// the GPU in one launch rather than in many small ones. Only problems of one size class fuse (P up
// to kMaxFusedP, within a factor of two): a launch lasts as long as its largest problem, and a small
// problem fused with a large one would advance at the large one's pace.
//
// Ordering is on the device: the request's stream records an event after its input is ready, the
// batcher's stream waits for it, runs the fused launch, records an event, and the request's stream
// waits for that before its next kernel. No host thread waits for the GPU here. A request waits on
// the host only for its partners: until every solve of its size class has submitted a product, or
// at most max_wait_us; then the first to notice becomes the leader and launches what is pending.
#include <algorithm>
#include <chrono>
#include <new>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <vector>

#include "aim_internal.h"

namespace aim {
namespace {
constexpr int kMaxFusedP = 512;      // larger grids keep their own (tuned) launches (measured: no gain at P = 1024)
constexpr int kClasses = 16;

int size_class(const aim_ctx* ctx) {
  int l = 0;
  while ((1 << l) < ctx->P) ++l;
  return std::min(kClasses - 1, l >> 1);   // P = 64..128, 256..512
}
}  // namespace
}  // namespace aim

struct aim_batcher {
  struct Req {
    aim_ctx* ctx;
    aim_op op;
    int nrhs;
    const double2* x;
    double2* y;
    int precision;
    cudaStream_t st;
    cudaEvent_t in = nullptr;
    aim_status status = AIM_OK;
    int state = 0;   // 0 pending, 2 served
  };
  std::mutex mu;
  std::condition_variable cv;
  int participants[aim::kClasses] = {};   // solves of each size class inside aim_solve_batched
  int pend[aim::kClasses] = {};           // their requests not yet launched
  std::deque<Req*> pending;
  cudaStream_t stream = nullptr;
  std::vector<cudaEvent_t> events;   // one per fused group, reused round robin
  size_t next_event = 0;
  aim::MultiLauncher ml;
  int max_wait_us = 200;
  long long products = 0, launches = 0, fused_products = 0;
  aim_status broken = AIM_OK;
};

namespace aim {

static thread_local aim_batcher* tl_batcher = nullptr;

aim_batcher* current_batcher() { return tl_batcher; }

// Launches every pending request: grouped by precision and size class; a group of one runs the
// single-context path, a larger group one multi-context launch per grid-pass stage. Called with
// the lock held.
static void lead(aim_batcher* b) {
  std::vector<aim_batcher::Req*> reqs(b->pending.begin(), b->pending.end());
  b->pending.clear();
  for (int& c : b->pend) c = 0;
  std::stable_sort(reqs.begin(), reqs.end(), [](const aim_batcher::Req* a, const aim_batcher::Req* c) {
    return a->precision != c->precision ? a->precision < c->precision : size_class(a->ctx) < size_class(c->ctx);
  });
  size_t i = 0;
  while (i < reqs.size()) {
    size_t j = i + 1;
    while (j < reqs.size() && reqs[j]->precision == reqs[i]->precision &&
           size_class(reqs[j]->ctx) == size_class(reqs[i]->ctx))
      ++j;
    // the batcher's stream waits for every input of the group
    aim_status s = b->broken;
    for (size_t q = i; q < j && s == AIM_OK; ++q)
      if (cudaStreamWaitEvent(b->stream, reqs[q]->in, 0) != cudaSuccess) s = fail(AIM_ECUDA, "batcher: wait for input");
    if (s == AIM_OK) {
      if (j - i == 1) {
        aim_batcher::Req* r = reqs[i];
        s = apply_op(r->ctx, r->op, r->nrhs, r->x, r->y, r->precision, b->stream);
      } else {
        std::vector<aim_ctx*> ctxs;
        std::vector<aim_op> ops;
        std::vector<int> nrhs;
        std::vector<const double2*> xs;
        std::vector<double2*> ys;
        for (size_t q = i; q < j; ++q) {
          ctxs.push_back(reqs[q]->ctx);
          ops.push_back(reqs[q]->op);
          nrhs.push_back(reqs[q]->nrhs);
          xs.push_back(reqs[q]->x);
          ys.push_back(reqs[q]->y);
        }
        s = apply_op_multi(b->ml, (int)(j - i), ctxs.data(), ops.data(), nrhs.data(), xs.data(), ys.data(),
                           reqs[i]->precision, b->stream);
        b->fused_products += (long long)(j - i);
      }
      b->launches += 1;
    }
    // the requests' streams wait for the result
    cudaEvent_t done = b->events[b->next_event++ % b->events.size()];
    if (s == AIM_OK && cudaEventRecord(done, b->stream) != cudaSuccess) s = fail(AIM_ECUDA, "batcher: record");
    for (size_t q = i; q < j; ++q) {
      if (s == AIM_OK && cudaStreamWaitEvent(reqs[q]->st, done, 0) != cudaSuccess) s = fail(AIM_ECUDA, "batcher: wait");
      reqs[q]->status = s;
      reqs[q]->state = 2;
    }
    i = j;
  }
  b->cv.notify_all();
}

aim_status batcher_product(aim_batcher* b, aim_ctx* ctx, aim_op op, int nrhs, const double2* x, double2* y,
                           int precision, cudaStream_t st) {
  if (ctx->P > kMaxFusedP) return apply_op(ctx, op, nrhs, x, y, precision, st);
  aim_batcher::Req r;
  r.ctx = ctx;
  r.op = op;
  r.nrhs = nrhs;
  r.x = x;
  r.y = y;
  r.precision = precision;
  r.st = st;
  // the input is ready when the stream reaches this point
  thread_local cudaEvent_t in_ev = nullptr;
  if (in_ev == nullptr) AIM_CUDA_TRY(cudaEventCreateWithFlags(&in_ev, cudaEventDisableTiming));
  AIM_CUDA_TRY(cudaEventRecord(in_ev, st));
  r.in = in_ev;
  const int cls = size_class(ctx);
  std::unique_lock<std::mutex> lk(b->mu);
  b->products += 1;
  b->pending.push_back(&r);
  b->pend[cls] += 1;
  b->cv.notify_all();
  const auto deadline = std::chrono::steady_clock::now() + std::chrono::microseconds(b->max_wait_us);
  while (r.state != 2) {
    if (b->pend[cls] >= b->participants[cls] || std::chrono::steady_clock::now() >= deadline) {
      lead(b);
      break;
    }
    b->cv.wait_until(lk, deadline);
  }
  return r.status;
}

}  // namespace aim

using namespace aim;

extern "C" {

aim_status aim_batcher_create(int max_wait_us, aim_batcher** out) {
  if (!out || max_wait_us < 0 || max_wait_us > 1000000) return fail(AIM_EINVAL, "bad argument");
  *out = nullptr;
  aim_batcher* b = new (std::nothrow) aim_batcher();
  if (!b) return fail(AIM_ENOMEM, "batcher allocation");
  b->max_wait_us = max_wait_us;
  aim_status s = AIM_OK;
  if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) s = fail(AIM_ECUDA, "batcher stream");
  b->events.resize(64, nullptr);
  for (auto& e : b->events)
    if (s == AIM_OK && cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) s = fail(AIM_ECUDA, "batcher event");
  if (s == AIM_OK) s = b->ml.init();
  if (s != AIM_OK) {
    aim_batcher_destroy(b);
    return s;
  }
  *out = b;
  return AIM_OK;
}

void aim_batcher_destroy(aim_batcher* b) {
  if (!b) return;
  if (b->stream) cudaStreamSynchronize(b->stream);
  for (auto e : b->events)
    if (e) cudaEventDestroy(e);
  if (b->stream) cudaStreamDestroy(b->stream);
  delete b;
}

aim_status aim_batcher_stats(aim_batcher* b, long long* products, long long* launches, long long* fused_products) {
  if (!b) return fail(AIM_EINVAL, "bad argument");
  std::lock_guard<std::mutex> lk(b->mu);
  if (products) *products = b->products;
  if (launches) *launches = b->launches;
  if (fused_products) *fused_products = b->fused_products;
  return AIM_OK;
}

aim_status aim_solve_batched(aim_batcher* b, aim_ctx* ctx, aim_op system, int nrhs, const void* rhs, void* x,
                             int x0_given, const aim_solve_opts* opts, aim_solve_info* info, void* stream) {
  if (!b || !ctx) return fail(AIM_EINVAL, "bad argument");
  if (tl_batcher != nullptr) return fail(AIM_ESTATE, "a batched solve is already running on this thread");
  const bool fusible = ctx->P <= kMaxFusedP;
  const int cls = size_class(ctx);
  if (fusible) {
    std::lock_guard<std::mutex> lk(b->mu);
    b->participants[cls] += 1;
  }
  tl_batcher = b;
  aim_status s = aim_solve(ctx, system, nrhs, rhs, x, x0_given, opts, info, stream);
  tl_batcher = nullptr;
  if (fusible) {
    std::lock_guard<std::mutex> lk(b->mu);
    b->participants[cls] -= 1;
    b->cv.notify_all();   // partners no longer wait for this solve
  }
  if (s == AIM_OK) {
    // a fused launch whose grid barrier gave up (its flag is read once the launches are done)
    std::lock_guard<std::mutex> lk(b->mu);
    if (cudaStreamQuery(b->stream) == cudaSuccess) {
      const aim_status e = b->ml.check();
      if (e != AIM_OK) b->broken = s = e;
    }
  }
  return s;
}

}  // extern "C"
