// Kernel launch counting and optional CUDA-event timing of every kernel the library enqueues.
// Counting is always on (one atomic increment per launch). Timing, when started, brackets
// each launch with a pair of events recorded on the launch's own stream.
#include <atomic>
#include <mutex>

#include "aim_internal.h"

namespace aim {

static const char* kKernelNames[K_COUNT] = {
    "row_fwd (anterpolation + forward row DFT)",
    "col_conv (column DFT x spectrum x inverse column DFT)",
    "row_inv (inverse row DFT + restriction)",
    "gather (interpolation + near-field SpMV)",
    "gram_inv (banded G^-1)",
    "setup_kernel_samples",
    "setup_even_dft",
    "setup_pack_spectrum",
    "setup_segment_pairs",
    "setup_near_entries",
    "rhs_planewave",
    "gmres_arnoldi (DCGS2 projections and updates; timed per step)",
    "grid_multi (persistent: row passes, column pass and gathers of several contexts)",
    "dft_stage (radix-16 pass measurement: CUDA cores or tensor cores)",
};

namespace {
struct Slot {
  cudaEvent_t a = nullptr, b = nullptr;
  int id = 0;
};
std::atomic<long long> g_launches[K_COUNT];
std::mutex g_mu;
bool g_timing = false;
std::vector<Slot> g_pool;
size_t g_used = 0;
}  // namespace

// the same counts per host thread (a capture reads its own launches without other threads')
thread_local long long tl_launches[K_COUNT];

void count_launches(int id, int n) {
  g_launches[id].fetch_add(n, std::memory_order_relaxed);
  tl_launches[id] += n;
}

void thread_launch_counts(long long* out) {
  for (int i = 0; i < K_COUNT; ++i) out[i] = tl_launches[i];
}

bool profiling_active() {
  std::lock_guard<std::mutex> lk(g_mu);
  return g_timing;
}

ProfScope::ProfScope(int id_, cudaStream_t st_, bool count_launch) : id(id_), st(st_), slot(-1) {
  if (count_launch) {
    g_launches[id].fetch_add(1, std::memory_order_relaxed);
    tl_launches[id] += 1;
  }
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_timing) return;
  if (g_used == g_pool.size()) {
    Slot s;
    if (cudaEventCreate(&s.a) != cudaSuccess || cudaEventCreate(&s.b) != cudaSuccess) {
      cudaGetLastError();
      return;
    }
    g_pool.push_back(s);
  }
  slot = (int)g_used++;
  g_pool[slot].id = id;
  cudaEventRecord(g_pool[slot].a, st);
}

ProfScope::~ProfScope() {
  if (slot < 0) return;
  std::lock_guard<std::mutex> lk(g_mu);
  cudaEventRecord(g_pool[slot].b, st);
}

}  // namespace aim

using namespace aim;

extern "C" {

long long aim_launch_count(void) {
  long long t = 0;
  for (int i = 0; i < K_COUNT; ++i) t += g_launches[i].load();
  return t;
}

aim_status aim_profile_start(void) {
  std::lock_guard<std::mutex> lk(g_mu);
  g_used = 0;
  g_timing = true;
  return AIM_OK;
}

aim_status aim_profile_stop(aim_kernel_stat* stats, int max_stats, int* count) {
  std::lock_guard<std::mutex> lk(g_mu);
  g_timing = false;
  long long launches[K_COUNT] = {};
  double ms[K_COUNT] = {};
  for (size_t i = 0; i < g_used; ++i) {
    Slot& s = g_pool[i];
    if (cudaEventSynchronize(s.b) != cudaSuccess) {
      cudaGetLastError();
      return fail(AIM_ECUDA, "profile event synchronisation failed");
    }
    float t = 0.f;
    if (cudaEventElapsedTime(&t, s.a, s.b) == cudaSuccess) {
      ms[s.id] += t;
      launches[s.id] += 1;
    } else {
      cudaGetLastError();
    }
  }
  g_used = 0;
  int c = 0;
  for (int i = 0; i < K_COUNT && c < max_stats; ++i) {
    if (!launches[i]) continue;
    if (stats) {
      stats[c].kernel = i;
      stats[c].name = kKernelNames[i];
      stats[c].launches = launches[i];
      stats[c].total_ms = ms[i];
    }
    ++c;
  }
  if (count) *count = c;
  return AIM_OK;
}

}  // extern "C"
