// Phase timing and launch counting (instrumentation; the paper has no
// counterpart).  When enabled, launchers record a CUDA event pair on their own
// stream around every kernel phase; jzt_profile_read waits on the recorded
// events and returns the summed durations.  The launch counter is always on.
#include <cuda_runtime.h>

#include <atomic>
#include <mutex>
#include <vector>

#include "common.cuh"

namespace jzt {

namespace {
struct Rec {
  int phase;
  cudaEvent_t a, b;
};
std::mutex g_mu;
std::vector<Rec> g_recs;
std::vector<cudaEvent_t> g_pool;
std::atomic<bool> g_on{false};
std::atomic<long long> g_launches{0};
thread_local int t_open_phase = -1;
thread_local cudaEvent_t t_open_event = nullptr;

cudaEvent_t get_event() {
  if (!g_pool.empty()) {
    cudaEvent_t e = g_pool.back();
    g_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

const char* kNames[kPhaseCount] = {"box",      "keys",     "sort",     "gather",  "splits",
                                   "nodes",    "knn_top",  "knn_n2n",  "knn_sort", "knn_l2l",
                                   "fof_top",  "fof_n2n",  "fof_l2l",  "fof_labels"};
}  // namespace

void note_launch(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

void prof_begin(int phase, cudaStream_t s) {
  if (!g_on.load(std::memory_order_relaxed)) return;
  std::lock_guard<std::mutex> lk(g_mu);
  t_open_phase = phase;
  t_open_event = get_event();
  cudaEventRecord(t_open_event, s);
}

void prof_end(int phase, cudaStream_t s) {
  if (!g_on.load(std::memory_order_relaxed) || t_open_phase != phase || !t_open_event) return;
  std::lock_guard<std::mutex> lk(g_mu);
  cudaEvent_t b = get_event();
  cudaEventRecord(b, s);
  g_recs.push_back({phase, t_open_event, b});
  t_open_phase = -1;
  t_open_event = nullptr;
}

const char* phase_name(int i) { return (i >= 0 && i < kPhaseCount) ? kNames[i] : nullptr; }

int profile_enable(int on) {
  g_on.store(on != 0);
  return 0;
}

int profile_read(double* ms, int64_t* counts, int n, long long* launches) {
  std::lock_guard<std::mutex> lk(g_mu);
  for (int i = 0; i < n; ++i) {
    if (ms) ms[i] = 0.0;
    if (counts) counts[i] = 0;
  }
  int rc = 0;
  for (const Rec& r : g_recs) {
    if (cudaEventSynchronize(r.b) != cudaSuccess) rc = -1;
    float t = 0.0f;
    if (cudaEventElapsedTime(&t, r.a, r.b) != cudaSuccess) rc = -1;
    if (r.phase < n) {
      if (ms) ms[r.phase] += t;
      if (counts) counts[r.phase] += 1;
    }
    g_pool.push_back(r.a);
    g_pool.push_back(r.b);
  }
  g_recs.clear();
  if (launches) *launches = g_launches.exchange(0);
  return rc;
}

}  // namespace jzt
