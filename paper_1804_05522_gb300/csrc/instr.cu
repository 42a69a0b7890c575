// Launch counting and per-family CUDA-event timing of the library's kernels.
#include <atomic>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "common.cuh"

namespace fde {

static std::atomic<unsigned long long> g_launches{0};
static std::atomic<int> g_prof_on{0};
static std::mutex g_prof_mu;
struct Rec {
  cudaEvent_t a, b;
  double work;
  int kind;
};
static std::map<std::string, std::vector<Rec>> g_prof;
static std::vector<cudaEvent_t> g_pool;  // reusable events

static cudaEvent_t take_event() {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  if (g_pool.empty()) {
    for (int i = 0; i < 256; ++i) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) {
        cudaGetLastError();
        break;
      }
      g_pool.push_back(e);
    }
    if (g_pool.empty()) return nullptr;
  }
  cudaEvent_t e = g_pool.back();
  g_pool.pop_back();
  return e;
}

// Allocations left before the injected failure (-1: none armed).
static std::atomic<long long> g_alloc_countdown{-1};
bool alloc_fail_now() {
  long long v = g_alloc_countdown.load();
  while (v >= 0)
    if (g_alloc_countdown.compare_exchange_weak(v, v - 1)) return v == 0;
  return false;
}
void fail_alloc_after(long long n) { g_alloc_countdown.store(n < 0 ? -1 : n); }

// Launches recorded while a thread captures a graph are not counted: the
// graph's kernels are counted when it runs.
static thread_local int t_count_suspended = 0;
void count_suspend(bool on) { t_count_suspended += on ? 1 : -1; }
void count_launch() {
  if (!t_count_suspended) g_launches.fetch_add(1, std::memory_order_relaxed);
}
void count_launches(size_t n) {
  if (!t_count_suspended) g_launches.fetch_add(n, std::memory_order_relaxed);
}
bool prof_enabled() { return g_prof_on.load(std::memory_order_relaxed) != 0; }

ProfScope::ProfScope(const char* family, cudaStream_t s, double w, int k)
    : fam(family), st(s), a(nullptr), work(w), kind(k) {
  if (!g_prof_on.load(std::memory_order_relaxed)) return;
  // nothing is timed while the stream is being captured into a graph (an
  // event recorded there belongs to the graph, not to this timeline)
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) {
    cudaGetLastError();
    return;
  }
  if (cs != cudaStreamCaptureStatusNone) return;
  a = take_event();
  if (a) cudaEventRecord(a, st);
}
ProfScope::~ProfScope() {
  if (!a) return;
  cudaEvent_t b = take_event();
  if (!b) return;
  cudaEventRecord(b, st);
  std::lock_guard<std::mutex> lk(g_prof_mu);
  g_prof[fam].push_back({a, b, work, kind});
}

}  // namespace fde

using namespace fde;

extern "C" unsigned long long fde_launch_count(void) { return g_launches.load(); }

extern "C" void fde_prof_enable(int on) { g_prof_on.store(on ? 1 : 0); }

extern "C" fde_status fde_prof_query(const char* family, double* ms, long long* launches, double* work,
                                     int* work_kind) {
  FDE_ARG(family != nullptr && ms != nullptr && launches != nullptr, "NULL argument");
  std::lock_guard<std::mutex> lk(g_prof_mu);
  *ms = 0.0;
  *launches = 0;
  if (work) *work = 0.0;
  if (work_kind) *work_kind = 1;
  auto it = g_prof.find(family);
  if (it == g_prof.end()) return FDE_OK;
  for (auto& e : it->second) {
    FDE_CUDA(cudaEventSynchronize(e.b));
    float t = 0.f;
    FDE_CUDA(cudaEventElapsedTime(&t, e.a, e.b));
    *ms += t;
    *launches += 1;
    if (work) *work += e.work;
    if (work_kind) *work_kind = e.kind;
  }
  return FDE_OK;
}

extern "C" void fde_prof_reset(void) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  for (auto& kv : g_prof)
    for (auto& e : kv.second) {
      if (cudaEventSynchronize(e.b) != cudaSuccess) cudaGetLastError();  // leave no error pending
      g_pool.push_back(e.a);
      g_pool.push_back(e.b);
    }
  g_prof.clear();
}

extern "C" void fde_fail_alloc_after(long long n) { fde::fail_alloc_after(n); }
