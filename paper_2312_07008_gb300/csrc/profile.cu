// Launch accounting (include/dsrg_fno_profile.h) and the log callback.
#include <stdarg.h>

#include <atomic>
#include <string>
#include <vector>

#include "../../include/dsrg_fno_profile.h"
#include "kernels.h"

namespace dsrg {

static std::atomic<long long> g_launches{0};
static bool g_prof = false;

struct ProfRec {
  std::string name;
  cudaEvent_t a, b;
  double flops;
};
struct ProfCount {
  std::string name;
  double value;
};
static std::vector<ProfCount> g_counts;
static std::vector<ProfRec> g_recs;
// Event pairs are kept across profiling sessions: creating events while
// other threads launch work contends on the driver, so a session reuses the
// pairs of earlier ones and creates only what it lacks.
static std::vector<std::pair<cudaEvent_t, cudaEvent_t>> g_event_pool;
static std::mutex g_prof_mutex;

// The caller's log sink; messages are dropped while none is set.
static std::mutex g_log_mutex;
static dsrg_fno_log_fn g_log_fn = nullptr;
static void* g_log_user = nullptr;

void log_message(int level, const char* fmt, ...) {
  std::lock_guard<std::mutex> lk(g_log_mutex);
  if (!g_log_fn) return;
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_log_fn(level, buf, g_log_user);
}

void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

bool profiling() { return g_prof; }

void prof_begin(const char* name, double flops, cudaStream_t st, void** token) {
  *token = nullptr;
  if (!g_prof) return;
  std::lock_guard<std::mutex> lk(g_prof_mutex);
  ProfRec r;
  r.name = name;
  r.flops = flops;
  if (g_recs.size() < g_event_pool.size()) {
    r.a = g_event_pool[g_recs.size()].first;
    r.b = g_event_pool[g_recs.size()].second;
  } else {
    cudaEventCreate(&r.a);
    cudaEventCreate(&r.b);
    g_event_pool.emplace_back(r.a, r.b);
  }
  cudaEventRecord(r.a, st);
  g_recs.push_back(r);
  *token = reinterpret_cast<void*>(g_recs.size());
}

void prof_count(const char* name, double value) {
  if (!g_prof) return;
  std::lock_guard<std::mutex> lk(g_prof_mutex);
  g_counts.push_back({name, value});
}

void prof_end(void* token, cudaStream_t st) {
  if (!token) return;
  std::lock_guard<std::mutex> lk(g_prof_mutex);
  size_t i = reinterpret_cast<size_t>(token) - 1;
  if (i < g_recs.size()) cudaEventRecord(g_recs[i].b, st);
}

}  // namespace dsrg

using namespace dsrg;

extern "C" void dsrg_fno_set_log_callback(dsrg_fno_log_fn fn, void* user) {
  std::lock_guard<std::mutex> lk(g_log_mutex);
  g_log_fn = fn;
  g_log_user = user;
}

extern "C" void dsrg_fno_profile_enable(int32_t enable) {
  std::lock_guard<std::mutex> lk(g_prof_mutex);
  if (enable) {
    // the pairs of the last session go back to the pool; wait until they
    // have been reached so that re-recording them is safe
    for (auto& r : g_recs) cudaEventSynchronize(r.b);
    g_recs.clear();
    g_counts.clear();
  }
  g_prof = enable != 0;
}

extern "C" int dsrg_fno_profile_query(const char* name, double* total_ms, int64_t* launches, double* flops) {
  std::lock_guard<std::mutex> lk(g_prof_mutex);
  double t = 0.0, f = 0.0;
  int64_t n = 0;
  for (auto& r : g_recs) {
    if (name && r.name != name) continue;
    cudaEventSynchronize(r.b);
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
      t += ms;
      f += r.flops;
      ++n;
    } else {
      cudaGetLastError();
    }
  }
  for (auto& c : g_counts) {
    if (name && c.name != name) continue;
    f += c.value;
    ++n;
  }
  if (total_ms) *total_ms = t;
  if (launches) *launches = n;
  if (flops) *flops = f;
  return DSRG_FNO_OK;
}

extern "C" int64_t dsrg_fno_launch_count(int32_t reset) {
  long long v = reset ? g_launches.exchange(0) : g_launches.load();
  return (int64_t)v;
}
