// Batched runs over ragged instances (dsrg_fno_batch_run).
//
// Instances of a batch are independent problems of different sizes.  Each is
// too small to fill the GPU by itself (a few hundred virtuals: the pair
// contractions cover a fraction of the SMs, and every stage ends in a host
// read of a scalar), so the runner keeps several instances in flight: host
// workers, each with its own CUDA stream and device workspace, take instances
// largest first (longest-processing-time order, by algorithmic flops) from a
// shared counter.  Kernels of different workers overlap on the device.
//
// Worker count: given by the caller, or tuned per batch shape: the first
// calls with a shape try each candidate once (the call's wall time decides),
// later calls reuse the fastest.
#include <math.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <map>
#include <thread>
#include <vector>

#include "../../include/dsrg_fno_profile.h"
#include "kernels.h"

namespace dsrg {

namespace {

constexpr int MAX_WORKERS = 16;
const int TUNE_CANDIDATES[] = {2, 4, 8};

struct Worker {
  Workspace ws;
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
};

struct DevicePool {
  Worker w[MAX_WORKERS];
  cudaEvent_t start = nullptr;
};

std::mutex g_batch_mutex;
DevicePool g_pool[64];

// batch shape -> (candidate index tried next, best seconds per candidate)
struct TuneState {
  int next = 0;
  double secs[3] = {0.0, 0.0, 0.0};
};
std::map<std::vector<long long>, TuneState> g_tune;
int g_last_workers = 0;

double item_flops(const dsrg_fno_problem& p) {
  const double nh = p.ncore + p.nact, nv = p.nvir, nq = p.naux;
  return nq * nv * nv * nh * (nh + 1.0) + nh * nh * nv * nv * nv;
}

int ensure_worker(Worker& w) {
  if (!w.stream) DSRG_CUDA(cudaStreamCreateWithFlags(&w.stream, cudaStreamNonBlocking));
  if (!w.done) DSRG_CUDA(cudaEventCreateWithFlags(&w.done, cudaEventDisableTiming));
  return DSRG_FNO_OK;
}

int run_item(Worker& w, size_t budget, dsrg_fno_batch_item& it) {
  const dsrg_fno_problem* p = &it.problem;
  it.e2 = 0.0;
  it.nkept = 0;
  it.de = 0.0;
  const bool cut = it.cut_mode >= 0;
  if (cut && (!it.dvv_out || !it.on_out || !it.no_out)) return DSRG_FNO_ERR_ARG;
  if (it.correction && !cut) return DSRG_FNO_ERR_ARG;
  if (it.dvv_out) {
    DSRG_TRY(impl_vv_opdm(w.ws, budget, p, it.dvv_out, &it.e2, w.stream));
  } else {
    DSRG_TRY(impl_pt2_energy(w.ws, budget, p, &it.e2, w.stream));
  }
  if (!cut) return DSRG_FNO_OK;
  int32_t nk = 0;
  DSRG_TRY(impl_truncate(w.ws, p->nvir, it.dvv_out, it.cut_mode, it.cut_threshold, it.cut_degen_ratio, it.on_out,
                         it.no_out, &nk, w.stream));
  it.nkept = nk;
  if (!it.correction) return DSRG_FNO_OK;
  const double e_mo = it.e2;
  DSRG_TRY(impl_correction(w.ws, budget, p, nk, it.no_out, &e_mo, &it.de, nullptr, nullptr, w.stream));
  return DSRG_FNO_OK;
}

}  // namespace

}  // namespace dsrg

using namespace dsrg;

extern "C" int dsrg_fno_batch_run(dsrg_fno_batch_item* items, int32_t n, int32_t nworkers, void* stream) {
  if (n < 0 || (n > 0 && !items) || nworkers < 0 || nworkers > MAX_WORKERS) return DSRG_FNO_ERR_ARG;
  if (n == 0) return DSRG_FNO_OK;
  std::lock_guard<std::mutex> lk(g_batch_mutex);
  int dev = 0;
  DSRG_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return DSRG_FNO_ERR_UNSUPPORTED;
  DevicePool& pool = g_pool[dev];
  cudaStream_t caller = (cudaStream_t)stream;

  // largest first
  std::vector<int> order(n);
  std::vector<double> cost(n);
  std::vector<long long> shape;
  shape.reserve(4 * (size_t)n);
  for (int i = 0; i < n; ++i) {
    order[i] = i;
    cost[i] = item_flops(items[i].problem);
    const dsrg_fno_problem& p = items[i].problem;
    shape.insert(shape.end(), {(long long)p.ncore, (long long)p.nact, (long long)p.nvir, (long long)p.naux});
  }
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost[a] > cost[b]; });

  TuneState* tune = nullptr;
  int workers = nworkers;
  if (workers == 0) {
    tune = &g_tune[shape];
    if (tune->next < 3) {
      workers = TUNE_CANDIDATES[tune->next];
    } else {
      int best = 0;
      for (int c = 1; c < 3; ++c)
        if (tune->secs[c] < tune->secs[best]) best = c;
      workers = TUNE_CANDIDATES[best];
    }
  }
  workers = std::max(1, std::min(workers, n));
  g_last_workers = workers;

  for (int k = 0; k < workers; ++k) DSRG_TRY(ensure_worker(pool.w[k]));
  if (!pool.start) DSRG_CUDA(cudaEventCreateWithFlags(&pool.start, cudaEventDisableTiming));
  DSRG_CUDA(cudaEventRecord(pool.start, caller));
  for (int k = 0; k < workers; ++k) DSRG_CUDA(cudaStreamWaitEvent(pool.w[k].stream, pool.start, 0));

  // each worker plans its passes within an equal share of the free memory
  size_t have = 0;
  for (int k = 0; k < workers; ++k) have += pool.w[k].ws.cap;
  const size_t share = device_budget(have) / (size_t)workers;

  const auto t0 = std::chrono::steady_clock::now();
  std::atomic<int> next{0};
  std::vector<int> status(n, DSRG_FNO_OK);
  auto body = [&](int k) {
    cudaSetDevice(dev);
    SharedDeviceScope shared(workers > 1);
    Worker& w = pool.w[k];
    for (;;) {
      const int j = next.fetch_add(1);
      if (j >= n) break;
      const int i = order[j];
      status[i] = run_item(w, share, items[i]);
    }
  };
  std::vector<std::thread> threads;
  for (int k = 1; k < workers; ++k) threads.emplace_back(body, k);
  body(0);
  for (auto& t : threads) t.join();
  const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  if (tune && tune->next < 3) tune->secs[tune->next++] = secs;

  for (int k = 0; k < workers; ++k) {
    DSRG_CUDA(cudaEventRecord(pool.w[k].done, pool.w[k].stream));
    DSRG_CUDA(cudaStreamWaitEvent(caller, pool.w[k].done, 0));
  }
  int first = DSRG_FNO_OK;
  for (int i = 0; i < n; ++i) {
    items[i].status = status[i];
    if (status[i] != DSRG_FNO_OK && first == DSRG_FNO_OK) first = status[i];
  }
  return first;
}

// Workers of the last dsrg_fno_batch_run (profiling header).
extern "C" int32_t dsrg_fno_batch_last_workers(void) { return g_last_workers; }

// Frees the batch workers' workspaces, streams and events (all devices).
namespace dsrg {
void release_batch_pools() {
  std::lock_guard<std::mutex> lk(g_batch_mutex);
  int cur = 0;
  cudaGetDevice(&cur);
  for (int d = 0; d < 64; ++d) {
    DevicePool& pool = g_pool[d];
    bool any = pool.start != nullptr;
    for (int k = 0; k < MAX_WORKERS; ++k) any = any || pool.w[k].ws.base || pool.w[k].stream;
    if (!any) continue;
    cudaSetDevice(d);
    cudaDeviceSynchronize();
    for (int k = 0; k < MAX_WORKERS; ++k) {
      Worker& w = pool.w[k];
      if (w.ws.base) cudaFree(w.ws.base);
      w.ws = Workspace{};
      if (w.stream) cudaStreamDestroy(w.stream);
      if (w.done) cudaEventDestroy(w.done);
      w.stream = nullptr;
      w.done = nullptr;
    }
    if (pool.start) cudaEventDestroy(pool.start);
    pool.start = nullptr;
  }
  cudaSetDevice(cur);
}
}  // namespace dsrg
