// Shared device/host helpers of the FNO SA-DSRG-PT2 library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>

#include <mutex>
#include <vector>

#include "../../include/dsrg_fno.h"

namespace dsrg {

// Status propagation inside the library (never across the ABI as exceptions).
// Messages go to the caller's log callback (dsrg_fno_set_log_callback);
// without one the library prints nothing.
void log_message(int level, const char* fmt, ...);
constexpr int LOG_ERROR = 0, LOG_WARNING = 1;

#define DSRG_CUDA(call)                                                       \
  do {                                                                        \
    cudaError_t e_ = (call);                                                  \
    if (e_ != cudaSuccess) {                                                  \
      log_message(LOG_ERROR, "%s failed: %s (%s:%d)", #call,                  \
                  cudaGetErrorString(e_), __FILE__, __LINE__);                \
      return DSRG_FNO_ERR_CUDA;                                               \
    }                                                                         \
  } while (0)

#define DSRG_TRY(call)                                                        \
  do {                                                                        \
    int s_ = (call);                                                          \
    if (s_ != DSRG_FNO_OK) return s_;                                         \
  } while (0)

// Every kernel launch of the library is followed by this check, which also
// feeds the launch counter of the profiling interface.
void count_launch();
bool profiling();
void prof_begin(const char* name, double flops, cudaStream_t st, void** token);
void prof_end(void* token, cudaStream_t st);
// A counter without timing (queried like a kernel: launches = calls, flops = summed value).
void prof_count(const char* name, double value);
// Scoped timing of a phase of a call (recorded only while profiling).
struct PhaseTimer {
  void* tok = nullptr;
  cudaStream_t st;
  PhaseTimer(const char* name, cudaStream_t s) : st(s) { prof_begin(name, 0.0, s, &tok); }
  ~PhaseTimer() { prof_end(tok, st); }
};
#define DSRG_CAT2(a, b) a##b
#define DSRG_CAT(a, b) DSRG_CAT2(a, b)
#define DSRG_PHASE(name, st) PhaseTimer DSRG_CAT(phase_timer_, __LINE__)(name, st)

#define DSRG_LAUNCH_CHECK() \
  do {                      \
    count_launch();         \
    DSRG_CUDA(cudaGetLastError()); \
  } while (0)

inline int ceil_div(long a, long b) { return (int)((a + b - 1) / b); }

// --------------------------------------------------------------------------
// Grow-only device workspace, one per device, carved into aligned pieces.
// --------------------------------------------------------------------------
struct Workspace {
  char* base = nullptr;
  size_t cap = 0;
  size_t off = 0;
  int device = -1;
};

Workspace& workspace_for_current_device();
std::mutex& workspace_mutex();

// Makes sure at least `bytes` are available; may synchronise the device.
int ws_reserve(Workspace& ws, size_t bytes);

template <typename T>
T* ws_take(Workspace& ws, size_t count) {
  size_t bytes = ((count * sizeof(T)) + 255) & ~(size_t)255;
  if (ws.off + bytes > ws.cap) return nullptr;
  T* p = reinterpret_cast<T*>(ws.base + ws.off);
  ws.off += bytes;
  return p;
}

inline size_t ws_bytes(size_t count, size_t elt) { return ((count * elt) + 255) & ~(size_t)255; }

// --------------------------------------------------------------------------
// Regulariser of Eq. A7:  R_c(Delta) = (1 - exp(-c s Delta^2)) / Delta.
// For x = c s Delta^2 below 1e-3 the Taylor series of 1 - exp(-x) is used
// (truncation error below x^5/720 relative); Delta = 0 gives 0.
// --------------------------------------------------------------------------
__host__ __device__ __forceinline__ double regularizer(double delta, double cs) {
  const double x = cs * delta * delta;
  if (x < 1.0e-3) {
    const double p = 1.0 - x * (0.5 - x * (1.0 / 6.0 - x * (1.0 / 24.0 - x * (1.0 / 120.0))));
    return cs * delta * p;
  }
  return -expm1(-x) / delta;
}

// Problem geometry used by the kernels.
struct Geometry {
  int nc, na, nv, nq;  // core, active, virtual, auxiliary
  int nh, np;          // holes, particles
  double s;
};

}  // namespace dsrg
