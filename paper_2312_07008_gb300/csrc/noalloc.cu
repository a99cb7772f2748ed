// Natural orbitals and truncation without any device allocation.
//
// Some callers cannot call cudaMalloc: a host framework that owns all device
// memory through its own pool and forbids stray allocations, or a latency-
// critical loop where an allocation (which may synchronise the whole device)
// is not acceptable.  dsrg_fno_truncate_noalloc serves them with the same
// eigensolver and cut as dsrg_fno_truncate, using as scratch one file-scope
// device array of fixed size instead of the library's workspace.
#include "kernels.h"

namespace dsrg {

// Largest nvir the array serves: A, V and the eigensolver work, then status,
// N' and the sort ranks (n + 8 ints) in its tail.
constexpr int NOALLOC_NVIR_MAX = 512;
constexpr size_t NOALLOC_DOUBLES = 2 * (size_t)NOALLOC_NVIR_MAX * NOALLOC_NVIR_MAX +
                                   eig_work_doubles(NOALLOC_NVIR_MAX) + (NOALLOC_NVIR_MAX + 8 + 1) / 2 + 1;

// Held by every device that loads the library, until the process exits.
static __device__ __align__(256) double g_noalloc_scratch[NOALLOC_DOUBLES];

// Device address of the array on the current device (host code cannot use
// the symbol itself: it names a host-side stand-in).  Looked up on every call,
// so a device reset by the host application cannot leave a stale address.
static int noalloc_scratch(double** out) {
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess || p == nullptr) {
    cudaGetLastError();
    log_message(LOG_ERROR, "dsrg_fno_truncate_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
    return DSRG_FNO_ERR_CUDA;
  }
  *out = static_cast<double*>(p);
  return DSRG_FNO_OK;
}

}  // namespace dsrg

using namespace dsrg;

extern "C" int dsrg_fno_truncate_noalloc(int32_t nvir, const double* dvv, int32_t mode, double threshold,
                                         double degen_ratio, double* on_out, double* no_out, int32_t* nkept_out,
                                         void* stream) {
  if (nvir > NOALLOC_NVIR_MAX) {
    log_message(LOG_ERROR, "dsrg_fno_truncate_noalloc: nvir = %d exceeds the fixed scratch limit of %d", nvir,
                NOALLOC_NVIR_MAX);
    return DSRG_FNO_ERR_ARG;
  }
  if (nvir <= 0 || !dvv || !on_out || !no_out || !nkept_out) return DSRG_FNO_ERR_ARG;
  if (mode < 0 || mode > 3 || !isfinite(threshold) || !(degen_ratio >= 0.0)) return DSRG_FNO_ERR_ARG;
  if (!is_device_ptr(dvv) || !is_device_ptr(on_out) || !is_device_ptr(no_out)) {
    log_message(LOG_ERROR, "dsrg_fno_truncate_noalloc: dvv, on_out and no_out must be device memory");
    return DSRG_FNO_ERR_ARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  double* base = nullptr;
  DSRG_TRY(noalloc_scratch(&base));
  const size_t n2 = (size_t)nvir * nvir;
  double* A = base;
  double* V = A + n2;
  double* work = V + n2;
  int* ib = reinterpret_cast<int*>(work + eig_work_doubles(nvir));
  int* status = ib;  // four words
  int* nk = ib + 4;
  int* rank = ib + 8;
  // Every scratch word read below is first written by this call: A is a copy
  // of dvv, the eigensolver initialises its own work and status words.
  DSRG_CUDA(cudaMemcpyAsync(A, dvv, n2 * sizeof(double), cudaMemcpyDeviceToDevice, st));
  DSRG_TRY(eig_sym_jacobi(nvir, A, V, work, status, 60, st));
  DSRG_TRY(eig_sort(nvir, A, V, on_out, no_out, rank, true, true, st));
  DSRG_TRY(truncate_ons(nvir, on_out, mode, threshold, degen_ratio, nk, st));
  int h = 0;
  DSRG_CUDA(cudaMemcpyAsync(&h, nk, sizeof(int), cudaMemcpyDeviceToHost, st));
  DSRG_CUDA(cudaStreamSynchronize(st));
  *nkept_out = h;
  return DSRG_FNO_OK;
}
