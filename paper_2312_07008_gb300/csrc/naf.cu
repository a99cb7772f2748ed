// Natural auxiliary functions (Sec. 4: the compression of the auxiliary
// basis the paper proposes for the PT2 step).
//
// W_PQ = sum_{ia} B^P_{ia} B^Q_{ia} over the hole-particle DF factors is
// diagonalised, W = U diag(w) U^T (w descending), and the factors are
// rotated to the eigenvectors with w > threshold:
//   B'^K_{ia} = sum_Q U_QK B^Q_{ia}.
// In the fast form both contractions run on the digit-plane kernel: W with
// 5 planes (its entries are sums of nh np products), B' with 6 (B' enters
// every integral, as the rotation to the frozen natural orbitals does);
// the eigensolve is the double-float Jacobi solver of the natural orbitals.
#include <math.h>

#include <vector>

#include "kernels.h"

namespace dsrg {

int impl_naf(Workspace& ws, int32_t nh, int32_t np, int32_t naux, const double* B, double threshold, int precision,
             double* B_out, double* w_out, int32_t* naux_out, cudaStream_t st) {
  if (nh <= 0 || np <= 0 || naux <= 0 || !B || !B_out || !naux_out || !isfinite(threshold)) return DSRG_FNO_ERR_ARG;
  if (precision != DSRG_FNO_FP64 && precision != DSRG_FNO_SLICED_BF16) return DSRG_FNO_ERR_UNSUPPORTED;
  if (!is_device_ptr(B) || !is_device_ptr(B_out) || (w_out && !is_device_ptr(w_out))) return DSRG_FNO_ERR_ARG;
  const long L = (long)nh * np;
  if (L * 2 > (1L << 31) || (long)naux * naux >= (1L << 31)) return DSRG_FNO_ERR_UNSUPPORTED;
  const size_t n2 = (size_t)naux * naux;
  const bool fast = precision == DSRG_FNO_SLICED_BF16;
  const int kw = 5, kb = 6;
  const int lpad = pad64((int)L), qpad = pad64(naux);
  size_t planes = 0;
  if (fast) {
    // the metric's planes, then (reusing the space) the rotation's
    const size_t p1 = ws_bytes((size_t)kw * naux * lpad, 2) + ws_bytes(naux, sizeof(int)) + ws_bytes(16, sizeof(int));
    const size_t p2 = ws_bytes((size_t)kb * L * qpad, 2) + ws_bytes((size_t)kb * naux * qpad, 2) +
                      ws_bytes(L, sizeof(int)) + ws_bytes(naux, sizeof(int)) + ws_bytes(16, sizeof(int));
    planes = std::max(p1, p2);
  }
  const size_t need = 3 * ws_bytes(n2, sizeof(double)) + ws_bytes(eig_work_doubles(naux), sizeof(double)) +
                      ws_bytes(naux + 16, sizeof(double)) + ws_bytes(naux + 16, sizeof(int)) + planes +
                      ws_bytes(8, sizeof(int));
  DSRG_TRY(ws_reserve(ws, need));
  {
    int* flag = ws_take<int>(ws, 8);
    int h = 0;
    DSRG_CUDA(cudaMemsetAsync(flag, 0, sizeof(int), st));
    DSRG_TRY(check_finite(B, (long)naux * L, flag, st));
    DSRG_CUDA(cudaMemcpyAsync(&h, flag, sizeof(int), cudaMemcpyDeviceToHost, st));
    DSRG_CUDA(cudaStreamSynchronize(st));
    if (h) return DSRG_FNO_ERR_NONFINITE;
  }
  double* W = ws_take<double>(ws, n2);
  double* V = ws_take<double>(ws, n2);
  double* U = ws_take<double>(ws, n2);
  double* work = ws_take<double>(ws, eig_work_doubles(naux));
  double* w = ws_take<double>(ws, naux + 16);
  int* ib = ws_take<int>(ws, naux + 16);
  if (!ib) return DSRG_FNO_ERR_NOMEM;
  const size_t base = ws.off;
  int* status = ib;
  int* rank = ib + 8;
  // ---- W = B2 B2^T, B2 = B as naux rows of length nh np
  {
    DSRG_PHASE("phase_naf_metric", st);
    if (fast) {
      ws.off = base;
      __nv_bfloat16* pl = ws_take<__nv_bfloat16>(ws, (size_t)kw * naux * lpad);
      int* ex = ws_take<int>(ws, naux);
      int* err = ws_take<int>(ws, 16);
      if (!err) return DSRG_FNO_ERR_NOMEM;
      DSRG_CUDA(cudaMemsetAsync(err, 0, sizeof(int), st));
      DSRG_TRY(slice_rows(kw, B, naux, (int)L, L, 1, lpad, pl, ex, st));
      DSRG_TRY(sliced_plain_gemm(kw, naux, naux, pl, ex, pl, ex, lpad, W, naux, err, st));
      int h = 0;
      DSRG_CUDA(cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, st));
      DSRG_CUDA(cudaStreamSynchronize(st));
      if (h) return DSRG_FNO_ERR_TIMEOUT;
    } else {
      DSRG_TRY(gemm_f64(naux, naux, (int)L, 1.0, B, L, true, B, L, true, 0.0, W, naux, 1, 0, 0, 0, st));
    }
  }
  // ---- W = U diag(w) U^T, w descending
  {
    DSRG_PHASE("phase_naf_eigen", st);
    DSRG_TRY(symmetrize(naux, W, st));
    DSRG_TRY(eig_sym_jacobi(naux, W, V, work, status, 60, st));
    DSRG_TRY(eig_sort(naux, W, V, w, U, rank, true, true, st));
  }
  std::vector<double> hw(naux);
  DSRG_CUDA(cudaMemcpyAsync(hw.data(), w, sizeof(double) * naux, cudaMemcpyDeviceToHost, st));
  DSRG_CUDA(cudaStreamSynchronize(st));
  int k = 0;
  while (k < naux && hw[k] > threshold) ++k;
  if (w_out) DSRG_CUDA(cudaMemcpyAsync(w_out, w, sizeof(double) * naux, cudaMemcpyDeviceToDevice, st));
  // ---- B'[K][ia] = sum_Q U[Q][K] B[Q][ia], K < k
  if (k > 0) {
    DSRG_PHASE("phase_naf_rotate", st);
    if (fast) {
      ws.off = base;
      __nv_bfloat16* pb = ws_take<__nv_bfloat16>(ws, (size_t)kb * L * qpad);
      __nv_bfloat16* pu = ws_take<__nv_bfloat16>(ws, (size_t)kb * naux * qpad);
      int* eb = ws_take<int>(ws, L);
      int* eu = ws_take<int>(ws, naux);
      int* err = ws_take<int>(ws, 16);
      if (!err) return DSRG_FNO_ERR_NOMEM;
      DSRG_CUDA(cudaMemsetAsync(err, 0, sizeof(int), st));
      // rows of U^T (eigenvector K over Q: stride naux) and of B2^T (column ia over Q: stride L)
      DSRG_TRY(slice_rows(kb, U, k, naux, 1, naux, qpad, pu, eu, st));
      DSRG_TRY(slice_rows(kb, B, L, naux, 1, L, qpad, pb, eb, st));
      DSRG_TRY(sliced_plain_gemm(kb, k, (int)L, pu, eu, pb, eb, qpad, B_out, L, err, st));
      int h = 0;
      DSRG_CUDA(cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, st));
      DSRG_CUDA(cudaStreamSynchronize(st));
      if (h) return DSRG_FNO_ERR_TIMEOUT;
    } else {
      DSRG_TRY(gemm_f64(k, (int)L, naux, 1.0, U, naux, false, B, L, false, 0.0, B_out, L, 1, 0, 0, 0, st));
    }
  }
  DSRG_CUDA(cudaStreamSynchronize(st));
  *naux_out = k;
  return DSRG_FNO_OK;
}

}  // namespace dsrg

using namespace dsrg;

extern "C" int dsrg_fno_naf(int32_t nh, int32_t np, int32_t naux, const double* B_hp, double threshold,
                            int32_t precision, double* B_out, double* w_out, int32_t* naux_out, void* stream) {
  std::lock_guard<std::mutex> lk(workspace_mutex());
  Workspace& ws = workspace_for_current_device();
  return impl_naf(ws, nh, np, naux, B_hp, threshold, precision, B_out, w_out, naux_out, (cudaStream_t)stream);
}
