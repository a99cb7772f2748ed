// Particle-particle ladder of Eq. 6 in the (truncated) virtual basis: the
// term of C2 = [O2, T2]_2 with four virtual indices, whose O(N_C^2 N_V^4)
// cost the FNO truncation cuts by (N_V'/N_V)^4:
//   C^{ij}_{ab} = sum_{cd} <ab|cd> T^{ij}_{cd},  <ab|cd> = sum_Q B^Q_{ac} B^Q_{bd}.
// Two contractions per block of A_BLK values of a:
//   1. I[(a c)][(b d)] = sum_Q B^Q_{ac} B^Q_{bd}          (M = A nv, N = nv^2, K = naux)
//      then the middle indices are swapped: I'[(a b)][(c d)]
//   2. C[p][(a b)] = sum_{(c d)} T[p][(c d)] I'[(a b)][(c d)]  (M = npairs, N = A nv, K = nv^2)
// Fast form: both on the digit-plane tensor-core kernel (5 planes); float64
// form: the float64 GEMM.  2 nv^4 (naux + npairs) flops in all.
#include <math.h>

#include "kernels.h"

namespace dsrg {

namespace {

// out[a][b][c][d] = in[a][c][b][d] for a < A (rows of d copied whole)
__global__ void swap_middle_kernel(int A, int nv, const double* __restrict__ in, double* __restrict__ out) {
  const long row = blockIdx.x;  // (a, b, c) of out
  const int c = (int)(row % nv);
  const long t = row / nv;
  const int b = (int)(t % nv);
  const int a = (int)(t / nv);
  const double* src = in + (((long)a * nv + c) * nv + b) * nv;
  double* dst = out + row * nv;
  for (int d = threadIdx.x; d < nv; d += blockDim.x) dst[d] = src[d];
}

}  // namespace

static const int LADDER_A_BLK = 16;

int impl_ladder(Workspace& ws, int32_t nv, int32_t naux, const double* Bvv, int32_t npairs, const double* T,
                int32_t precision, double* C, cudaStream_t st) {
  if (nv <= 0 || naux <= 0 || npairs <= 0 || !Bvv || !T || !C) return DSRG_FNO_ERR_ARG;
  if (precision != DSRG_FNO_FP64 && precision != DSRG_FNO_SLICED_BF16) return DSRG_FNO_ERR_UNSUPPORTED;
  if (!is_device_ptr(Bvv) || !is_device_ptr(T) || !is_device_ptr(C)) return DSRG_FNO_ERR_ARG;
  const long nv2 = (long)nv * nv;
  if (nv2 * LADDER_A_BLK * nv >= (1L << 31) || (long)npairs * nv2 >= (1L << 31)) return DSRG_FNO_ERR_UNSUPPORTED;
  const bool fast = precision == DSRG_FNO_SLICED_BF16;
  const int A = std::min(LADDER_A_BLK, (int)nv);
  const long blk = (long)A * nv;  // rows (a c) or (a b) of one block
  const int ks = 5;
  const int qpad = pad64(naux), vpad = pad64((int)nv2);
  size_t need = 2 * ws_bytes((size_t)blk * nv2, sizeof(double)) + ws_bytes(16, sizeof(int));
  if (fast)
    need += ws_bytes((size_t)ks * nv2 * qpad, 2) + ws_bytes((size_t)ks * blk * qpad, 2) +
            ws_bytes((size_t)ks * npairs * vpad, 2) + ws_bytes((size_t)ks * blk * vpad, 2) +
            ws_bytes(nv2, sizeof(int)) + ws_bytes(blk, sizeof(int)) + ws_bytes(npairs, sizeof(int)) +
            ws_bytes(blk + 16, sizeof(int));
  need += ws_bytes(8, sizeof(int));
  DSRG_TRY(ws_reserve(ws, need));
  {
    int* flag = ws_take<int>(ws, 8);
    int h = 0;
    DSRG_CUDA(cudaMemsetAsync(flag, 0, sizeof(int), st));
    DSRG_TRY(check_finite(Bvv, (long)naux * nv2, flag, st));
    DSRG_TRY(check_finite(T, (long)npairs * nv2, flag, st));
    DSRG_CUDA(cudaMemcpyAsync(&h, flag, sizeof(int), cudaMemcpyDeviceToHost, st));
    DSRG_CUDA(cudaStreamSynchronize(st));
    if (h) return DSRG_FNO_ERR_NONFINITE;
  }
  double* I1 = ws_take<double>(ws, (size_t)blk * nv2);
  double* I2 = ws_take<double>(ws, (size_t)blk * nv2);
  int* err = ws_take<int>(ws, 16);
  __nv_bfloat16 *pY = nullptr, *pX = nullptr, *pT = nullptr, *pI = nullptr;
  int *eY = nullptr, *eX = nullptr, *eT = nullptr, *eI = nullptr;
  if (fast) {
    pY = ws_take<__nv_bfloat16>(ws, (size_t)ks * nv2 * qpad);
    pX = ws_take<__nv_bfloat16>(ws, (size_t)ks * blk * qpad);
    pT = ws_take<__nv_bfloat16>(ws, (size_t)ks * npairs * vpad);
    pI = ws_take<__nv_bfloat16>(ws, (size_t)ks * blk * vpad);
    eY = ws_take<int>(ws, nv2);
    eX = ws_take<int>(ws, blk);
    eT = ws_take<int>(ws, npairs);
    eI = ws_take<int>(ws, blk + 16);
    if (!eI) return DSRG_FNO_ERR_NOMEM;
    DSRG_CUDA(cudaMemsetAsync(err, 0, sizeof(int), st));
    // rows (b d) of the factors over Q, and rows p of the amplitudes over (c d)
    DSRG_TRY(slice_rows(ks, Bvv, nv2, naux, 1, nv2, qpad, pY, eY, st));
    DSRG_TRY(slice_rows(ks, T, npairs, (int)nv2, nv2, 1, vpad, pT, eT, st));
  }
  for (int a0 = 0; a0 < nv; a0 += A) {
    const int na = std::min(A, nv - a0);
    const long rows = (long)na * nv;
    {
      DSRG_PHASE("phase_ladder_integrals", st);
      if (fast) {
        DSRG_TRY(slice_rows(ks, Bvv + (long)a0 * nv, rows, naux, 1, nv2, qpad, pX, eX, st));
        DSRG_TRY(sliced_plain_gemm(ks, (int)rows, (int)nv2, pX, eX, pY, eY, qpad, I1, nv2, err, st));
      } else {
        DSRG_TRY(gemm_f64((int)rows, (int)nv2, naux, 1.0, Bvv + (long)a0 * nv, nv2, false, Bvv, nv2, false, 0.0, I1,
                          nv2, 1, 0, 0, 0, st));
      }
      swap_middle_kernel<<<(unsigned)(rows * nv), 128, 0, st>>>(na, nv, I1, I2);
      DSRG_LAUNCH_CHECK();
    }
    {
      DSRG_PHASE("phase_ladder_contract", st);
      if (fast) {
        DSRG_TRY(slice_rows(ks, I2, rows, (int)nv2, nv2, 1, vpad, pI, eI, st));
        DSRG_TRY(sliced_plain_gemm(ks, npairs, (int)rows, pT, eT, pI, eI, vpad, C + (long)a0 * nv, nv2, err, st));
      } else {
        DSRG_TRY(gemm_f64(npairs, (int)rows, (int)nv2, 1.0, T, nv2, true, I2, nv2, true, 0.0, C + (long)a0 * nv, nv2,
                          1, 0, 0, 0, st));
      }
    }
  }
  int h = 0;
  if (fast) DSRG_CUDA(cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, st));
  DSRG_CUDA(cudaStreamSynchronize(st));
  return h ? DSRG_FNO_ERR_TIMEOUT : DSRG_FNO_OK;
}

}  // namespace dsrg

using namespace dsrg;

extern "C" int dsrg_fno_ladder(int32_t nv, int32_t naux, const double* B_vv, int32_t npairs, const double* T,
                               int32_t precision, double* C_out, void* stream) {
  std::lock_guard<std::mutex> lk(workspace_mutex());
  Workspace& ws = workspace_for_current_device();
  return impl_ladder(ws, nv, naux, B_vv, npairs, T, precision, C_out, (cudaStream_t)stream);
}
