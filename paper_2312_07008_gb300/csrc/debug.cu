// Test hooks of the fast form (include/dsrg_fno_debug.h).
#include <cuda_bf16.h>

#include <vector>

#include "../../include/dsrg_fno_debug.h"
#include "kernels.h"
#include "mma_schedule.cuh"

using namespace dsrg;

namespace {
struct DevBuf {
  void* p = nullptr;
  ~DevBuf() {
    if (p) cudaFree(p);
  }
};
}  // namespace

extern "C" int dsrg_fno_debug_sliced_gemm(int32_t ks, int32_t M, int32_t N, int32_t K, const double* A,
                                          const double* B, double* C) {
  if (ks < 3 || ks > 6 || M <= 0 || N <= 0 || K <= 0 || !A || !B || !C) return DSRG_FNO_ERR_ARG;
  const int kp = pad64(K);
  DevBuf dA, dB, dC, pa, pb, ea, eb, err;
  DSRG_CUDA(cudaMalloc(&dA.p, sizeof(double) * M * K));
  DSRG_CUDA(cudaMalloc(&dB.p, sizeof(double) * N * K));
  DSRG_CUDA(cudaMalloc(&dC.p, sizeof(double) * M * N));
  DSRG_CUDA(cudaMalloc(&pa.p, 2L * ks * M * kp));
  DSRG_CUDA(cudaMalloc(&pb.p, 2L * ks * N * kp));
  DSRG_CUDA(cudaMalloc(&ea.p, sizeof(int) * M));
  DSRG_CUDA(cudaMalloc(&eb.p, sizeof(int) * N));
  DSRG_CUDA(cudaMalloc(&err.p, sizeof(int)));
  DSRG_CUDA(cudaMemset(err.p, 0, sizeof(int)));
  DSRG_CUDA(cudaMemcpy(dA.p, A, sizeof(double) * M * K, cudaMemcpyHostToDevice));
  DSRG_CUDA(cudaMemcpy(dB.p, B, sizeof(double) * N * K, cudaMemcpyHostToDevice));
  cudaStream_t st = 0;
  DSRG_TRY(slice_rows(ks, (double*)dA.p, M, K, K, 1, kp, (__nv_bfloat16*)pa.p, (int*)ea.p, st));
  DSRG_TRY(slice_rows(ks, (double*)dB.p, N, K, K, 1, kp, (__nv_bfloat16*)pb.p, (int*)eb.p, st));
  DSRG_TRY(sliced_plain_gemm(ks, M, N, (__nv_bfloat16*)pa.p, (int*)ea.p, (__nv_bfloat16*)pb.p, (int*)eb.p, kp,
                             (double*)dC.p, N, (int*)err.p, st));
  DSRG_CUDA(cudaDeviceSynchronize());
  int h = 0;
  DSRG_CUDA(cudaMemcpy(&h, err.p, sizeof(int), cudaMemcpyDeviceToHost));
  DSRG_CUDA(cudaMemcpy(C, dC.p, sizeof(double) * M * N, cudaMemcpyDeviceToHost));
  return h ? DSRG_FNO_ERR_TIMEOUT : DSRG_FNO_OK;
}

extern "C" int dsrg_fno_debug_slice_rows(int32_t ks, int32_t R, int32_t K, const double* rows, float* planes,
                                         int32_t* exps) {
  if (ks < 3 || ks > 6 || R <= 0 || K <= 0 || !rows || !planes || !exps) return DSRG_FNO_ERR_ARG;
  const int kp = pad64(K);
  DevBuf d, p, e;
  DSRG_CUDA(cudaMalloc(&d.p, sizeof(double) * R * K));
  DSRG_CUDA(cudaMalloc(&p.p, 2L * ks * R * kp));
  DSRG_CUDA(cudaMalloc(&e.p, sizeof(int) * R));
  DSRG_CUDA(cudaMemcpy(d.p, rows, sizeof(double) * R * K, cudaMemcpyHostToDevice));
  DSRG_TRY(slice_rows(ks, (double*)d.p, R, K, K, 1, kp, (__nv_bfloat16*)p.p, (int*)e.p, 0));
  DSRG_CUDA(cudaDeviceSynchronize());
  std::vector<__nv_bfloat16> h((size_t)ks * R * kp);
  DSRG_CUDA(cudaMemcpy(h.data(), p.p, h.size() * 2, cudaMemcpyDeviceToHost));
  for (size_t i = 0; i < h.size(); ++i) planes[i] = __bfloat162float(h[i]);
  DSRG_CUDA(cudaMemcpy(exps, e.p, sizeof(int) * R, cudaMemcpyDeviceToHost));
  return DSRG_FNO_OK;
}

extern "C" int dsrg_fno_debug_slice_rows_dd(int32_t ks, int32_t R, int32_t K, const float* rows, float* planes,
                                            int32_t* exps) {
  if (ks < 3 || ks > 5 || R <= 0 || K <= 0 || !rows || !planes || !exps) return DSRG_FNO_ERR_ARG;
  const int kp = pad64(K);
  DevBuf d, p, e;
  DSRG_CUDA(cudaMalloc(&d.p, sizeof(float2) * R * K));
  DSRG_CUDA(cudaMalloc(&p.p, 2L * ks * R * kp));
  DSRG_CUDA(cudaMalloc(&e.p, sizeof(int) * R));
  DSRG_CUDA(cudaMemcpy(d.p, rows, sizeof(float2) * R * K, cudaMemcpyHostToDevice));
  DSRG_TRY(slice_rows_dd(ks, (float2*)d.p, R, K, K, 1, kp, (__nv_bfloat16*)p.p, (int*)e.p, nullptr, 0));
  DSRG_CUDA(cudaDeviceSynchronize());
  std::vector<__nv_bfloat16> h((size_t)ks * R * kp);
  DSRG_CUDA(cudaMemcpy(h.data(), p.p, h.size() * 2, cudaMemcpyDeviceToHost));
  for (size_t i = 0; i < h.size(); ++i) planes[i] = __bfloat162float(h[i]);
  DSRG_CUDA(cudaMemcpy(exps, e.p, sizeof(int) * R, cudaMemcpyDeviceToHost));
  return DSRG_FNO_OK;
}

extern "C" int dsrg_fno_debug_regularizer(int32_t n, const double* delta, double s, double* r1, double* y) {
  if (n <= 0 || !delta || !r1 || !y || !(s >= 0.0)) return DSRG_FNO_ERR_ARG;
  DevBuf d, a, b;
  DSRG_CUDA(cudaMalloc(&d.p, sizeof(double) * n));
  DSRG_CUDA(cudaMalloc(&a.p, sizeof(double) * n));
  DSRG_CUDA(cudaMalloc(&b.p, sizeof(double) * n));
  DSRG_CUDA(cudaMemcpy(d.p, delta, sizeof(double) * n, cudaMemcpyHostToDevice));
  DSRG_TRY(regularize_test(n, (double*)d.p, s, (double*)a.p, (double*)b.p, 0));
  DSRG_CUDA(cudaDeviceSynchronize());
  DSRG_CUDA(cudaMemcpy(r1, a.p, sizeof(double) * n, cudaMemcpyDeviceToHost));
  DSRG_CUDA(cudaMemcpy(y, b.p, sizeof(double) * n, cudaMemcpyDeviceToHost));
  return DSRG_FNO_OK;
}

extern "C" int dsrg_fno_debug_mma_schedule(int32_t ks, int32_t* entries, int32_t max_entries) {
  if (ks < 3 || ks > 6 || !entries) return DSRG_FNO_ERR_ARG;
  const int n = stacked_mma_count(ks);
  if (max_entries < n) return DSRG_FNO_ERR_ARG;
  for (int i = 0; i < n; ++i) {
    const StackedMma m = stacked_mma(ks, i);
    entries[5 * i + 0] = m.a;
    entries[5 * i + 1] = m.b0;
    entries[5 * i + 2] = m.nb;
    entries[5 * i + 3] = m.level;
    entries[5 * i + 4] = m.nb * plane_tile_n(ks);
  }
  return n;
}

extern "C" int dsrg_fno_debug_eig_batch(int32_t count, const int32_t* n, double* const* A, double* const* V) {
  if (count < 1 || count > 4 || !n || !A || !V) return DSRG_FNO_ERR_ARG;
  for (int e = 0; e < count; ++e)
    if (n[e] < 0 || n[e] > 4096 || (n[e] > 0 && (!A[e] || !V[e]))) return DSRG_FNO_ERR_ARG;
  DevBuf dA[4], dV[4], dW[4], stat;
  double *pa[4] = {}, *pv[4] = {}, *pw[4] = {};
  int nn[4] = {};
  for (int e = 0; e < count; ++e) {
    nn[e] = n[e];
    const size_t n2 = (size_t)n[e] * n[e];
    DSRG_CUDA(cudaMalloc(&dA[e].p, sizeof(double) * (n2 + 1)));
    DSRG_CUDA(cudaMalloc(&dV[e].p, sizeof(double) * (n2 + 1)));
    DSRG_CUDA(cudaMalloc(&dW[e].p, sizeof(double) * eig_work_doubles(n[e])));
    if (n2) DSRG_CUDA(cudaMemcpy(dA[e].p, A[e], sizeof(double) * n2, cudaMemcpyHostToDevice));
    pa[e] = (double*)dA[e].p;
    pv[e] = (double*)dV[e].p;
    pw[e] = (double*)dW[e].p;
  }
  DSRG_CUDA(cudaMalloc(&stat.p, sizeof(int) * 16));
  const int rc = eig_sym_jacobi_batch(count, nn, pa, pv, pw, (int*)stat.p, 60, 0);
  DSRG_CUDA(cudaDeviceSynchronize());
  if (rc != DSRG_FNO_OK) return rc;
  for (int e = 0; e < count; ++e) {
    const size_t n2 = (size_t)n[e] * n[e];
    if (!n2) continue;
    DSRG_CUDA(cudaMemcpy(A[e], pa[e], sizeof(double) * n2, cudaMemcpyDeviceToHost));
    DSRG_CUDA(cudaMemcpy(V[e], pv[e], sizeof(double) * n2, cudaMemcpyDeviceToHost));
  }
  return DSRG_FNO_OK;
}

extern "C" int64_t dsrg_fno_debug_workspace_bytes(void) {
  std::lock_guard<std::mutex> lk(workspace_mutex());
  return (int64_t)workspace_for_current_device().cap;
}

extern "C" int dsrg_fno_debug_pair_tiles(int32_t nslices, int32_t ncore, int32_t nact, int32_t nvir,
                                         const int32_t* pairs, int32_t npairs, int32_t energy_only,
                                         int32_t* tiles, int32_t max_tiles) {
  if (nslices < 3 || nslices > 5 || ncore < 0 || nact < 0 || nvir <= 0 || ncore + nact <= 0 || npairs < 0 ||
      (npairs > 0 && !pairs) || !tiles)
    return DSRG_FNO_ERR_ARG;
  Geometry g{};
  g.nc = ncore;
  g.na = nact;
  g.nv = nvir;
  g.nh = ncore + nact;
  g.np = nact + nvir;
  std::vector<int2> pr(npairs), out;
  for (int k = 0; k < npairs; ++k) {
    pr[k] = make_int2(pairs[2 * k], pairs[2 * k + 1]);
    if (pr[k].x < 0 || pr[k].y < pr[k].x || pr[k].y >= g.nh) return DSRG_FNO_ERR_ARG;
  }
  const int bn = pair_tile_n(FORM_DIGITS, nslices);
  DSRG_TRY(pair_tiles(bn, g, pr.data(), npairs, energy_only != 0, out));
  if ((long)out.size() > max_tiles || (long)out.size() > pair_tile_bound(bn, g, npairs)) return DSRG_FNO_ERR_ARG;
  for (size_t t = 0; t < out.size(); ++t) {
    tiles[2 * t] = out[t].x;
    tiles[2 * t + 1] = out[t].y;
  }
  return (int)out.size();
}

extern "C" int dsrg_fno_debug_set_barrier_limit(int64_t spins) {
  std::lock_guard<std::mutex> lk(workspace_mutex());
  return eig_set_barrier_limit((long long)spins);
}

extern "C" int dsrg_fno_debug_literal_gemm(int32_t precision, int32_t nterms, int32_t M, int32_t N, int32_t K,
                                           const double* A, const double* B, double* C) {
  int form, parts;
  if (precision == DSRG_FNO_BF16X3 && (nterms == 0 || nterms == 3)) {
    form = FORM_BF16X3;
    parts = 2;
  } else if (precision == DSRG_FNO_TF32 && (nterms == 0 || nterms == 1 || nterms == 3)) {
    form = FORM_TF32;
    parts = nterms == 1 ? 1 : 2;
  } else {
    return DSRG_FNO_ERR_ARG;
  }
  if (M <= 0 || N <= 0 || K <= 0 || !A || !B || !C) return DSRG_FNO_ERR_ARG;
  const int kp = pad64(K);
  const int eb = form == FORM_TF32 ? 4 : 2;
  DevBuf dA, dB, dC, pa, pb, ea, eb_, err;
  DSRG_CUDA(cudaMalloc(&dA.p, sizeof(double) * M * K));
  DSRG_CUDA(cudaMalloc(&dB.p, sizeof(double) * N * K));
  DSRG_CUDA(cudaMalloc(&dC.p, sizeof(double) * M * N));
  DSRG_CUDA(cudaMalloc(&pa.p, (size_t)eb * parts * M * kp));
  DSRG_CUDA(cudaMalloc(&pb.p, (size_t)eb * parts * N * kp));
  DSRG_CUDA(cudaMalloc(&ea.p, sizeof(int) * M));
  DSRG_CUDA(cudaMalloc(&eb_.p, sizeof(int) * N));
  DSRG_CUDA(cudaMalloc(&err.p, sizeof(int)));
  DSRG_CUDA(cudaMemset(err.p, 0, sizeof(int)));
  DSRG_CUDA(cudaMemcpy(dA.p, A, sizeof(double) * M * K, cudaMemcpyHostToDevice));
  DSRG_CUDA(cudaMemcpy(dB.p, B, sizeof(double) * N * K, cudaMemcpyHostToDevice));
  cudaStream_t st = 0;
  DSRG_TRY(stage_literal(form, parts, (double*)dA.p, M, K, K, 1, kp, pa.p, (int*)ea.p, st));
  DSRG_TRY(stage_literal(form, parts, (double*)dB.p, N, K, K, 1, kp, pb.p, (int*)eb_.p, st));
  DSRG_TRY(sliced_plain_gemm(parts, M, N, pa.p, (int*)ea.p, pb.p, (int*)eb_.p, kp, (double*)dC.p, N, (int*)err.p, st,
                             form));
  int h = 0;
  DSRG_CUDA(cudaMemcpy(&h, err.p, sizeof(int), cudaMemcpyDeviceToHost));
  if (h) return DSRG_FNO_ERR_TIMEOUT;
  DSRG_CUDA(cudaMemcpy(C, dC.p, sizeof(double) * M * N, cudaMemcpyDeviceToHost));
  return DSRG_FNO_OK;
}

extern "C" int dsrg_fno_debug_set_fused_epilogue(int32_t on) {
  std::lock_guard<std::mutex> lk(workspace_mutex());
  set_fused_epilogue(on != 0);
  return DSRG_FNO_OK;
}

extern "C" int dsrg_fno_debug_set_syrk_planes(int32_t nslices) {
  if (nslices != 0 && (nslices < 3 || nslices > 5)) return DSRG_FNO_ERR_ARG;
  std::lock_guard<std::mutex> lk(workspace_mutex());
  set_syrk_planes(nslices);
  return DSRG_FNO_OK;
}

extern "C" int dsrg_fno_debug_set_eig_colpair(int32_t on) {
  std::lock_guard<std::mutex> lk(workspace_mutex());
  set_eig_colpair(on != 0);
  return DSRG_FNO_OK;
}
