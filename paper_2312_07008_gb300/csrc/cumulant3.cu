// State-averaged spin-free 3-cumulant Lambda^{xyz}_{uvw} (the 3-body density
// cumulant that Eq. A12 term 13 contracts), dsrg_fno_sa_lambda3.
//
// The ensemble 3-RDM is the weighted sum of the per-state spin-free 3-RDMs
// (Eq. A1 applied to three-body densities).  The cumulant is the spin-orbital
// one (Gamma3 minus its antisymmetrised Gamma1 x lambda2 and Gamma1^3 parts)
// summed over the spins of the index pairs (x,u), (y,v), (z,w), with the
// spin-orbital 1-RDM Gamma1 / 2 for either spin:
//   - a Gamma1 that joins an upper index to its own lower partner enters with
//     weight 1, one that joins it to another lower index ties two spins and
//     enters with 1/2, the remaining pair of the 2-cumulant following the spins;
//   - a Gamma1^3 product of a permutation P of the lower indices enters with
//     sign(P) 2^(cycles(P) - 3).
// As for Lambda2, the cumulant of the averaged densities is formed, not an
// average of per-state cumulants.
#include <math.h>

#include "kernels.h"

namespace dsrg {
namespace {

constexpr int L3_MAX_STATES = 32;

struct L3Weights {
  int nstates;
  double w[L3_MAX_STATES];
};

// one thread per element, index ((((x na + y) na + z) na + u) na + v) na + w
__global__ void lambda3_kernel(int na, L3Weights W, const double* __restrict__ g1, const double* __restrict__ l2,
                               const double* __restrict__ g3s, double* __restrict__ out) {
  const long n2 = (long)na * na, n3 = n2 * na, n6 = n3 * n3;
  const long idx = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (idx >= n6) return;
  long r = idx;
  const int w = (int)(r % na);
  r /= na;
  const int v = (int)(r % na);
  r /= na;
  const int u = (int)(r % na);
  r /= na;
  const int z = (int)(r % na);
  r /= na;
  const int y = (int)(r % na);
  const int x = (int)(r / na);
  auto G = [&](int a, int b) { return g1[a * na + b]; };
  auto L = [&](int a, int b, int c, int d) { return l2[((a * na + b) * na + c) * na + d]; };
  double g3 = 0.0;
  for (int k = 0; k < W.nstates; ++k) g3 = fma(W.w[k], g3s[k * n6 + idx], g3);
  // Gamma1 x Lambda2, diagonal links
  const double d1 = G(x, u) * L(y, z, v, w) + G(y, v) * L(x, z, u, w) + G(z, w) * L(x, y, u, v);
  // Gamma1 x Lambda2, cross links (weight 1/2)
  const double d2 = G(x, v) * L(y, z, u, w) + G(x, w) * L(y, z, v, u) + G(y, u) * L(x, z, v, w) +
                    G(y, w) * L(x, z, u, v) + G(z, u) * L(x, y, w, v) + G(z, v) * L(x, y, u, w);
  // Gamma1^3: identity, the three transpositions, the two 3-cycles
  const double p0 = G(x, u) * G(y, v) * G(z, w);
  const double p2 = G(x, v) * G(y, u) * G(z, w) + G(x, w) * G(y, v) * G(z, u) + G(x, u) * G(y, w) * G(z, v);
  const double p3 = G(x, v) * G(y, w) * G(z, u) + G(x, w) * G(y, u) * G(z, v);
  out[idx] = g3 - d1 + 0.5 * d2 - p0 + 0.5 * p2 - 0.25 * p3;
}

}  // namespace
}  // namespace dsrg

using namespace dsrg;

extern "C" int dsrg_fno_sa_lambda3(int32_t nact, int32_t nstates, const double* weights, const double* gamma1,
                                   const double* lambda2, const double* gamma3_states, double* lambda3_out,
                                   void* stream) {
  if (nact < 1 || nact > 16 || nstates < 1 || nstates > L3_MAX_STATES || !weights) return DSRG_FNO_ERR_ARG;
  if (!gamma1 || !lambda2 || !gamma3_states || !lambda3_out) return DSRG_FNO_ERR_ARG;
  L3Weights W{};
  W.nstates = nstates;
  double sum = 0.0;
  for (int k = 0; k < nstates; ++k) {
    if (!(weights[k] >= 0.0) || !isfinite(weights[k])) return DSRG_FNO_ERR_ARG;
    W.w[k] = weights[k];
    sum += weights[k];
  }
  if (fabs(sum - 1.0) > 1e-12) return DSRG_FNO_ERR_ARG;
  for (const void* p : {(const void*)gamma1, (const void*)lambda2, (const void*)gamma3_states,
                        (const void*)lambda3_out}) {
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
      cudaGetLastError();
      return DSRG_FNO_ERR_ARG;
    }
    if (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged) return DSRG_FNO_ERR_ARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  const long n3 = (long)nact * nact * nact, n6 = n3 * n3;
  lambda3_kernel<<<ceil_div(n6, 256), 256, 0, st>>>(nact, W, gamma1, lambda2, gamma3_states, lambda3_out);
  DSRG_LAUNCH_CHECK();
  std::lock_guard<std::mutex> lk(workspace_mutex());
  Workspace& ws = workspace_for_current_device();
  DSRG_TRY(ws_reserve(ws, 256));
  int* flag = ws_take<int>(ws, 8);
  DSRG_CUDA(cudaMemsetAsync(flag, 0, sizeof(int), st));
  DSRG_TRY(check_finite(lambda3_out, n6, flag, st));
  int h = 0;
  DSRG_CUDA(cudaMemcpyAsync(&h, flag, sizeof(int), cudaMemcpyDeviceToHost, st));
  DSRG_CUDA(cudaStreamSynchronize(st));
  return h ? DSRG_FNO_ERR_NONFINITE : DSRG_FNO_OK;
}
