// State-averaged densities of Eq. A1 (host helper, dsrg_fno_sa_densities).
//
// Gamma1 and Gamma2 of the ensemble are the weighted sums of the per-state
// spin-free densities; the 2-cumulant of the ensemble follows from them by the
// spin-free relation Gamma^{uv}_{xy} = Lambda^{uv}_{xy} + Gamma^u_x Gamma^v_y
// - 1/2 Gamma^v_x Gamma^u_y (definitions after Eq. A12).  It is formed from the
// averaged Gamma1 and Gamma2, not as an average of per-state cumulants.
#include <math.h>

#include "kernels.h"

extern "C" int dsrg_fno_sa_densities(int32_t nact, int32_t nstates, const double* w, const double* g1_states,
                                     const double* g2_states, double* gamma1_out, double* lambda2_out) {
  if (nact < 1 || nstates < 1 || !w || !g1_states || !g2_states || !gamma1_out || !lambda2_out)
    return DSRG_FNO_ERR_ARG;
  double sum = 0.0;
  for (int a = 0; a < nstates; ++a) {
    if (!(w[a] >= 0.0) || !isfinite(w[a])) return DSRG_FNO_ERR_ARG;
    sum += w[a];
  }
  if (fabs(sum - 1.0) > 1e-12) return DSRG_FNO_ERR_ARG;
  const long n = nact, n2 = n * n, n4 = n2 * n2;
  for (long k = 0; k < n2; ++k) {
    double g = 0.0;
    for (int a = 0; a < nstates; ++a) g += w[a] * g1_states[a * n2 + k];
    gamma1_out[k] = g;
  }
  for (long u = 0; u < n; ++u)
    for (long v = 0; v < n; ++v)
      for (long x = 0; x < n; ++x)
        for (long y = 0; y < n; ++y) {
          const long k = ((u * n + v) * n + x) * n + y;
          double g2 = 0.0;
          for (int a = 0; a < nstates; ++a) g2 += w[a] * g2_states[a * n4 + k];
          lambda2_out[k] = g2 - gamma1_out[u * n + x] * gamma1_out[v * n + y] +
                           0.5 * gamma1_out[u * n + y] * gamma1_out[v * n + x];
        }
  for (long k = 0; k < n4; ++k)
    if (!isfinite(lambda2_out[k])) return DSRG_FNO_ERR_NONFINITE;
  return DSRG_FNO_OK;
}
