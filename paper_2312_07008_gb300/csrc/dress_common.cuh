// Shared pieces of the dressing kernels (float64 and double-float forms):
// tile geometry, active-pair enumeration and the coefficients of the dressed
// matrices of one hole-pair group (see dress.cu for the derivation).
#pragma once
#include "kernels.h"

namespace dsrg {
namespace dressc {

constexpr int GT = 16;          // tile edge (16 x 16 elements, one per thread)
constexpr int GNT = 256;        // threads
constexpr int MAXSLOT = 136;    // slots of one group (nact <= 16: na (na+1) / 2)
constexpr double RSQ2 = 0.70710678118654752440;

// unordered active pair (u <= v) of index s in the row-major enumeration
__device__ inline void aa_sym_pair(int s, int na, int* uo, int* vo) {
  int u = 0;
  while (s >= na - u) {
    s -= na - u;
    ++u;
  }
  *uo = u;
  *vo = u + s;
}

__device__ inline int aa_pair_offset(int u, int v, int na) { return u * na - u * (u - 1) / 2 + (v - u); }

// the d-th strictly upper active pair (u < v)
__device__ inline void aa_anti_pair(int d, int na, int* uo, int* vo) {
  int u = 0;
  while (d >= na - 1 - u) {
    d -= na - 1 - u;
    ++u;
  }
  *uo = u;
  *vo = u + 1 + d;
}

// Coefficients of the outputs o_begin .. o_begin + o_count of one group:
//   sigma_o = sum_u cd[u][o] (tau_u + s_o dg_u tau_u^T),   lambda_o, s_o = +1 (sym) / -1 (antisym),
// dg_u = 0 for a slot whose tau is symmetric (a diagonal pair), else 1.
template <int OCT>
__device__ inline void group_coefficients(const DressDesc& D, const DressAux& X, int na, double (*cd)[OCT],
                                   double* lam, double* sgn, double* dg) {
  for (int idx = threadIdx.x; idx < D.nslots * OCT; idx += blockDim.x) cd[idx / OCT][idx % OCT] = 0.0;
  for (int u = threadIdx.x; u < D.nslots; u += blockDim.x) dg[u] = 1.0;
  __syncthreads();
  switch (D.kind) {
    case GROUP_CC_DIAG:  // sigma = tau^{mm}, lambda 2
      if (threadIdx.x == 0) {
        cd[0][0] = 1.0;
        lam[0] = 2.0;
        sgn[0] = 1.0;
        dg[0] = 0.0;
      }
      break;
    case GROUP_CC_PAIR:  // (tau +- tau^T)/sqrt2, lambda 2 and 6
      if (threadIdx.x == 0) {
        cd[0][0] = RSQ2;
        cd[0][1] = RSQ2;
        lam[0] = 2.0;
        lam[1] = 6.0;
        sgn[0] = 1.0;
        sgn[1] = -1.0;
      }
      break;
    case GROUP_CA:  // output 2k: sum_u W[u][k] (tau^{mu} + tau^{mu T})/sqrt2 (g_k); 2k+1: minus (3 g_k)
      for (int idx = threadIdx.x; idx < D.nslots * D.o_count; idx += blockDim.x) {
        const int u = idx / D.o_count, ol = idx % D.o_count, o = D.o_begin + ol, k = o >> 1;
        cd[u][ol] = X.g1_evec[u * na + k] * RSQ2;
        if (u == 0) {
          const double gk = X.g1_eval[k * (na + 1)];
          lam[ol] = (o & 1) ? 3.0 * gk : gk;
          sgn[ol] = (o & 1) ? -1.0 : 1.0;
        }
      }
      break;
    case GROUP_AA: {  // outputs < ns: symmetric-block eigenvectors; then antisymmetric block
      const int ns = na * (na + 1) / 2, nd = na * (na - 1) / 2;
      for (int u = threadIdx.x; u < D.nslots; u += blockDim.x) {
        int a, b;
        aa_sym_pair(u, na, &a, &b);
        if (a == b) dg[u] = 0.0;
      }
      for (int ol = threadIdx.x; ol < D.o_count; ol += blockDim.x) {
        const int o = D.o_begin + ol;
        if (o < ns) {
          lam[ol] = X.aas_eval[o * (ns + 1)];
          sgn[ol] = 1.0;
          for (int u = 0; u < ns; ++u) {
            int a, b;
            aa_sym_pair(u, na, &a, &b);
            const double y = X.aas_evec[u * ns + o];
            cd[u][ol] = (a == b) ? y : y * RSQ2;
          }
        } else {
          const int k = o - ns;
          lam[ol] = X.aaa_eval[k * (nd + 1)];
          sgn[ol] = -1.0;
          for (int d = 0; d < nd; ++d) {
            int a, b;
            aa_anti_pair(d, na, &a, &b);
            cd[aa_pair_offset(a, b, na)][ol] = X.aaa_evec[d * nd + k] * RSQ2;
          }
        }
      }
      break;
    }
  }
  __syncthreads();
}


}  // namespace dressc
}  // namespace dsrg
