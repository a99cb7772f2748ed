// Dressing of the vv-class amplitudes by the SA 2-RDM over holes.
//
// With both particles virtual, the vv-class parts of D_vv (Eq. A12 terms 4,
// 5, 7) and of the energy (Eq. A4 scalar) read
//   D_ef = 1/2 sum_{kl,ij} G[kl][ij] (tau^{kl} tau^{ij T} + tau^{kl T} tau^{ij})_ef
//   E    = 1/2 sum_{kl,ij} G[kl][ij] <tau^{ij}, kappa^{kl}>,   kappa = 2 nu - Delta tau
// where G is the spin-free SA 2-RDM over holes (Gamma^{kl}_{ij} = Lambda +
// Gamma^k_i Gamma^l_j - 1/2 Gamma^l_i Gamma^k_j, core Gamma = 2 delta).  G
// couples only pairs of one group: {mn, nm} (core-core), {mu, um}_u for a
// fixed core m, and all active pairs.  In each group G is diagonalised in a
// basis that is symmetric or antisymmetric under the pair swap, so every
// dressed matrix sigma_r = sum_a U_r[a] tau^a is symmetric or antisymmetric
// and the group contributes
//   D += sum_r lambda_r sigma_r sigma_r^T,   E += 1/2 sum_r lambda_r <sigma_r[tau], sigma_r[kappa]>.
// Core-core:   G = [[4,-2],[-2,4]]  -> lambda 2 (sym), 6 (antisym); diagonal pair 2.
// Core-active: G = [[2,-1],[-1,2]] (x) Gamma1 -> lambda g_k (sym), 3 g_k (antisym).
// Active:      eigen-decomposition of the aa block of G (computed on device).
#include "kernels.h"

namespace dsrg {

namespace {

constexpr int DT = 32;         // tile edge
constexpr int DNT = 256;       // threads (32 x 8)
constexpr int MAXENT = 136;    // entries of one dressed matrix (nact <= 16)
constexpr double RSQ2 = 0.70710678118654752440;

struct Ent {
  int slot;
  double cd, ct;  // coefficient of tau^{slot} and of its transpose
};

__device__ int aa_pair_offset(int u, int v, int na) {
  // offset of unordered pair (u <= v) in the row-major enumeration u<=v
  return u * na - u * (u - 1) / 2 + (v - u);
}

// decode the d-th strictly-upper pair (u < v)
__device__ void aa_anti_pair(int d, int na, int* uo, int* vo) {
  int u = 0;
  while (d >= na - 1 - u) {
    d -= na - 1 - u;
    ++u;
  }
  *uo = u;
  *vo = u + 1 + d;
}

__device__ void build_entries(const DressDesc& D, const DressAux& X, int na, Ent* ent, int* nent,
                              double* lam) {
  const int t = threadIdx.x;
  switch (D.kind) {
    case DRESS_CC_DIAG:
      if (t == 0) {
        ent[0] = {D.slot, 1.0, 0.0};
        *nent = 1;
        *lam = 2.0;
      }
      break;
    case DRESS_CC_SYM:
    case DRESS_CC_ANTI:
      if (t == 0) {
        ent[0] = {D.slot, RSQ2, D.kind == DRESS_CC_SYM ? RSQ2 : -RSQ2};
        *nent = 1;
        *lam = D.kind == DRESS_CC_SYM ? 2.0 : 6.0;
      }
      break;
    case DRESS_CA_SYM:
    case DRESS_CA_ANTI: {
      const int k = D.a;
      if (t < na) {
        double w = X.g1_evec[t * na + k] * RSQ2;
        ent[t] = {D.slot + t, w, D.kind == DRESS_CA_SYM ? w : -w};
      }
      if (t == 0) {
        *nent = na;
        double g = X.g1_eval[k * (na + 1)];
        *lam = D.kind == DRESS_CA_SYM ? g : 3.0 * g;
      }
      break;
    }
    case DRESS_AA_SYM: {
      const int ns = na * (na + 1) / 2, k = D.a;
      for (int s = t; s < ns; s += blockDim.x) {
        // s enumerates (u <= v) in the same order as the aa slots
        int u = 0, rem = s;
        while (rem >= na - u) {
          rem -= na - u;
          ++u;
        }
        int v = u + rem;
        double y = X.aas_evec[s * ns + k];
        if (u == v) ent[s] = {D.slot + s, y, 0.0};
        else ent[s] = {D.slot + s, y * RSQ2, y * RSQ2};
      }
      if (t == 0) {
        *nent = ns;
        *lam = X.aas_eval[k * (ns + 1)];
      }
      break;
    }
    case DRESS_AA_ANTI: {
      const int nd = na * (na - 1) / 2, k = D.a;
      for (int d = t; d < nd; d += blockDim.x) {
        int u, v;
        aa_anti_pair(d, na, &u, &v);
        double y = X.aaa_evec[d * nd + k] * RSQ2;
        ent[d] = {D.slot + aa_pair_offset(u, v, na), y, -y};
      }
      if (t == 0) {
        *nent = nd;
        *lam = X.aaa_eval[k * (nd + 1)];
      }
      break;
    }
  }
}

__global__ void __launch_bounds__(DNT) dress_kernel(int nv, int na, const DressDesc* __restrict__ desc,
                                                    DressAux aux, const double* __restrict__ tau,
                                                    const double* __restrict__ kap,
                                                    double* __restrict__ sig, double* __restrict__ sig_sign,
                                                    double* __restrict__ e_part, int want_sig) {
  __shared__ Ent ent[MAXENT];
  __shared__ int nent;
  __shared__ double lam;
  __shared__ double tT[DT][DT + 1], tK[DT][DT + 1];
  __shared__ double red[DNT / 32];
  const DressDesc D = desc[blockIdx.y];
  build_entries(D, aux, na, ent, &nent, &lam);
  __syncthreads();
  const int ntd = (nv + DT - 1) / DT;
  const int E0 = (blockIdx.x / ntd) * DT, F0 = (blockIdx.x % ntd) * DT;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8
  const long nv2 = (long)nv * nv;
  double st[4] = {0, 0, 0, 0}, sk[4] = {0, 0, 0, 0};
  for (int q = 0; q < nent; ++q) {
    const Ent en = ent[q];
    const double* T = tau + (long)en.slot * nv2;
    const double* K = kap + (long)en.slot * nv2;
    // transposed tile: tT[fl][el] = T[F0+fl][E0+el]
    if (en.ct != 0.0) {
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        int fl = ty + 8 * r, f = F0 + fl, e = E0 + tx;
        double a = 0.0, b = 0.0;
        if (f < nv && e < nv) {
          a = T[(long)f * nv + e];
          b = K[(long)f * nv + e];
        }
        tT[fl][tx] = a;
        tK[fl][tx] = b;
      }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      int el = ty + 8 * r, e = E0 + el, f = F0 + tx;
      if (e < nv && f < nv) {
        double a = en.cd * T[(long)e * nv + f];
        double b = en.cd * K[(long)e * nv + f];
        if (en.ct != 0.0) {
          a = fma(en.ct, tT[tx][el], a);
          b = fma(en.ct, tK[tx][el], b);
        }
        st[r] += a;
        sk[r] += b;
      }
    }
    __syncthreads();
  }
  const double l = lam;
  const double sq = sqrt(fabs(l));
  double part = 0.0;
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    int e = E0 + ty + 8 * r, f = F0 + tx;
    if (e < nv && f < nv) {
      part = fma(st[r], sk[r], part);
      if (want_sig) sig[(long)D.out * nv2 + (long)e * nv + f] = sq * st[r];
    }
  }
  // warp then block reduction, fixed order
  for (int o = 16; o > 0; o >>= 1) part += __shfl_down_sync(0xffffffffu, part, o);
  if (tx == 0) red[ty] = part;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < DNT / 32; ++w) s += red[w];
    e_part[(long)blockIdx.y * gridDim.x + blockIdx.x] = 0.5 * l * s;
    if (want_sig && blockIdx.x == 0) sig_sign[D.out] = (l >= 0.0) ? 1.0 : -1.0;
  }
}

// aa block of G in the swap-symmetric (sym) and swap-antisymmetric (anti) bases
__global__ void aa_blocks_kernel(int na, const double* __restrict__ g1, const double* __restrict__ lam2,
                                 double* Ms, double* Ma) {
  const int ns = na * (na + 1) / 2, nd = na * (na - 1) / 2;
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  auto G2 = [&](int u, int v, int x, int y) {
    return lam2[((u * na + v) * na + x) * na + y] + g1[u * na + x] * g1[v * na + y] -
           0.5 * g1[v * na + x] * g1[u * na + y];
  };
  auto sym_pair = [&](int s, int* u, int* v) {
    int uu = 0, rem = s;
    while (rem >= na - uu) {
      rem -= na - uu;
      ++uu;
    }
    *u = uu;
    *v = uu + rem;
  };
  if (idx < ns * ns) {
    int s = idx / ns, t = idx % ns, u, v, x, y;
    sym_pair(s, &u, &v);
    sym_pair(t, &x, &y);
    double cs = (u == v) ? 1.0 : RSQ2, ct = (x == y) ? 1.0 : RSQ2;
    double val;
    if (u == v && x == y) val = G2(u, u, x, x);
    else if (u == v) val = ct * (G2(u, u, x, y) + G2(u, u, y, x));
    else if (x == y) val = cs * (G2(u, v, x, x) + G2(v, u, x, x));
    else val = cs * ct * (G2(u, v, x, y) + G2(u, v, y, x) + G2(v, u, x, y) + G2(v, u, y, x));
    Ms[idx] = val;
  } else if (idx < ns * ns + nd * nd) {
    int k = idx - ns * ns;
    int s = k / nd, t = k % nd, u, v, x, y;
    aa_anti_pair(s, na, &u, &v);
    aa_anti_pair(t, na, &x, &y);
    Ma[k] = 0.5 * (G2(u, v, x, y) - G2(u, v, y, x) - G2(v, u, x, y) + G2(v, u, y, x));
  }
}

// out[0] += sum of x[0..n) in a fixed order (single block)
__global__ void ordered_sum_kernel(const double* __restrict__ x, long n, double* out, int accumulate) {
  __shared__ double red[256];
  double s = 0.0;
  for (long i = threadIdx.x; i < n; i += 256) s += x[i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[0] = (accumulate ? out[0] : 0.0) + red[0];
}

}  // namespace

int dress_f64(const Geometry& g, const DressDesc* d_desc, int ndesc, const DressAux& aux, const double* tau,
              const double* kap, double* sig, double* sig_sign, double* e_part, bool want_sig,
              cudaStream_t st) {
  if (ndesc <= 0) return DSRG_FNO_OK;
  const int ntd = ceil_div(g.nv, DT);
  dim3 grid(ntd * ntd, ndesc);
  dress_kernel<<<grid, DNT, 0, st>>>(g.nv, g.na, d_desc, aux, tau, kap, sig, sig_sign, e_part,
                                     want_sig ? 1 : 0);
  DSRG_LAUNCH_CHECK();
  return DSRG_FNO_OK;
}

int aa_blocks(int na, const double* g1, const double* lam2, double* Ms, double* Ma, cudaStream_t st) {
  const int ns = na * (na + 1) / 2, nd = na * (na - 1) / 2;
  const int tot = ns * ns + nd * nd;
  if (tot == 0) return DSRG_FNO_OK;
  aa_blocks_kernel<<<ceil_div(tot, 128), 128, 0, st>>>(na, g1, lam2, Ms, Ma);
  DSRG_LAUNCH_CHECK();
  return DSRG_FNO_OK;
}

int ordered_sum(const double* x, long n, double* out, bool accumulate, cudaStream_t st) {
  ordered_sum_kernel<<<1, 256, 0, st>>>(x, n, out, accumulate ? 1 : 0);
  DSRG_LAUNCH_CHECK();
  return DSRG_FNO_OK;
}

}  // namespace dsrg
