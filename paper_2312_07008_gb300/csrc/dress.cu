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
// (A work item forms up to DRESS_OC outputs of one group in one pass.)
// Core-active: G = [[2,-1],[-1,2]] (x) Gamma1 -> lambda g_k (sym), 3 g_k (antisym).
// Active:      eigen-decomposition of the aa block of G (computed on device).
#include "kernels.h"
#include "dress_common.cuh"

namespace dsrg {

namespace {
using namespace dressc;

// One pass over the upper tiles of a group: every slot tile is read once and
// all outputs of the work item are formed in registers.  Dressed matrices are
// symmetric or antisymmetric, so the (F, E) tile of Sig is the signed
// transpose of the (E, F) tile; the energy of an off-diagonal tile counts
// twice.
template <int OCT>
__global__ void __launch_bounds__(GNT) dress_kernel(int nv, int na, const DressDesc* __restrict__ desc,
                                                    DressAux aux, const double* __restrict__ tau,
                                                    const double* __restrict__ kap,
                                                    double* __restrict__ sig, double* __restrict__ sig_sign,
                                                    double* __restrict__ e_part, int want_sig) {
  constexpr int NS = (OCT == 2) ? 1 : MAXSLOT;  // core-core groups have one slot
  __shared__ double cd[NS][OCT];
  __shared__ double lam[OCT], sgn[OCT], dg[NS];
  __shared__ double tT[GT][GT + 1], tK[GT][GT + 1], sA[GT][GT + 1];
  __shared__ double red[GNT / 32];
  const DressDesc D = desc[blockIdx.y];
  group_coefficients<OCT>(D, aux, na, cd, lam, sgn, dg);
  const int oc = D.o_count;
  const int ntd = (nv + GT - 1) / GT;
  const int nup = ntd * (ntd + 1) / 2;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const long nv2 = (long)nv * nv;
  double part = 0.0;
  for (int t = blockIdx.x; t < nup; t += gridDim.x) {
    int rem = t, te = 0;
    while (rem >= ntd - te) {
      rem -= ntd - te;
      ++te;
    }
    const int tf = te + rem;
    const int E0 = te * GT, F0 = tf * GT;
    const int e = E0 + ty, f = F0 + tx;
    const bool inside = e < nv && f < nv;
    const double w = (te == tf) ? 1.0 : 2.0;
    double at[OCT], ak[OCT];
#pragma unroll
    for (int o = 0; o < OCT; ++o) {
      at[o] = 0.0;
      ak[o] = 0.0;
    }
    for (int u = 0; u < D.nslots; ++u) {
      const double* T = tau + (long)(D.slot + u) * nv2;
      const double* K = kap + (long)(D.slot + u) * nv2;
      {
        // transposed tile: tT[fl][el] = T[F0 + fl][E0 + el]
        const int fr = F0 + ty, ec = E0 + tx;
        const bool ok = fr < nv && ec < nv;
        tT[ty][tx] = ok ? T[(long)fr * nv + ec] : 0.0;
        tK[ty][tx] = ok ? K[(long)fr * nv + ec] : 0.0;
      }
      __syncthreads();
      const double a = inside ? T[(long)e * nv + f] : 0.0;
      const double b = inside ? K[(long)e * nv + f] : 0.0;
      const double att = tT[tx][ty], btt = tK[tx][ty];
      const double du = dg[u];
#pragma unroll
      for (int o = 0; o < OCT; ++o) {
        if (o < oc) {
          const double c = cd[u][o];
          const double c2 = c * sgn[o] * du;
          at[o] = fma(c, a, fma(c2, att, at[o]));
          ak[o] = fma(c, b, fma(c2, btt, ak[o]));
        }
      }
      __syncthreads();
    }
#pragma unroll
    for (int o = 0; o < OCT; ++o) {
      if (o < oc) {
        const double l = lam[o];
        if (inside) part = fma(0.5 * l * w * at[o], ak[o], part);
        if (want_sig) {
          const double v = sqrt(fabs(l)) * at[o];
          double* S = sig + (long)(D.out + D.o_begin + o) * nv2;
          if (inside) S[(long)e * nv + f] = v;
          if (te != tf) {
            sA[ty][tx] = v;
            __syncthreads();
            const int fr = F0 + ty, ec = E0 + tx;  // S[f][e] = sgn S[e][f]
            if (fr < nv && ec < nv) S[(long)fr * nv + ec] = sgn[o] * sA[tx][ty];
            __syncthreads();
          }
        }
      }
    }
  }
  for (int o = 16; o > 0; o >>= 1) part += __shfl_down_sync(0xffffffffu, part, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = part;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int wv = 0; wv < GNT / 32; ++wv) s += red[wv];
    e_part[(long)blockIdx.y * gridDim.x + blockIdx.x] = s;
  }
  if (want_sig && blockIdx.x == 0 && threadIdx.x < oc)
    sig_sign[D.out + D.o_begin + threadIdx.x] = (lam[threadIdx.x] >= 0.0) ? 1.0 : -1.0;
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

// Work items [0, ncc) are core-core groups (at most two outputs, one slot).
int dress_f64(const Geometry& g, const DressDesc* d_desc, int ndesc, int ncc, const DressAux& aux,
              const double* tau, const double* kap, double* sig, double* sig_sign, double* e_part, bool want_sig,
              cudaStream_t st) {
  if (ncc > 0) {
    dim3 grid(DRESS_TILE_BLOCKS, ncc);
    dress_kernel<2><<<grid, GNT, 0, st>>>(g.nv, g.na, d_desc, aux, tau, kap, sig, sig_sign, e_part,
                                          want_sig ? 1 : 0);
    DSRG_LAUNCH_CHECK();
  }
  if (ndesc > ncc) {
    dim3 grid(DRESS_TILE_BLOCKS, ndesc - ncc);
    dress_kernel<DRESS_OC><<<grid, GNT, 0, st>>>(g.nv, g.na, d_desc + ncc, aux, tau, kap, sig, sig_sign,
                                                 e_part + (long)ncc * DRESS_TILE_BLOCKS, want_sig ? 1 : 0);
    DSRG_LAUNCH_CHECK();
  }
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
