// Elementwise stages of the fast form in double-float arithmetic:
//   - the Eq. A7 regulariser applied to the contraction tiles (tau, kappa),
//     regularizer.cuh,
//   - the 2-RDM dressing of the vv classes with the energy partials.
// Their float64 counterparts are gemm_f64.cu (fused epilogue) and dress.cu.
#include "dd.cuh"
#include "regularizer.cuh"
#include "dress_common.cuh"
#include "kernels.h"

namespace dsrg {

namespace {

using namespace dressc;

// Filled once per device (float64 exp2 / expm1, then split); kernels copy it
// to shared memory.
__device__ RegTables g_reg;

__global__ void reg_tables_fill_kernel() {
  for (int j = threadIdx.x; j < 64; j += blockDim.x) {
    g_reg.T[j] = dd_from_double(exp2(-j / 64.0));
    g_reg.C[j] = dd_from_double(-expm1(-j * 0.69314718055994530942 / 64.0));
  }
  if (threadIdx.x == 0) {
    g_reg.log2e = dd_from_double(1.44269504088896340736);
    g_reg.ln2 = dd_from_double(0.69314718055994530942);
    g_reg.sixth = dd_from_double(1.0 / 6.0);
  }
}

__device__ __forceinline__ void reg_tables_load(RegTables& R) {
  const float* src = reinterpret_cast<const float*>(&g_reg);
  float* dst = reinterpret_cast<float*>(&R);
  for (int k = threadIdx.x; k < (int)(sizeof(RegTables) / sizeof(float)); k += blockDim.x) dst[k] = src[k];
}

__global__ void eps_dd_kernel(int n, const double* __restrict__ eps, float2* __restrict__ out) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n) {
    const dd v = dd_from_double(eps[k]);
    out[k] = make_float2(v.hi, v.lo);
  }
}

constexpr int EPI_ROWS = 8;  // rows a of one pair per block

// tau / kappa (vv, double-float) and t^{ij}_{ex} (va / av, float64) from the
// double-float contraction tiles nu[slot][a][b].  One block per EPI_ROWS rows
// of one pair.
__global__ void __launch_bounds__(256) pair_epilogue_dd_kernel(Geometry g, const double* __restrict__ eps,
                                                               const float2* __restrict__ eps_dd,
                                                               const int2* __restrict__ pairs,
                                                               const float2* __restrict__ nu,
                                                               float2* __restrict__ tau, float2* __restrict__ kap,
                                                               double* __restrict__ ts) {
  __shared__ RegTables R;
  __shared__ float2 s_ca[EPI_ROWS];
  reg_tables_load(R);
  const int a0 = blockIdx.x * EPI_ROWS, slot = blockIdx.y;
  const int na = g.na, nv = g.nv, np = g.np;
  const int2 pr = pairs[slot];
  const int i = pr.x, j = pr.y;
  const double* ep = eps + g.nc;
  // Delta = (eps_i + eps_j - eps_a) - eps_b, the row part rounded once to double-float
  if (threadIdx.x < EPI_ROWS && a0 + threadIdx.x < np) {
    const dd ca = dd_from_double(eps[i] + eps[j] - ep[a0 + threadIdx.x]);
    s_ca[threadIdx.x] = make_float2(ca.hi, ca.lo);
  }
  __syncthreads();
  const dd s = dd_from_double(g.s);
  const int rows = min(EPI_ROWS, np - a0);
  for (int ra = 0; ra < rows; ++ra)
  for (int b = threadIdx.x; b < np; b += blockDim.x) {
    const int a = a0 + ra;
    const bool av = a >= na, bv = b >= na;
    if (!av && !bv) continue;
    if (ts == nullptr && !(av && bv)) continue;
    const float2 nn = nu[((long)slot * np + a) * np + b];
    const dd n = {nn.x, nn.y};
    const float2 eb = eps_dd[g.nc + b];
    const float2 ca2 = s_ca[a - a0];
    const dd delta = dd_sub(dd{ca2.x, ca2.y}, dd{eb.x, eb.y});
    dd r1, y;
    regularize(delta, s, R, &r1, &y);
    const dd t = dd_mul(n, r1);
    if (av && bv) {
      const dd k = dd_mul(n, dd_add_f(y, 1.0f));
      const long o = ((long)slot * nv + (a - na)) * nv + (b - na);
      tau[o] = make_float2(t.hi, t.lo);
      kap[o] = make_float2(k.hi, k.lo);
    } else if (av) {
      ts[(((long)i * g.nh + j) * nv + (a - na)) * na + b] = dd_to_double(t);
    } else if (i != j) {
      ts[(((long)j * g.nh + i) * nv + (b - na)) * na + a] = dd_to_double(t);
    }
  }
}

__device__ __forceinline__ dd ld(const float2* p, long i) {
  const float2 v = p[i];
  return {v.x, v.y};
}

// acc + c s: the product's high part is added error-free (TwoSum), its low
// parts and the accumulator's low word in float32; one renormalisation.
__device__ __forceinline__ dd dd_fma_acc(dd acc, dd c, dd s) {
  const dd p = two_prod(c.hi, s.hi);
  const float e = __fmaf_rn(c.hi, s.lo, __fmaf_rn(c.lo, s.hi, p.lo));
  dd t = two_sum(acc.hi, p.hi);
  t.lo = __fadd_rn(t.lo, __fadd_rn(acc.lo, e));
  return quick_two_sum(t.hi, t.lo);
}

// Double-float form of the group dressing (same structure as dress.cu).
template <int OCT>
__global__ void __launch_bounds__(GNT, (OCT == 2) ? 4 : 3)
    dress_dd_kernel(int nv, int na, const DressDesc* __restrict__ desc, DressAux aux,
                    const float2* __restrict__ tau, const float2* __restrict__ kap, float2* __restrict__ sig,
                    double* __restrict__ sig_sign, double* __restrict__ e_part, int want_sig,
                    unsigned* __restrict__ rowmax) {
  static_assert(OCT % 2 == 0, "coefficients are read two outputs at a time");
  constexpr int NS = (OCT == 2) ? 1 : MAXSLOT;
  // float64 coefficients, converted in place to double-float (same size)
  __shared__ __align__(16) union {
    double d[NS][OCT];
    dd f[NS][OCT];
  } cf;
  __shared__ double lam[OCT], sgn[OCT], dg[NS];
  __shared__ dd lamw[OCT], sqd[OCT];
  __shared__ float sgnf[OCT], dgf[NS];  // float copies: no float64 op in the loops
  // transposed tiles double-buffered: one barrier per slot
  __shared__ float2 tT[2][GT][GT + 1], tK[2][GT][GT + 1], sA[GT][GT + 1];
  __shared__ double red[GNT / 32];
  const DressDesc D = desc[blockIdx.y];
  group_coefficients<OCT>(D, aux, na, cf.d, lam, sgn, dg);
  const int oc = D.o_count;
  for (int idx = threadIdx.x; idx < D.nslots * OCT; idx += blockDim.x) {
    const int u = idx / OCT, o = idx % OCT;
    const double v = cf.d[u][o];
    cf.f[u][o] = dd_from_double(v);
  }
  for (int o = threadIdx.x; o < oc; o += blockDim.x) {
    lamw[o] = dd_from_double(0.5 * lam[o]);
    sqd[o] = dd_from_double(sqrt(fabs(lam[o])));
    sgnf[o] = sgn[o] > 0.0 ? 1.0f : -1.0f;
  }
  for (int u = threadIdx.x; u < D.nslots; u += blockDim.x) dgf[u] = (float)dg[u];
  __syncthreads();
  const int ntd = (nv + GT - 1) / GT;
  const int nup = ntd * (ntd + 1) / 2;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const long nv2 = (long)nv * nv;
  const int ns = D.nslots;
  unsigned posmask = 0;  // bit o: output o is symmetric (sgn +1)
#pragma unroll
  for (int o = 0; o < OCT; ++o)
    if (o < oc && sgnf[o] > 0.0f) posmask |= 1u << o;
  // upper tile t -> (te, tf), te <= tf; t only grows, so the row search
  // resumes where the last one ended (row_te starts at tile row_base)
  int row_te = 0, row_base = 0;
  auto decode = [&](int t, int* te_, int* tf_) {
    while (t >= row_base + (ntd - row_te)) {
      row_base += ntd - row_te;
      ++row_te;
    }
    *te_ = row_te;
    *tf_ = row_te + (t - row_base);
  };
  // this thread's operands of slot u in tile (te, tf): tau and kappa at (e, f)
  // and at (f, e) (the latter staged transposed through shared memory)
  float2 na_ = make_float2(0.f, 0.f), nb_ = na_, nt_ = na_, nk_ = na_;
  auto fetch = [&](int te, int tf, int u) {
    const float2* T = tau + (long)(D.slot + u) * nv2;
    const float2* K = kap + (long)(D.slot + u) * nv2;
    const int e = te * GT + ty, f = tf * GT + tx;
    const bool in = e < nv && f < nv;
    na_ = in ? T[(long)e * nv + f] : make_float2(0.f, 0.f);
    nb_ = in ? K[(long)e * nv + f] : make_float2(0.f, 0.f);
    const int fr = tf * GT + ty, ec = te * GT + tx;
    const bool ok = fr < nv && ec < nv;
    nt_ = ok ? T[(long)fr * nv + ec] : make_float2(0.f, 0.f);
    nk_ = ok ? K[(long)fr * nv + ec] : make_float2(0.f, 0.f);
  };
  dd part = dd_make(0.0f);
  // OCT = 2 (core pairs): sum_o lambda_o <sigma_o[tau], sigma_o[kappa]> is
  // accumulated per output and weighted once at the end (two outputs' sums
  // fit in registers; with 8 outputs they would lower the occupancy)
  dd eacc[2] = {dd_make(0.0f), dd_make(0.0f)};
  int t = blockIdx.x, te = 0, tf = 0, buf = 0;
  if (t < nup) {
    decode(t, &te, &tf);
    fetch(te, tf, 0);
  }
  while (t < nup) {
    const int tn = t + gridDim.x;
    int ten = 0, tfn = 0;
    if (tn < nup) decode(tn, &ten, &tfn);
    const int E0 = te * GT, F0 = tf * GT;
    const int e = E0 + ty, f = F0 + tx;
    const bool inside = e < nv && f < nv;
    const float w = (te == tf) ? 1.0f : 2.0f;
    dd at[OCT], ak[OCT];
#pragma unroll
    for (int o = 0; o < OCT; ++o) {
      at[o] = dd_make(0.0f);
      ak[o] = dd_make(0.0f);
    }
    for (int u = 0; u < ns; ++u) {
      tT[buf][ty][tx] = nt_;
      tK[buf][ty][tx] = nk_;
      const dd a = {na_.x, na_.y}, b = {nb_.x, nb_.y};
      // the next slot's (or the next tile's first slot's) loads fly during
      // this slot's arithmetic
      if (u + 1 < ns) fetch(te, tf, u + 1);
      else if (tn < nup) fetch(ten, tfn, 0);
      __syncthreads();
      // c T + c sgn dg T^T = c (T + sgn dg T^T) with sgn = +-1, dg in {0, 1}:
      // the two signed combinations are formed once per slot
      const float du = dgf[u];
      const float2 xt = tT[buf][tx][ty], xk = tK[buf][tx][ty];
      const dd att = {du * xt.x, du * xt.y}, btt = {du * xk.x, du * xk.y};
      const dd tp = dd_add_fast(a, att), tm = dd_sub_fast(a, att);
      const dd kp = dd_add_fast(b, btt), km = dd_sub_fast(b, btt);
      // the slot's coefficients, two outputs per 16-byte shared load
      const float4* cu = reinterpret_cast<const float4*>(&cf.f[u][0]);
#pragma unroll
      for (int o2 = 0; o2 < OCT; o2 += 2) {
        if (o2 < oc) {
          const float4 c2 = cu[o2 >> 1];
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int o = o2 + h;
            if (o < oc) {
              const dd c = h ? dd{c2.z, c2.w} : dd{c2.x, c2.y};
              const bool pos = (posmask >> o) & 1u;
              at[o] = dd_fma_acc(at[o], c, pos ? tp : tm);
              ak[o] = dd_fma_acc(ak[o], c, pos ? kp : km);
            }
          }
        }
      }
      buf ^= 1;
    }
#pragma unroll
    for (int o = 0; o < OCT; ++o) {
      if (o < oc) {
        if constexpr (OCT == 2) {
          // w = 1 or 2: the scaling of at is exact
          if (inside) eacc[o] = dd_fma_acc(eacc[o], dd{at[o].hi * w, at[o].lo * w}, ak[o]);
        } else {
          if (inside) part = dd_add(part, dd_mul_f(dd_mul(lamw[o], dd_mul(at[o], ak[o])), w));
        }
        if (want_sig) {
          const dd v = dd_mul(sqd[o], at[o]);
          const long mat = D.out + D.o_begin + o;
          float2* S = sig + mat * nv2;
          if (inside) S[(long)e * nv + f] = make_float2(v.hi, v.lo);
          if (rowmax) {
            // max |hi| of row e over this tile (16 lanes share ty)
            float m = inside ? fabsf(v.hi) : 0.0f;
#pragma unroll
            for (int w = 8; w > 0; w >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, w));
            if (tx == 0 && e < nv) atomicMax(rowmax + mat * nv + e, __float_as_uint(m));
          }
          if (te != tf) {
            sA[ty][tx] = make_float2(v.hi, v.lo);
            __syncthreads();
            const int fr = F0 + ty, ec = E0 + tx;
            const float sg = sgnf[o];
            const bool ok = fr < nv && ec < nv;
            if (ok) S[(long)fr * nv + ec] = make_float2(sg * sA[tx][ty].x, sg * sA[tx][ty].y);
            if (rowmax) {
              float m = ok ? fabsf(sA[tx][ty].x) : 0.0f;
#pragma unroll
              for (int w = 8; w > 0; w >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, w));
              if (tx == 0 && fr < nv) atomicMax(rowmax + mat * nv + fr, __float_as_uint(m));
            }
            __syncthreads();
          }
        }
      }
    }
    t = tn;
    te = ten;
    tf = tfn;
  }
  if constexpr (OCT == 2) {
#pragma unroll
    for (int o = 0; o < 2; ++o)
      if (o < oc) part = dd_add(part, dd_mul(lamw[o], eacc[o]));
  }
  double pd = dd_to_double(part);
  for (int o = 16; o > 0; o >>= 1) pd += __shfl_down_sync(0xffffffffu, pd, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = pd;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int wv = 0; wv < GNT / 32; ++wv) s += red[wv];
    e_part[(long)blockIdx.y * gridDim.x + blockIdx.x] = s;
  }
  if (want_sig && blockIdx.x == 0 && threadIdx.x < oc)
    sig_sign[D.out + D.o_begin + threadIdx.x] = (lam[threadIdx.x] >= 0.0) ? 1.0 : -1.0;
}

// n regulariser values for tests: r1[k] = R1(delta[k]), y[k] = exp(-s delta^2)
__global__ void regularize_test_kernel(int n, const double* delta, double s, double* r1, double* y) {
  __shared__ RegTables R;
  reg_tables_load(R);
  __syncthreads();
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    dd a, b;
    regularize(dd_from_double(delta[k]), dd_from_double(s), R, &a, &b);
    r1[k] = dd_to_double(a);
    y[k] = dd_to_double(b);
  }
}

}  // namespace

int eps_to_dd(int n, const double* eps, float2* out, cudaStream_t st) {
  if (n <= 0) return DSRG_FNO_OK;
  eps_dd_kernel<<<ceil_div(n, 256), 256, 0, st>>>(n, eps, out);
  DSRG_LAUNCH_CHECK();
  return DSRG_FNO_OK;
}

// The regulariser table of the current device, filled on first use.
static int ensure_reg_tables() {
  static std::mutex mu;
  static bool ready[64] = {};
  int dev = 0;
  DSRG_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return DSRG_FNO_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lk(mu);
  if (!ready[dev]) {
    // on a private stream, waited for: later kernels of every stream see it
    cudaStream_t s0;
    DSRG_CUDA(cudaStreamCreateWithFlags(&s0, cudaStreamNonBlocking));
    reg_tables_fill_kernel<<<1, 64, 0, s0>>>();
    DSRG_LAUNCH_CHECK();
    DSRG_CUDA(cudaStreamSynchronize(s0));
    DSRG_CUDA(cudaStreamDestroy(s0));
    ready[dev] = true;
  }
  return DSRG_FNO_OK;
}

// Device address of the current device's regulariser tables (filled first).
int reg_tables_device(const RegTables** out) {
  DSRG_TRY(ensure_reg_tables());
  void* p = nullptr;
  DSRG_CUDA(cudaGetSymbolAddress(&p, g_reg));
  *out = static_cast<const RegTables*>(p);
  return DSRG_FNO_OK;
}

__global__ void hole_particle_dd_kernel(Geometry g, const double* __restrict__ eps, float2* __restrict__ out) {
  const long R = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (R >= (long)g.nh * g.np) return;
  const int i = (int)(R / g.np), a = (int)(R - (long)i * g.np);
  const dd v = dd_from_double(eps[i] - eps[g.nc + a]);
  out[R] = make_float2(v.hi, v.lo);
}

// hp[i np + a] = eps_i - eps_a (hole i, particle a) in double-float: the
// denominator Delta^{ij}_{ab} = hp[i a] + hp[j b] of the fused epilogue.
int hole_particle_dd(const Geometry& g, const double* eps, float2* out, cudaStream_t st) {
  const long n = (long)g.nh * g.np;
  if (n <= 0) return DSRG_FNO_OK;
  hole_particle_dd_kernel<<<ceil_div(n, 256), 256, 0, st>>>(g, eps, out);
  DSRG_LAUNCH_CHECK();
  return DSRG_FNO_OK;
}

int pair_epilogue_dd(const Geometry& g, const double* eps, const float2* eps_dd, const int2* pairs, int npairs,
                     const float2* nu, float2* tau, float2* kap, double* ts, cudaStream_t st) {
  if (npairs <= 0) return DSRG_FNO_OK;
  DSRG_TRY(ensure_reg_tables());
  dim3 grid(ceil_div(g.np, EPI_ROWS), npairs);
  pair_epilogue_dd_kernel<<<grid, 256, 0, st>>>(g, eps, eps_dd, pairs, nu, tau, kap, ts);
  DSRG_LAUNCH_CHECK();
  return DSRG_FNO_OK;
}

int dress_dd(const Geometry& g, const DressDesc* d_desc, int ndesc, int ncc, const DressAux& aux,
             const float2* tau, const float2* kap, float2* sig, double* sig_sign, double* e_part, bool want_sig,
             unsigned* rowmax, cudaStream_t st) {
  if (ncc > 0) {
    dim3 grid(DRESS_TILE_BLOCKS, ncc);
    dress_dd_kernel<2><<<grid, GNT, 0, st>>>(g.nv, g.na, d_desc, aux, tau, kap, sig, sig_sign, e_part,
                                             want_sig ? 1 : 0, rowmax);
    DSRG_LAUNCH_CHECK();
  }
  if (ndesc > ncc) {
    dim3 grid(DRESS_TILE_BLOCKS, ndesc - ncc);
    dress_dd_kernel<DRESS_OC><<<grid, GNT, 0, st>>>(g.nv, g.na, d_desc + ncc, aux, tau, kap, sig, sig_sign,
                                                    e_part + (long)ncc * DRESS_TILE_BLOCKS, want_sig ? 1 : 0,
                                                    rowmax);
    DSRG_LAUNCH_CHECK();
  }
  return DSRG_FNO_OK;
}

int regularize_test(int n, const double* delta, double s, double* r1, double* y, cudaStream_t st) {
  if (n <= 0) return DSRG_FNO_OK;
  DSRG_TRY(ensure_reg_tables());
  regularize_test_kernel<<<ceil_div(n, 256), 256, 0, st>>>(n, delta, s, r1, y);
  DSRG_LAUNCH_CHECK();
  return DSRG_FNO_OK;
}

}  // namespace dsrg
