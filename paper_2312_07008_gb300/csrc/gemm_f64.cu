// Float64 contractions on the CUDA cores: generic batched GEMM, the pair
// contraction with the Eq. A7 epilogue, and the dressed symmetric rank-K
// update that accumulates the vv classes of D_vv.
//
// GB300 runs float64 at a small fraction of its float32 rate, so these
// kernels are float64-pipe bound by construction; they are the plain form
// the sliced tensor-core form is measured against.
#include "kernels.h"

namespace dsrg {

namespace {

constexpr int TM = 64, TN = 64, TK = 16, NT = 256;

template <bool A_KC>
__device__ __forceinline__ void load_a_tile(double (*As)[TM + 1], const double* A, long lda, int m0,
                                            int k0, int M, int K) {
  // 64 x 16 elements, 4 per thread
#pragma unroll
  for (int it = 0; it < (TM * TK) / NT; ++it) {
    int idx = threadIdx.x + it * NT;
    int m, k;
    if (A_KC) {
      k = idx % TK;
      m = idx / TK;
    } else {
      m = idx % TM;
      k = idx / TM;
    }
    int gm = m0 + m, gk = k0 + k;
    double v = 0.0;
    if (gm < M && gk < K) v = A_KC ? A[(long)gm * lda + gk] : A[(long)gk * lda + gm];
    As[k][m] = v;
  }
}

template <bool B_KC>
__device__ __forceinline__ void load_b_tile(double (*Bs)[TN + 1], const double* B, long ldb, int n0,
                                            int k0, int N, int K) {
#pragma unroll
  for (int it = 0; it < (TN * TK) / NT; ++it) {
    int idx = threadIdx.x + it * NT;
    int n, k;
    if (B_KC) {
      k = idx % TK;
      n = idx / TK;
    } else {
      n = idx % TN;
      k = idx / TN;
    }
    int gn = n0 + n, gk = k0 + k;
    double v = 0.0;
    if (gn < N && gk < K) v = B_KC ? B[(long)gn * ldb + gk] : B[(long)gk * ldb + gn];
    Bs[k][n] = v;
  }
}

__device__ __forceinline__ void mma_tile(const double (*As)[TM + 1], const double (*Bs)[TN + 1],
                                         double acc[4][4]) {
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
#pragma unroll
  for (int k = 0; k < TK; ++k) {
    double a[4], b[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) a[i] = As[k][ty + 16 * i];
#pragma unroll
    for (int j = 0; j < 4; ++j) b[j] = Bs[k][tx + 16 * j];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
  }
}

template <bool A_KC, bool B_KC>
__global__ void __launch_bounds__(NT) gemm_f64_kernel(int M, int N, int K, double alpha,
                                                      const double* __restrict__ A, long lda,
                                                      const double* __restrict__ B, long ldb,
                                                      double beta, double* C, long ldc, long sa,
                                                      long sb, long sc) {
  __shared__ double As[TK][TM + 1];
  __shared__ double Bs[TK][TN + 1];
  A += sa * blockIdx.z;
  B += sb * blockIdx.z;
  C += sc * blockIdx.z;
  const int m0 = blockIdx.y * TM, n0 = blockIdx.x * TN;
  double acc[4][4] = {};
  for (int k0 = 0; k0 < K; k0 += TK) {
    load_a_tile<A_KC>(As, A, lda, m0, k0, M, K);
    load_b_tile<B_KC>(Bs, B, ldb, n0, k0, N, K);
    __syncthreads();
    mma_tile(As, Bs, acc);
    __syncthreads();
  }
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    int m = m0 + ty + 16 * i;
    if (m >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int n = n0 + tx + 16 * j;
      if (n >= N) continue;
      double* c = C + (long)m * ldc + n;
      *c = alpha * acc[i][j] + (beta == 0.0 ? 0.0 : beta * *c);
    }
  }
}

// ---------------------------------------------------------------------------
// Pair contraction with the regulariser epilogue.
// Rows a and columns b run over the particles (active first).  The operands
// are B[:, i, :] and B[:, j, :], each [naux][np] with row stride nh*np.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(NT) pair_gemm_f64_kernel(Geometry g, const double* __restrict__ B,
                                                           const double* __restrict__ eps,
                                                           const int2* __restrict__ pairs,
                                                           double* __restrict__ tau,
                                                           double* __restrict__ kap,
                                                           double* __restrict__ ts) {
  __shared__ double As[TK][TM + 1];
  __shared__ double Bs[TK][TN + 1];
  const int slot = blockIdx.z;
  const int2 pr = pairs[slot];
  const int i = pr.x, j = pr.y;
  const int m0 = blockIdx.y * TM, n0 = blockIdx.x * TN;
  const int na = g.na, nv = g.nv, np = g.np;
  // tiles entirely inside the active x active block carry no needed element
  if (m0 + TM <= na && n0 + TN <= na) return;
  // energy-only passes need only the vv block
  if (ts == nullptr && (m0 + TM <= na || n0 + TN <= na)) return;
  const long ld = (long)g.nh * np;
  const double* Ai = B + (long)i * np;
  const double* Bj = B + (long)j * np;
  double acc[4][4] = {};
  for (int k0 = 0; k0 < g.nq; k0 += TK) {
    load_a_tile<false>(As, Ai, ld, m0, k0, np, g.nq);
    load_b_tile<false>(Bs, Bj, ld, n0, k0, np, g.nq);
    __syncthreads();
    mma_tile(As, Bs, acc);
    __syncthreads();
  }
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const double ei_ej = eps[i] + eps[j];
  const double* ep = eps + g.nc;  // particle energies, active first
  const long pair_off = (long)slot * nv * nv;
#pragma unroll
  for (int ii = 0; ii < 4; ++ii) {
    const int a = m0 + ty + 16 * ii;
    if (a >= np) continue;
    const bool a_vir = a >= na;
#pragma unroll
    for (int jj = 0; jj < 4; ++jj) {
      const int b = n0 + tx + 16 * jj;
      if (b >= np) continue;
      const bool b_vir = b >= na;
      if (!a_vir && !b_vir) continue;
      const double nu = acc[ii][jj];
      const double delta = ei_ej - ep[a] - ep[b];
      const double r1 = regularizer(delta, g.s);
      const double t = nu * r1;
      if (a_vir && b_vir) {
        const long o = pair_off + (long)(a - na) * nv + (b - na);
        tau[o] = t;
        kap[o] = 2.0 * nu - delta * t;
      } else if (ts != nullptr) {
        if (a_vir) {  // t^{ij}_{ex}, e = a - na, x = b
          ts[(((long)i * g.nh + j) * nv + (a - na)) * na + b] = t;
        } else if (i != j) {  // t^{ij}_{xe} = t^{ji}_{ex}
          ts[(((long)j * g.nh + i) * nv + (b - na)) * na + a] = t;
        }
      }
    }
  }
}

// ---------------------------------------------------------------------------
// D(upper 64x64 tiles) partial sums over a split of the dressed matrices:
//   dpart[split][e][f] = sum_{r in split} sign_r sum_e' Sig[r][e][e'] Sig[r][f][e']
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(NT) syrk_dressed_kernel(int nv, int nr, const double* __restrict__ sig,
                                                          const double* __restrict__ sig_sign,
                                                          int nt, int nsplit, double* __restrict__ dpart) {
  __shared__ double As[TK][TM + 1];
  __shared__ double Bs[TK][TN + 1];
  // blockIdx.x enumerates the upper tiles (a <= b) row by row
  int rem = blockIdx.x, ta = 0;
  while (rem >= nt - ta) {
    rem -= nt - ta;
    ++ta;
  }
  const int m0 = ta * TM, n0 = (ta + rem) * TN;
  const int split = blockIdx.y;
  const int r_begin = (int)((long)nr * split / nsplit), r_end = (int)((long)nr * (split + 1) / nsplit);
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  double acc[4][4] = {};
  for (int r = r_begin; r < r_end; ++r) {
    const double* S = sig + (long)r * nv * nv;
    const double sg = sig_sign[r];
    double part[4][4] = {};
    for (int k0 = 0; k0 < nv; k0 += TK) {
      load_a_tile<true>(As, S, nv, m0, k0, nv, nv);
      load_b_tile<true>(Bs, S, nv, n0, k0, nv, nv);
      __syncthreads();
      mma_tile(As, Bs, part);
      __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = fma(sg, part[i][j], acc[i][j]);
  }
  double* Dp = dpart + (long)split * nv * nv;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    int m = m0 + ty + 16 * i;
    if (m >= nv) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int n = n0 + tx + 16 * j;
      if (n >= nv) continue;
      Dp[(long)m * nv + n] = acc[i][j];
    }
  }
}

// D[e][f] += sum_split dpart (upper tiles), mirrored to the lower triangle.
__global__ void syrk_reduce_kernel(int nv, int nsplit, const double* __restrict__ dpart, double* D) {
  long idx = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (idx >= (long)nv * nv) return;
  int e = (int)(idx / nv), f = (int)(idx % nv);
  // the element lives in an upper tile iff tile(e) <= tile(f)
  int te = e / TM, tf = f / TN;
  long src;
  if (te <= tf) src = (long)e * nv + f;
  else src = (long)f * nv + e;
  double s = 0.0;
  for (int k = 0; k < nsplit; ++k) s += dpart[(long)k * nv * nv + src];
  D[idx] += s;
}

}  // namespace

int gemm_f64(int M, int N, int K, double alpha, const double* A, long lda, bool a_kcontig,
             const double* B, long ldb, bool b_kcontig, double beta, double* C, long ldc, int batch,
             long sa, long sb, long sc, cudaStream_t st) {
  if (M <= 0 || N <= 0 || batch <= 0) return DSRG_FNO_OK;
  dim3 grid(ceil_div(N, TN), ceil_div(M, TM), batch);
  if (a_kcontig && b_kcontig)
    gemm_f64_kernel<true, true><<<grid, NT, 0, st>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, sa, sb, sc);
  else if (a_kcontig && !b_kcontig)
    gemm_f64_kernel<true, false><<<grid, NT, 0, st>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, sa, sb, sc);
  else if (!a_kcontig && b_kcontig)
    gemm_f64_kernel<false, true><<<grid, NT, 0, st>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, sa, sb, sc);
  else
    gemm_f64_kernel<false, false><<<grid, NT, 0, st>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, sa, sb, sc);
  DSRG_LAUNCH_CHECK();
  return DSRG_FNO_OK;
}

int pair_gemm_f64(const Geometry& g, const double* B, const double* eps, const int2* pairs, int npairs,
                  double* tau, double* kap, double* ts, cudaStream_t st) {
  if (npairs <= 0) return DSRG_FNO_OK;
  dim3 grid(ceil_div(g.np, TN), ceil_div(g.np, TM), npairs);
  void* tok = nullptr;
  if (profiling()) prof_begin("pair_gemm_f64", 2.0 * g.np * (double)g.np * g.nq * npairs, st, &tok);
  pair_gemm_f64_kernel<<<grid, NT, 0, st>>>(g, B, eps, pairs, tau, kap, ts);
  DSRG_LAUNCH_CHECK();
  prof_end(tok, st);
  return DSRG_FNO_OK;
}

int syrk_dressed_f64(int nv, int nr, const double* sig, const double* sig_sign, double* dpart, int nsplit,
                     double* D, cudaStream_t st) {
  if (nr <= 0 || nv <= 0) return DSRG_FNO_OK;
  const int nt = ceil_div(nv, TM);
  dim3 grid((unsigned)(nt * (nt + 1) / 2), nsplit);
  syrk_dressed_kernel<<<grid, NT, 0, st>>>(nv, nr, sig, sig_sign, nt, nsplit, dpart);
  DSRG_LAUNCH_CHECK();
  long n2 = (long)nv * nv;
  syrk_reduce_kernel<<<ceil_div(n2, 256), 256, 0, st>>>(nv, nsplit, dpart, D);
  DSRG_LAUNCH_CHECK();
  return DSRG_FNO_OK;
}

}  // namespace dsrg
