// Truncation of the natural orbitals (Eqs. 9, 10 and the near-degeneracy
// widening of Sec. 2) and small helpers of the discarded-orbital correction.
#include "kernels.h"

namespace dsrg {

namespace {

// Single-thread decision, identical arithmetic order on every call.
//   mode 0: smallest N' with sum_{p<=N'} n_p >= (thr/100) sum_all n_p   (Eq. 10)
//   mode 1: N' = ceil(thr/100 * nv)                                       (Eq. 9)
//   mode 2: number of n_p >= thr                                          (n_kappa)
// then while N' < nv and n_{N'} - n_{N'+1} < ratio * max(n_{N'}, n_{N'+1}): N'++.
__global__ void truncate_kernel(int nv, const double* __restrict__ ons, int mode, double thr, double ratio,
                                int* nkept) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  int k = nv;
  if (mode == 0) {
    double tot = 0.0;
    for (int p = 0; p < nv; ++p) tot += ons[p];
    const double target = thr / 100.0 * tot;
    double cum = 0.0;
    for (int p = 0; p < nv; ++p) {
      cum += ons[p];
      if (cum >= target) {
        k = p + 1;
        break;
      }
    }
  } else if (mode == 1) {
    k = (int)ceil(thr / 100.0 * nv - 1e-12);
  } else if (mode == 3) {
    k = (int)rint(fmin(fmax(thr, 0.0), (double)nv));
  } else {
    k = 0;
    for (int p = 0; p < nv; ++p) k += (ons[p] >= thr) ? 1 : 0;
  }
  k = k < 0 ? 0 : (k > nv ? nv : k);
  while (k > 0 && k < nv && (ons[k - 1] - ons[k]) < ratio * fmax(ons[k - 1], ons[k])) ++k;
  *nkept = k;
}

__global__ void symmetrize_kernel(int n, double* D) {
  long idx = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (idx >= (long)n * n) return;
  int e = (int)(idx / n), f = (int)(idx % n);
  if (e >= f) return;
  double a = D[(long)e * n + f], b = D[(long)f * n + e];
  double s = 0.5 * (a + b);
  D[(long)e * n + f] = s;
  D[(long)f * n + e] = s;
}

// W[e][l] = eps_v[e] * V[e][l]  (first ncol columns, leading dimension ld)
__global__ void scale_rows_kernel(int nv, int ncol, long ld, const double* __restrict__ ev,
                                  const double* __restrict__ V, double* __restrict__ W) {
  long idx = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (idx >= (long)nv * ncol) return;
  int e = (int)(idx / ncol), l = (int)(idx % ncol);
  W[(long)e * ncol + l] = ev[e] * V[(long)e * ld + l];
}

// Bf[Q][h][x] = B[Q][h][x] for the active particle columns
__global__ void copy_active_kernel(long rows, int na, int np, int npf, const double* __restrict__ B,
                                   double* __restrict__ Bf) {
  long idx = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (idx >= rows * na) return;
  long r = idx / na;
  int x = (int)(idx % na);
  Bf[r * npf + x] = B[r * np + x];
}

__global__ void finite_kernel(const double* __restrict__ x, long n, int* flag) {
  long idx = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (idx < n && !isfinite(x[idx])) atomicExch(flag, 1);
}

}  // namespace

int truncate_ons(int nv, const double* ons, int mode, double thr, double ratio, int* nkept, cudaStream_t st) {
  truncate_kernel<<<1, 32, 0, st>>>(nv, ons, mode, thr, ratio, nkept);
  DSRG_LAUNCH_CHECK();
  return DSRG_FNO_OK;
}

int symmetrize(int n, double* D, cudaStream_t st) {
  long n2 = (long)n * n;
  if (n2 == 0) return DSRG_FNO_OK;
  symmetrize_kernel<<<ceil_div(n2, 256), 256, 0, st>>>(n, D);
  DSRG_LAUNCH_CHECK();
  return DSRG_FNO_OK;
}

int scale_rows(int nv, int ncol, long ld, const double* ev, const double* V, double* W, cudaStream_t st) {
  long n = (long)nv * ncol;
  if (n == 0) return DSRG_FNO_OK;
  scale_rows_kernel<<<ceil_div(n, 256), 256, 0, st>>>(nv, ncol, ld, ev, V, W);
  DSRG_LAUNCH_CHECK();
  return DSRG_FNO_OK;
}

int copy_active(long rows, int na, int np, int npf, const double* B, double* Bf, cudaStream_t st) {
  long n = rows * na;
  if (n == 0) return DSRG_FNO_OK;
  copy_active_kernel<<<ceil_div(n, 256), 256, 0, st>>>(rows, na, np, npf, B, Bf);
  DSRG_LAUNCH_CHECK();
  return DSRG_FNO_OK;
}

int check_finite(const double* x, long n, int* flag, cudaStream_t st) {
  if (n <= 0) return DSRG_FNO_OK;
  finite_kernel<<<ceil_div(n, 256), 256, 0, st>>>(x, n, flag);
  DSRG_LAUNCH_CHECK();
  return DSRG_FNO_OK;
}

}  // namespace dsrg
