// Float64 symmetric eigensolver (Eq. 8: Gamma V = n V) and helpers.
//
// Cyclic two-sided Jacobi with round-robin pair ordering: in each round the
// indices form n/2 disjoint pairs, so A' = J^T A J and V' = V J are computed
// out of place in one launch, every output element reading the 2 x 2
// neighbourhood it depends on.  Rotation angles follow the classical
// symmetric Schur decomposition (Golub and Van Loan, "Matrix Computations",
// Sec. 8.5): tau = (a_qq - a_pp) / (2 a_pq), t = sign(tau)/(|tau| +
// sqrt(1 + tau^2)), c = 1/sqrt(1 + t^2), s = t c.  Sweeps repeat until the
// off-diagonal Frobenius norm falls below 1e-15 of the total.
#include "kernels.h"

namespace dsrg {

namespace {

constexpr int ET = 32;   // tile edge of the update kernel
constexpr int ENT = 256; // threads per update block

// partner of index i in round r of the round-robin schedule over m (even) slots
__device__ __forceinline__ int rr_partner(int i, int r, int m) {
  // slot position: index 0 fixed; index k>0 sits at position ((k - 1 - r) mod (m-1)) + 1
  int pos;
  if (i == 0) pos = 0;
  else pos = ((i - 1 - r) % (m - 1) + (m - 1)) % (m - 1) + 1;
  int ppos = m - 1 - pos;  // positions pos and m-1-pos face each other
  if (ppos == 0) return 0;
  return ((ppos - 1 + r) % (m - 1)) + 1;
}

struct Rot {
  int k2;     // partner index (or -1)
  double w1;  // J[i][i]
  double w2;  // J[partner][i]
};

__device__ __forceinline__ Rot make_rot(const double* A, int n, int i, int r, int m) {
  Rot R;
  int q = rr_partner(i, r, m);
  if (q >= n || q == i) {
    R.k2 = -1;
    R.w1 = 1.0;
    R.w2 = 0.0;
    return R;
  }
  int p = min(i, q), qq = max(i, q);
  double apq = A[(long)p * n + qq];
  double c = 1.0, s = 0.0;
  if (apq != 0.0) {
    double app = A[(long)p * n + p], aqq = A[(long)qq * n + qq];
    double tau = (aqq - app) / (2.0 * apq);
    double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
    c = 1.0 / sqrt(1.0 + t * t);
    s = t * c;
  }
  // J = [[c, s], [-s, c]] on (p, q):  J[p][p] = c, J[q][p] = -s, J[p][q] = s, J[q][q] = c
  R.k2 = q;
  R.w1 = c;
  R.w2 = (i == p) ? -s : s;
  return R;
}

// One round: Aout = J^T A J, Vout = V J.  Grid: tiles of A then tiles of V.
__global__ void __launch_bounds__(ENT) jacobi_round_kernel(int n, int m, int r, const double* __restrict__ A,
                                                           double* __restrict__ Aout,
                                                           const double* __restrict__ V,
                                                           double* __restrict__ Vout,
                                                           const int* __restrict__ done) {
  if (*done) return;
  __shared__ Rot rrow[ET], rcol[ET];
  const int nt = (n + ET - 1) / ET;
  int tile = blockIdx.x;
  const bool isV = tile >= nt * nt;
  if (isV) tile -= nt * nt;
  const int i0 = (tile / nt) * ET, j0 = (tile % nt) * ET;
  if (threadIdx.x < ET) {
    int i = i0 + threadIdx.x;
    if (i < n) rrow[threadIdx.x] = make_rot(A, n, i, r, m);
  } else if (threadIdx.x < 2 * ET) {
    int j = j0 + threadIdx.x - ET;
    if (j < n) rcol[threadIdx.x - ET] = make_rot(A, n, j, r, m);
  }
  __syncthreads();
  for (int e = threadIdx.x; e < ET * ET; e += ENT) {
    const int ti = e / ET, tj = e % ET;
    const int i = i0 + ti, j = j0 + tj;
    if (i >= n || j >= n) continue;
    const Rot cj = rcol[tj];
    if (isV) {
      double v = cj.w1 * V[(long)i * n + j];
      if (cj.k2 >= 0) v += cj.w2 * V[(long)i * n + cj.k2];
      Vout[(long)i * n + j] = v;
    } else {
      const Rot ci = rrow[ti];
      // the rotated pair's off-diagonal element is annihilated
      if (ci.k2 == j) {
        Aout[(long)i * n + j] = 0.0;
        continue;
      }
      double a11 = A[(long)i * n + j];
      double v = ci.w1 * cj.w1 * a11;
      if (cj.k2 >= 0) v += ci.w1 * cj.w2 * A[(long)i * n + cj.k2];
      if (ci.k2 >= 0) {
        v += ci.w2 * cj.w1 * A[(long)ci.k2 * n + j];
        if (cj.k2 >= 0) v += ci.w2 * cj.w2 * A[(long)ci.k2 * n + cj.k2];
      }
      Aout[(long)i * n + j] = v;
    }
  }
}

// off-diagonal and total squared norms -> done flag (single block)
__global__ void jacobi_check_kernel(int n, const double* __restrict__ A, int* done, double* norms) {
  __shared__ double s_off[256], s_tot[256];
  double off = 0.0, tot = 0.0;
  for (long idx = threadIdx.x; idx < (long)n * n; idx += blockDim.x) {
    double a = A[idx];
    tot += a * a;
    if (idx / n != idx % n) off += a * a;
  }
  s_off[threadIdx.x] = off;
  s_tot[threadIdx.x] = tot;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      s_off[threadIdx.x] += s_off[threadIdx.x + w];
      s_tot[threadIdx.x] += s_tot[threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    norms[0] = s_off[0];
    norms[1] = s_tot[0];
    // rounding floor of a converged sweep is about (n eps)^2 relative
    const double tol = fmax(1e-30, (2.2e-16 * n) * (2.2e-16 * n));
    if (s_off[0] <= tol * s_tot[0] || s_tot[0] == 0.0) *done = 1;
  }
}

__global__ void identity_kernel(int n, double* V) {
  long idx = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (idx < (long)n * n) V[idx] = (idx / n == idx % n) ? 1.0 : 0.0;
}

// ranks by (value descending | ascending, index ascending)
__global__ void eig_rank_kernel(int n, const double* __restrict__ A, bool descending, int* rank) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  double vj = A[(long)j * n + j];
  int rk = 0;
  for (int k = 0; k < n; ++k) {
    double vk = A[(long)k * n + k];
    bool before = descending ? (vk > vj) : (vk < vj);
    if (before || (vk == vj && k < j)) ++rk;
  }
  rank[j] = rk;
}

// evals[rank[j]] = A[j][j]; evecs[:, rank[j]] = V[:, j] (sign fixed)
__global__ void eig_permute_kernel(int n, const double* __restrict__ A, const double* __restrict__ V,
                                   const int* __restrict__ rank, bool fix_sign, double* evals,
                                   double* evecs) {
  int j = blockIdx.x;  // one block per column
  __shared__ double s_val[256];
  __shared__ int s_idx[256];
  double best = -1.0;
  int bi = 0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    double a = fabs(V[(long)i * n + j]);
    if (a > best) {
      best = a;
      bi = i;
    }
  }
  s_val[threadIdx.x] = best;
  s_idx[threadIdx.x] = bi;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      double o = s_val[threadIdx.x + w];
      int oi = s_idx[threadIdx.x + w];
      if (o > s_val[threadIdx.x] || (o == s_val[threadIdx.x] && oi < s_idx[threadIdx.x])) {
        s_val[threadIdx.x] = o;
        s_idx[threadIdx.x] = oi;
      }
    }
    __syncthreads();
  }
  double sign = 1.0;
  if (fix_sign && V[(long)s_idx[0] * n + j] < 0.0) sign = -1.0;
  const int dst = rank[j];
  for (int i = threadIdx.x; i < n; i += blockDim.x) evecs[(long)i * n + dst] = sign * V[(long)i * n + j];
  if (threadIdx.x == 0) evals[dst] = A[(long)j * n + j];
}

}  // namespace

// A (n x n, symmetric) is destroyed: on return its diagonal holds the
// eigenvalues; V (n x n) receives the eigenvectors (column j <-> A[j][j]).
// work: 2 n^2 + 8 doubles.  status_dev: one int of device memory.
int eig_sym_jacobi(int n, double* A, double* V, double* work, int* status_dev, int max_sweeps,
                   cudaStream_t st) {
  if (n <= 0) return DSRG_FNO_OK;
  double* A2 = work;
  double* V2 = work + (long)n * n;
  double* norms = work + 2L * n * n;
  long n2 = (long)n * n;
  identity_kernel<<<ceil_div(n2, 256), 256, 0, st>>>(n, V);
  DSRG_LAUNCH_CHECK();
  DSRG_CUDA(cudaMemsetAsync(status_dev, 0, sizeof(int), st));
  if (n == 1) return DSRG_FNO_OK;
  const int m = (n % 2 == 0) ? n : n + 1;
  const int nt = ceil_div(n, ET);
  double* a = A;
  double* a2 = A2;
  double* v = V;
  double* v2 = V2;
  int converged = 0;
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    jacobi_check_kernel<<<1, 256, 0, st>>>(n, a, status_dev, norms);
    DSRG_LAUNCH_CHECK();
    DSRG_CUDA(cudaMemcpyAsync(&converged, status_dev, sizeof(int), cudaMemcpyDeviceToHost, st));
    DSRG_CUDA(cudaStreamSynchronize(st));
    if (converged) break;
    for (int r = 0; r < m - 1; ++r) {
      jacobi_round_kernel<<<2 * nt * nt, ENT, 0, st>>>(n, m, r, a, a2, v, v2, status_dev);
      DSRG_LAUNCH_CHECK();
      std::swap(a, a2);
      std::swap(v, v2);
    }
  }
  if (!converged) {
    jacobi_check_kernel<<<1, 256, 0, st>>>(n, a, status_dev, norms);
    DSRG_CUDA(cudaMemcpyAsync(&converged, status_dev, sizeof(int), cudaMemcpyDeviceToHost, st));
    DSRG_CUDA(cudaStreamSynchronize(st));
  }
  if (a != A) {
    DSRG_CUDA(cudaMemcpyAsync(A, a, n2 * sizeof(double), cudaMemcpyDeviceToDevice, st));
    DSRG_CUDA(cudaMemcpyAsync(V, v, n2 * sizeof(double), cudaMemcpyDeviceToDevice, st));
  }
  return converged ? DSRG_FNO_OK : DSRG_FNO_ERR_NOCONV;
}

// evals/evecs sorted (descending or ascending) from the Jacobi output;
// rank: n ints of device scratch.
int eig_sort(int n, const double* A, const double* V, double* evals, double* evecs, int* rank,
             bool descending, bool fix_sign, cudaStream_t st) {
  if (n <= 0) return DSRG_FNO_OK;
  eig_rank_kernel<<<ceil_div(n, 128), 128, 0, st>>>(n, A, descending, rank);
  DSRG_LAUNCH_CHECK();
  eig_permute_kernel<<<n, 256, 0, st>>>(n, A, V, rank, fix_sign, evals, evecs);
  DSRG_LAUNCH_CHECK();
  return DSRG_FNO_OK;
}

}  // namespace dsrg
