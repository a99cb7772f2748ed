// Full multi-reference PT2 energy: the part beyond E_vv (every doubles class
// with an active particle, the singles, and their cumulant couplings); the
// element stages and sums in float64.
//
// Order of the stages (element bodies and the tensor layouts in mr_terms.cuh):
//   1. BA[Q][j][y] = B[Q][j][y] for the active particles y (gather), and the
//      integrals <ay|ij> = sum_Q B[Q][i][a] BA[Q][j][y] as one GEMM (M = nh np
//      rows (i, a), N = nh na columns (j, y), K = naux): in the fast form on
//      the tensor cores from exact bf16 digit planes of both operands (the
//      plain mode of the digit-plane contraction kernel), else float64.
//   2. Eq. A7 amplitudes tp and the vertex xp; Eq. A6 singles t1 and x1.
//   3. The images of T under Theta (particles) and Gamma (holes): z1, tpp,
//      z2, z3, g2t, w3, tt1, gt1.
//   4. sum over the elements of X times their images: fixed-order block sums
//      (grid-stride loop over a fixed grid) and a fixed-order final sum, so
//      the result does not depend on scheduling.
#include "kernels.h"
#include "mr_terms.cuh"

namespace dsrg {

namespace {

constexpr int MR_NT = 256;
constexpr int MR_EBLOCKS = 1216;  // 8 blocks per SM of a 152-SM GB300

#define MR_ELEM_KERNEL(kname, fn)                                 \
  __global__ void kname(MRArgs A, long n) {                       \
    const long i = blockIdx.x * (long)blockDim.x + threadIdx.x;   \
    if (i < n) fn(A, i);                                          \
  }
MR_ELEM_KERNEL(mr_amp_kernel, mr_amp_elem)
MR_ELEM_KERNEL(mr_t1_kernel, mr_t1_elem)
MR_ELEM_KERNEL(mr_z1_kernel, mr_z1_elem)
MR_ELEM_KERNEL(mr_tpp_kernel, mr_tpp_elem)
MR_ELEM_KERNEL(mr_z23_kernel, mr_z23_elem)
MR_ELEM_KERNEL(mr_g2t_kernel, mr_g2t_elem)
MR_ELEM_KERNEL(mr_w3_kernel, mr_w3_elem)
MR_ELEM_KERNEL(mr_t1img_kernel, mr_t1img_elem)
#undef MR_ELEM_KERNEL

// BA[Q][j][y] = B[Q][j][y], y < na
__global__ void mr_gather_active_kernel(long n, int nh, int np, int na, const double* __restrict__ B,
                                        double* __restrict__ BA) {
  const long idx = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (idx >= n) return;
  const int y = (int)(idx % na);
  const long qj = idx / na;  // Q nh + j
  BA[idx] = B[qj * np + y];
}

// partial[b] = sum over the elements b, b + grid, ... of X times its image,
// summed in a fixed order (thread order, then a shared-memory tree).
template <int ONEBODY>
__global__ void __launch_bounds__(MR_NT) mr_energy_kernel(MRArgs A, long n, double* __restrict__ partial) {
  __shared__ double red[MR_NT];
  double s = 0.0;
  const long stride = (long)gridDim.x * blockDim.x;
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < n; idx += stride)
    s += ONEBODY ? mr_energy1_elem(A, idx) : mr_energy_elem(A, idx);
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = MR_NT / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

template <typename F>
int launch_elems(F kernel, const MRArgs& A, long n, cudaStream_t st) {
  if (n <= 0) return DSRG_FNO_OK;
  kernel<<<(unsigned)ceil_div(n, MR_NT), MR_NT, 0, st>>>(A, n);
  DSRG_LAUNCH_CHECK();
  return DSRG_FNO_OK;
}

struct MRSizes {
  long n4, n4a, ng2t, nw3, n1, ngt1, nba;
};

MRSizes mr_sizes(const Geometry& g) {
  MRSizes z;
  z.n4 = (long)g.nh * g.nh * g.np * g.na;
  z.n4a = (long)g.na * g.nh * g.np * g.na;
  z.ng2t = (long)g.nh * g.nh * g.na * g.na;
  z.nw3 = (long)g.nh * g.na * g.na * g.na;
  z.n1 = (long)g.nh * g.np;
  z.ngt1 = (long)g.nh * g.na;
  z.nba = (long)g.nq * g.nh * g.na;
  return z;
}

}  // namespace

// doubles of a buffer, rounded up to 256 bytes so that every carved buffer stays 256-byte aligned
static size_t mr_dbl(size_t bytes) { return (bytes + 255) / 256 * 32; }

static bool mr_tensor_gemm(const Geometry& g, int ks) { return ks > 0 && g.na > 0 && g.nq >= SLICED_MIN_K; }

size_t mr_energy_work_doubles(const Geometry& g, int ks) {
  const MRSizes z = mr_sizes(g);
  // nu (reused for tpp), tp, xp, z1; z2, z3; g2t, w3; t1, x1, tt1; gt1; BA; 2 x partials
  size_t n = 4 * mr_dbl(8 * (size_t)z.n4) + 2 * mr_dbl(8 * (size_t)z.n4a) + mr_dbl(8 * (size_t)z.ng2t) +
             mr_dbl(8 * (size_t)z.nw3) + 3 * mr_dbl(8 * (size_t)z.n1) + mr_dbl(8 * (size_t)z.ngt1) +
             mr_dbl(8 * (size_t)z.nba) + mr_dbl(8 * (2 * (size_t)MR_EBLOCKS + 16));
  if (mr_tensor_gemm(g, ks)) {
    const size_t kp = pad64(g.nq), ra = (size_t)g.nh * g.np, rb = (size_t)g.nh * g.na;
    n += mr_dbl(2 * (size_t)ks * ra * kp) + mr_dbl(2 * (size_t)ks * rb * kp) + mr_dbl(4 * (ra + rb)) + mr_dbl(32);
  }
  return n;
}

int mr_energy_rest(const Geometry& g, int ks, const double* B, const double* eps, const double* f_hp,
                   const double* g1, const double* l2, const double* l3, double* work, double* e_out,
                   cudaStream_t st) {
  *e_out = 0.0;
  if (g.na == 0 && !f_hp) return DSRG_FNO_OK;
  const MRSizes z = mr_sizes(g);
  MRArgs A{};
  A.nc = g.nc;
  A.na = g.na;
  A.nv = g.nv;
  A.nh = g.nh;
  A.np = g.np;
  A.s = g.s;
  A.eps = eps;
  A.f_hp = f_hp;
  A.g1 = g.na ? g1 : nullptr;
  A.l2 = g.na ? l2 : nullptr;
  A.l3 = g.na ? l3 : nullptr;
  double* p = work;
  auto take = [&p](size_t bytes) {
    double* q = p;
    p += mr_dbl(bytes);
    return q;
  };
  double* nu = take(8 * (size_t)z.n4);
  A.tp = take(8 * (size_t)z.n4);
  A.xp = take(8 * (size_t)z.n4);
  A.z1 = take(8 * (size_t)z.n4);
  A.z2 = take(8 * (size_t)z.n4a);
  A.z3 = take(8 * (size_t)z.n4a);
  A.g2t = take(8 * (size_t)z.ng2t);
  A.w3 = take(8 * (size_t)z.nw3);
  A.t1 = take(8 * (size_t)z.n1);
  A.x1 = take(8 * (size_t)z.n1);
  A.tt1 = take(8 * (size_t)z.n1);
  A.gt1 = take(8 * (size_t)z.ngt1);
  double* BA = take(8 * (size_t)z.nba);
  double* partial = take(8 * (2 * (size_t)MR_EBLOCKS + 16));
  double* e_dev = partial + 2 * MR_EBLOCKS;
  A.nu = nu;
  A.tpp = nu;  // nu is consumed by the amplitude stage before tpp is formed

  if (g.na > 0) {
    DSRG_PHASE("phase_mr_integrals", st);
    mr_gather_active_kernel<<<(unsigned)ceil_div(z.nba, MR_NT), MR_NT, 0, st>>>(z.nba, g.nh, g.np, g.na, B, BA);
    DSRG_LAUNCH_CHECK();
    const int M = g.nh * g.np, N = g.nh * g.na;
    if (mr_tensor_gemm(g, ks)) {
      // rows (i, a) of B and (j, y) of BA, contraction over Q: exact digit planes
      const int kp = pad64(g.nq);
      __nv_bfloat16* pa = reinterpret_cast<__nv_bfloat16*>(take(2 * (size_t)ks * M * kp));
      __nv_bfloat16* pb = reinterpret_cast<__nv_bfloat16*>(take(2 * (size_t)ks * N * kp));
      int* ea = reinterpret_cast<int*>(take(4 * (size_t)(M + N)));
      int* eb = ea + M;
      int* err = reinterpret_cast<int*>(take(32));
      DSRG_CUDA(cudaMemsetAsync(err, 0, sizeof(int), st));
      DSRG_TRY(slice_rows(ks, B, M, g.nq, 1, M, kp, pa, ea, st));
      DSRG_TRY(slice_rows(ks, BA, N, g.nq, 1, N, kp, pb, eb, st));
      DSRG_TRY(sliced_plain_gemm(ks, M, N, pa, ea, pb, eb, kp, nu, N, err, st));
      int h = 0;
      DSRG_CUDA(cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, st));
      DSRG_CUDA(cudaStreamSynchronize(st));
      if (h) return DSRG_FNO_ERR_TIMEOUT;
    } else {
      DSRG_TRY(gemm_f64(M, N, g.nq, 1.0, B, M, false, BA, N, false, 0.0, nu, N, 1, 0, 0, 0, st));
    }
  }
  DSRG_PHASE("phase_mr_terms", st);
  DSRG_TRY(launch_elems(mr_amp_kernel, A, z.n4, st));
  DSRG_TRY(launch_elems(mr_t1_kernel, A, z.n1, st));
  DSRG_TRY(launch_elems(mr_z1_kernel, A, z.n4, st));
  DSRG_TRY(launch_elems(mr_tpp_kernel, A, z.n4, st));
  DSRG_TRY(launch_elems(mr_z23_kernel, A, z.n4a, st));
  DSRG_TRY(launch_elems(mr_g2t_kernel, A, z.ng2t, st));
  DSRG_TRY(launch_elems(mr_w3_kernel, A, z.nw3, st));
  DSRG_TRY(launch_elems(mr_t1img_kernel, A, z.n1, st));
  if (z.n4 > 0) {
    mr_energy_kernel<0><<<MR_EBLOCKS, MR_NT, 0, st>>>(A, z.n4, partial);
    DSRG_LAUNCH_CHECK();
  } else {
    DSRG_CUDA(cudaMemsetAsync(partial, 0, MR_EBLOCKS * sizeof(double), st));
  }
  mr_energy_kernel<1><<<MR_EBLOCKS, MR_NT, 0, st>>>(A, z.n1, partial + MR_EBLOCKS);
  DSRG_LAUNCH_CHECK();
  DSRG_TRY(ordered_sum(partial, 2 * MR_EBLOCKS, e_dev, false, st));
  double e = 0.0;
  DSRG_CUDA(cudaMemcpyAsync(&e, e_dev, sizeof(double), cudaMemcpyDeviceToHost, st));
  DSRG_CUDA(cudaStreamSynchronize(st));
  *e_out = 2.0 * e;
  return DSRG_FNO_OK;
}

}  // namespace dsrg
