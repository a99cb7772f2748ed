// Symmetric eigensolver (Eq. 8: Gamma V = n V) and helpers.
//
// Cyclic two-sided Jacobi with round-robin pair ordering: in each round the
// indices form m/2 disjoint pairs (m = n rounded up to even, a padding index
// never rotates), so A' = J^T A J and V' = V J update every 2 x 2 block of A
// and every column pair of V independently.  The rotation of a pair (p, q)
// annihilates a_pq: tau = (a_qq - a_pp) / (2 a_pq), t = sign(tau) / (|tau| +
// sqrt(1 + tau^2)), c = 1/sqrt(1 + t^2), s = t c (Golub and Van Loan, "Matrix
// Computations", Sec. 8.5).
//
// GB300 runs float64 at a small fraction of its float32 rate, so the matrix
// and the vectors are kept in double-float (hi + lo float32 pairs, ~48 bits)
// and all rounds and sweeps run in one cooperative launch, separated by a
// grid barrier whose waits are bounded.  t is formed in float32 from the
// double-float difference a_qq - a_pp; c and s are then formed in
// double-float from that float t so that c^2 + s^2 = 1 to double-float
// accuracy: the rotation is orthogonal to working precision even where t
// is not the exact annihilating angle, and the next sweep removes what is
// left of a_pq.  A is double-buffered (every block of A' reads four entries
// of A); V is updated in place (a thread owns a column pair).
#include <atomic>

#include "dd.cuh"
#include "kernels.h"

namespace dsrg {

namespace {

#ifndef JACOBI_THREADS
#define JACOBI_THREADS 256
#endif
#ifndef JACOBI_BLOCKS_PER_SM
#define JACOBI_BLOCKS_PER_SM 3
#endif
constexpr int JNT = JACOBI_THREADS;      // threads per block
constexpr int JMAX_BLOCKS = EIG_MAX_BLOCKS;
constexpr long long BAR_SPIN_LIMIT = 20000000;  // ~2 s of 100 ns naps
// The grid barrier's spin limit on this device (a test hook may lower it to
// make the wait run out; dsrg_fno_debug_set_barrier_limit).
__device__ long long g_bar_spin_limit = BAR_SPIN_LIMIT;
constexpr int SMEM_JACOBI_N = 80;               // largest n solved in shared memory (150 KB)

// index at position pos of round r (position 0 fixed, the others rotate)
__device__ __forceinline__ int rr_index(int pos, int r, int m) {
  return pos == 0 ? 0 : ((pos - 1 + r) % (m - 1)) + 1;
}

struct JacobiArgs {
  int n, m;
  const double* A_in;
  double* A_out;  // full matrix: diagonal = eigenvalues
  double* V_out;
  float2* A0;     // double-float ping-pong buffers, n x n
  float2* A1;
  float2* V;      // double-float, n x n
  double* red;    // 2 * gridDim.x partial norms
  unsigned* bar;  // [0] arrivals, [1] generation
  int* status;    // [0] 1 = no convergence, [1] 1 = barrier wait expired, [2] sweeps
  int max_sweeps;
};

// Grid barrier (all blocks are co-resident: cooperative launch).  Returns
// false once any block's wait has expired; the kernel then returns.
// bar: [0] arrivals, [1] generation; status[1] is set when a wait expires.
__device__ bool grid_barrier_at(unsigned* bar, int* status) {
  __syncthreads();
  if (gridDim.x == 1) return true;  // one block: the block barrier is the grid barrier
  __shared__ int s_ok;
  if (threadIdx.x == 0) {
    volatile unsigned* gen = bar + 1;
    volatile int* st = status + 1;
    const unsigned g = *gen;
    __threadfence();
    int ok = *st == 0;
    const long long limit = g_bar_spin_limit;
    if (atomicAdd(bar, 1u) == gridDim.x - 1) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      long long it = 0;
      while (ok && *gen == g) {
        if (++it > limit || *st != 0) {
          atomicExch(status + 1, 1);
          ok = 0;
        }
        __nanosleep(100);
      }
    }
    __threadfence();
    s_ok = ok && *st == 0;
  }
  __syncthreads();
  return s_ok != 0;
}

__device__ bool grid_barrier(const JacobiArgs& P) { return grid_barrier_at(P.bar, P.status); }

__device__ __forceinline__ dd ldd(const float2* p, int i) {
  const float2 v = __ldcg(p + i);
  return {v.x, v.y};
}
__device__ __forceinline__ void sdd(float2* p, int i, dd v) { __stcg(p + i, make_float2(v.hi, v.lo)); }

// A, the ping-pong copy and V live in global memory (L2, bypassing L1 since
// other blocks write them), or, for a one-block solve of a small matrix, in
// shared memory (SM = true).
template <bool SM>
__device__ __forceinline__ dd ldx(const float2* p, int i) {
  if (SM) {
    const float2 v = p[i];
    return {v.x, v.y};
  }
  return ldd(p, i);
}
template <bool SM>
__device__ __forceinline__ void stx(float2* p, int i, dd v) {
  if (SM) p[i] = make_float2(v.hi, v.lo);
  else sdd(p, i, v);
}
template <bool SM>
__device__ __forceinline__ float2 ldx2(const float2* p, long i) {
  return SM ? p[i] : __ldcg(p + i);
}

// c a +- s b with double-float operands.  The sum keeps an absolute error
// of a few units of 2^-48 max(|c a|, |s b|), which is what the backward
// stability of the rotations needs (no relative accuracy under cancellation).
// The two products' high parts are exact (FMA TwoProduct) and summed with
// TwoSum; their low parts and the cross terms go into one float32 word.
__device__ __forceinline__ dd rot_combine(dd ca, dd a, dd sb, dd b, bool minus) {
  const float sh = minus ? -sb.hi : sb.hi, sl = minus ? -sb.lo : sb.lo;
  const float ph = __fmul_rn(ca.hi, a.hi), pl = __fmaf_rn(ca.hi, a.hi, -ph);
  const float qh = __fmul_rn(sh, b.hi), ql = __fmaf_rn(sh, b.hi, -qh);
  dd t = two_sum(ph, qh);
  float lo = __fadd_rn(t.lo, __fadd_rn(pl, ql));
  lo = __fmaf_rn(ca.hi, a.lo, lo);
  lo = __fmaf_rn(ca.lo, a.hi, lo);
  lo = __fmaf_rn(sh, b.lo, lo);
  lo = __fmaf_rn(sl, b.hi, lo);
  return quick_two_sum(t.hi, lo);
}

// 1 / sqrt(x) for x in [1, 2] in double-float: float estimate, two Newton steps
__device__ __forceinline__ dd dd_rsqrt12(dd x) {
  dd y = dd_make(rsqrtf(x.hi));
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const dd e = dd_sub(dd_make(1.0f), dd_mul(x, dd_mul(y, y)));
    y = dd_add_f(y, 0.5f * y.hi * e.hi);
  }
  return y;
}

// The shared-memory solve (SM) is block-local: one block per matrix (a grid
// may solve several), its barrier the block barrier.
template <bool SM>
__device__ __forceinline__ int jb_index() { return SM ? 0 : (int)blockIdx.x; }
template <bool SM>
__device__ __forceinline__ int jb_count() { return SM ? 1 : (int)gridDim.x; }
template <bool SM>
__device__ __forceinline__ bool jb_barrier(const JacobiArgs& P) {
  if (SM) {
    __syncthreads();
    return true;
  }
  return grid_barrier(P);
}

// squared off-diagonal and total Frobenius norms of A (fixed summation order)
template <bool SM>
__device__ void norms(const JacobiArgs& P, const float2* A, double* off, double* tot) {
  __shared__ double s_o[JNT], s_t[JNT];
  double o = 0.0, t = 0.0;
  const int n2 = P.n * P.n;
  const int bi = jb_index<SM>(), nb = jb_count<SM>();
  for (int idx = bi * JNT + threadIdx.x; idx < n2; idx += nb * JNT) {
    const float2 v = ldx2<SM>(A, idx);
    const double a = (double)v.x + (double)v.y;
    t += a * a;
    if (idx / P.n != idx % P.n) o += a * a;
  }
  s_o[threadIdx.x] = o;
  s_t[threadIdx.x] = t;
  __syncthreads();
  for (int w = JNT / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      s_o[threadIdx.x] += s_o[threadIdx.x + w];
      s_t[threadIdx.x] += s_t[threadIdx.x + w];
    }
    __syncthreads();
  }
  if (SM) {
    *off = s_o[0];
    *tot = s_t[0];
    __syncthreads();  // s_o, s_t are reused by the next call
    return;
  }
  if (threadIdx.x == 0) {
    __stcg(P.red + 2 * bi, s_o[0]);
    __stcg(P.red + 2 * bi + 1, s_t[0]);
  }
  if (!grid_barrier(P)) {
    *off = -1.0;
    return;
  }
  double so = 0.0, st = 0.0;
  for (int b = 0; b < nb; ++b) {
    so += __ldcg(P.red + 2 * b);
    st += __ldcg(P.red + 2 * b + 1);
  }
  *off = so;
  *tot = st;
}

template <bool SM>
__device__ void jacobi_solve(const JacobiArgs& P) {
  const int bi = jb_index<SM>(), nb = jb_count<SM>();
  // per pair k of the round: c (hi, lo), s (hi, lo), then the pair (p < q);
  // with SM, then A, its ping-pong copy and V (n^2 float2 each)
  extern __shared__ float4 s_cs[];
  int2* s_pq = reinterpret_cast<int2*>(s_cs + P.m / 2);
  const int n = P.n, m = P.m, half = m / 2;
  const long n2 = (long)n * n;
  float2* const A0 = SM ? reinterpret_cast<float2*>(s_cs + P.m) : P.A0;  // after s_pq (8 B x m/2 <= 16 B x m/2)
  float2* const A1 = SM ? A0 + n2 : P.A1;
  float2* const VV = SM ? A1 + n2 : P.V;
  for (long idx = bi * (long)JNT + threadIdx.x; idx < n2; idx += (long)nb * JNT) {
    const dd a = dd_from_double(P.A_in[idx]);
    stx<SM>(A0, (int)idx, a);
    stx<SM>(VV, (int)idx, dd_make(idx / n == idx % n ? 1.0f : 0.0f));
  }
  if (!jb_barrier<SM>(P)) return;
  float2* A = A0;
  float2* B = A1;
  // rounding floor of a converged double-float sweep, relative and squared
  const double tol = fmax(1e-30, ((double)n * 4e-15) * ((double)n * 4e-15));
  double prev = -1.0;
  int converged = 0, sweeps_done = 0;
  for (int sweep = 0; sweep <= P.max_sweeps; ++sweep) {
    sweeps_done = sweep;
    double off, tot;
    norms<SM>(P, A, &off, &tot);
    if (off < 0.0) return;
    if (tot == 0.0 || off <= tol * tot || (off <= 1e-22 * tot && prev >= 0.0 && off > 0.25 * prev)) {
      converged = 1;
      break;
    }
    prev = off;
    if (sweep == P.max_sweeps) break;
    for (int r = 0; r < m - 1; ++r) {
      // pairs and rotations of this round (each block forms all of them)
      for (int k = threadIdx.x; k < half; k += JNT) {
        const int i1 = rr_index(k, r, m), i2 = rr_index(m - 1 - k, r, m);
        const int p = min(i1, i2), q = max(i1, i2);
        float4 cs = make_float4(1.f, 0.f, 0.f, 0.f);
        if (q < n) {
          const dd apq = dd_mul_f(dd_add(ldx<SM>(A, p * n + q), ldx<SM>(A, q * n + p)), 0.5f);
          if (apq.hi != 0.0f) {
            const dd d = dd_sub(ldx<SM>(A, q * n + q), ldx<SM>(A, p * n + p));
            const float th = d.hi / (2.0f * apq.hi);
            const float t = (th >= 0.0f ? 1.0f : -1.0f) / (fabsf(th) + sqrtf(fmaf(th, th, 1.0f)));
            dd c = dd_rsqrt12(dd_add_f(two_prod(t, t), 1.0f));
            dd sn = dd_mul_f(c, t);
            // one first-order renormalisation: c^2 + s^2 = 1 to the last bits
            const float g = dd_sub(dd_add(dd_mul(c, c), dd_mul(sn, sn)), dd_make(1.0f)).hi;
            c = dd_add(c, dd_mul_f(c, -0.5f * g));
            sn = dd_add(sn, dd_mul_f(sn, -0.5f * g));
            cs = make_float4(c.hi, c.lo, sn.hi, sn.lo);
          }
        }
        s_cs[k] = cs;
        s_pq[k] = make_int2(p, q);
      }
      __syncthreads();
      // warp tasks: (item, 32 column pairs); items are the half row pairs of
      // A, then the n rows of V; lane = column pair within the task
      const int nchunks = (half + 31) >> 5;
      const int ntasks = (half + n) * nchunks;
      const float2* __restrict__ Ar = A;
      float2* __restrict__ Bw = B;
      float2* __restrict__ Vw = VV;
      const int lane = threadIdx.x & 31;
      const int nwarps = nb * (JNT / 32);
#pragma unroll 2
      for (int task = bi * (JNT / 32) + (threadIdx.x >> 5); task < ntasks; task += nwarps) {
        const int it = task / nchunks;
        const int k = (task - it * nchunks) * 32 + lane;
        if (k >= half) continue;
        const int2 pqc = s_pq[k];
        const int pc = pqc.x, qc = pqc.y;
        const bool qcr = qc < n;
        const float4 cc = s_cs[k];
        const dd cR = {cc.x, cc.y}, sR = {cc.z, cc.w};
        if (it < half) {
          const int2 pq = s_pq[it];
          const int p = pq.x, q = pq.y;
          const float4 rc = s_cs[it];
          const dd cP = {rc.x, rc.y}, sP = {rc.z, rc.w};
          // M = A[{p,q}, {pc,qc}] J_R
          const dd a_pp = ldx<SM>(Ar, p * n + pc);
          const dd a_pq = qcr ? ldx<SM>(Ar, p * n + qc) : dd_make(0.f);
          const dd m_p0 = qcr ? rot_combine(cR, a_pp, sR, a_pq, true) : a_pp;
          const dd m_p1 = qcr ? rot_combine(sR, a_pp, cR, a_pq, false) : dd_make(0.f);
          if (q < n) {
            const dd a_qp = ldx<SM>(Ar, q * n + pc);
            const dd a_qq = qcr ? ldx<SM>(Ar, q * n + qc) : dd_make(0.f);
            const dd m_q0 = qcr ? rot_combine(cR, a_qp, sR, a_qq, true) : a_qp;
            const dd m_q1 = qcr ? rot_combine(sR, a_qp, cR, a_qq, false) : dd_make(0.f);
            // A' = J_P^T M
            stx<SM>(Bw, p * n + pc, rot_combine(cP, m_p0, sP, m_q0, true));
            stx<SM>(Bw, q * n + pc, rot_combine(sP, m_p0, cP, m_q0, false));
            if (qcr) {
              stx<SM>(Bw, p * n + qc, rot_combine(cP, m_p1, sP, m_q1, true));
              stx<SM>(Bw, q * n + qc, rot_combine(sP, m_p1, cP, m_q1, false));
            }
          } else {
            stx<SM>(Bw, p * n + pc, m_p0);
            if (qcr) stx<SM>(Bw, p * n + qc, m_p1);
          }
        } else if (qcr) {
          const int i = it - half;
          const dd v0 = ldx<SM>(Vw, i * n + pc), v1 = ldx<SM>(Vw, i * n + qc);
          stx<SM>(Vw, i * n + pc, rot_combine(cR, v0, sR, v1, true));
          stx<SM>(Vw, i * n + qc, rot_combine(sR, v0, cR, v1, false));
        }
      }
      if (!jb_barrier<SM>(P)) return;
      float2* tmp = A;
      A = B;
      B = tmp;
    }
  }
  // Columns of V drift from unit length by rounding of the rotations; with
  // V = Vn N (N the column norms) the Rayleigh quotients become a_jj / N_j^2.
  double* nrm2 = reinterpret_cast<double*>(B);  // the free ping-pong buffer (n^2 >= n doubles)
  for (int j = bi * JNT + threadIdx.x; j < n; j += nb * JNT) {
    dd acc = dd_make(0.0f);
    for (int i = 0; i < n; ++i) {
      const dd v = ldx<SM>(VV, i * n + j);
      acc = dd_add(acc, dd_mul(v, v));
    }
    if (SM) nrm2[j] = dd_to_double(acc);
    else __stcg(nrm2 + j, dd_to_double(acc));
  }
  if (!jb_barrier<SM>(P)) return;
  for (long idx = bi * (long)JNT + threadIdx.x; idx < n2; idx += (long)nb * JNT) {
    const int i = (int)(idx / n), j = (int)(idx % n);
    const float2 a = ldx2<SM>(A, idx), v = ldx2<SM>(VV, idx);
    const double nj = SM ? nrm2[j] : __ldcg(nrm2 + j);
    const double ni = SM ? nrm2[i] : __ldcg(nrm2 + i);
    P.A_out[idx] = ((double)a.x + (double)a.y) / (i == j ? nj : sqrt(nj * ni));
    P.V_out[idx] = ((double)v.x + (double)v.y) / sqrt(nj);
  }
  if (bi == 0 && threadIdx.x == 0) {
    P.status[0] = converged ? 0 : 1;
    P.status[2] = sweeps_done;
  }
}

template <bool SM>
__global__ void __launch_bounds__(JNT, JACOBI_BLOCKS_PER_SM) jacobi_coop_kernel(JacobiArgs P) {
  jacobi_solve<SM>(P);
}

// several small matrices in shared memory, one block each
constexpr int JBATCH_MAX = 4;
struct JacobiBatch {
  JacobiArgs a[JBATCH_MAX];
};
__global__ void __launch_bounds__(JNT, 1) jacobi_smem_batch_kernel(const __grid_constant__ JacobiBatch B) {
  jacobi_solve<true>(B.a[blockIdx.x]);
}


// The rotation (c, s) that annihilates a_pq (a_pp, a_qq, a_pq double-float):
// t from float32 arithmetic on the double-float difference, c and s in
// double-float renormalised so that c^2 + s^2 = 1 to working precision.
__device__ __forceinline__ float4 jacobi_rotation(dd app, dd aqq, dd apq) {
  if (apq.hi == 0.0f) return make_float4(1.f, 0.f, 0.f, 0.f);
  const dd d = dd_sub(aqq, app);
  const float th = d.hi / (2.0f * apq.hi);
  const float t = (th >= 0.0f ? 1.0f : -1.0f) / (fabsf(th) + sqrtf(fmaf(th, th, 1.0f)));
  dd c = dd_rsqrt12(dd_add_f(two_prod(t, t), 1.0f));
  dd sn = dd_mul_f(c, t);
  const float g = dd_sub(dd_add(dd_mul(c, c), dd_mul(sn, sn)), dd_make(1.0f)).hi;
  c = dd_add(c, dd_mul_f(c, -0.5f * g));
  sn = dd_add(sn, dd_mul_f(sn, -0.5f * g));
  return make_float4(c.hi, c.lo, sn.hi, sn.lo);
}

// position of index j in round r of the round-robin ordering (inverse of rr_index)
__device__ __forceinline__ int rr_position(int j, int r, int m) {
  return j == 0 ? 0 : ((j - 1 - r) % (m - 1) + (m - 1)) % (m - 1) + 1;
}

// ---------------------------------------------------------------------------
// Column-pair Jacobi.  The same cyclic two-sided Jacobi with round-robin
// pairs, organised around column pairs: in a round, block b owns the column
// pairs k in [b cp, (b+1) cp) of A and V.  For its pair (p, q) it reads
// columns p and q (A in column-major double-float; A stays symmetric), forms
// M = A J on them, then A' = J^T M for every row pair of the round (the
// rotations of all pairs are known to every block), rotates V's columns p, q,
// and writes the columns back.  With the new columns it publishes a_jj and
// a_{partner(j), j} for the next round's pairing, from which every block
// forms all rotations of the next round: one grid barrier per round, the
// matrix moving through L2 once per round.
struct ColPairArgs {
  int n, m, half, cp, cpc;  // pairs per block, pairs held in shared memory at a time
  const double* A_in;
  double* A_out;
  double* V_out;
  float2* Ac;    // [n][n]: Ac[j][i] = A[i][j]
  float2* Vc;    // [n][n]: Vc[j][i] = V[i][j]
  float2* pub;   // [2][2][m]: per parity, a_jj and a_{partner(j), j}
  double* nrm2;  // [n] squared column norms of V
  double* red;   // 2 * gridDim.x partial norms
  unsigned* bar;
  int* status;   // [0] 1 = no convergence, [1] 1 = barrier wait expired, [2] sweeps
  int max_sweeps;
};

// threads per block of the column-pair kernel: one block per SM, so the
// latency of its column loads is hidden by the warps of that one block
constexpr int CPT = 1024;

// the round that follows round r of sweep `sw` (the next sweep starts at round 0)
__device__ __forceinline__ int next_round(int r, int m) { return r + 1 < m - 1 ? r + 1 : 0; }

__global__ void __launch_bounds__(CPT) jacobi_colpair_kernel(ColPairArgs P) {
  extern __shared__ float4 s_rot[];                              // [half]
  int2* s_pair = reinterpret_cast<int2*>(s_rot + P.half);       // [half]
  float2* colP = reinterpret_cast<float2*>(s_pair + P.half);   // [2 cpc][n]: p and q columns of each pair
  const int n = P.n, m = P.m, half = P.half;
  const long n2 = (long)n * n;
  // ---- set-up: A (symmetrised) and V = 1 in columns, round 0's inputs
  for (long idx = blockIdx.x * (long)CPT + threadIdx.x; idx < n2; idx += (long)gridDim.x * CPT) {
    const int j = (int)(idx / n), i = (int)(idx % n);
    const dd a = dd_from_double(0.5 * (P.A_in[(long)i * n + j] + P.A_in[(long)j * n + i]));
    P.Ac[idx] = make_float2(a.hi, a.lo);
    P.Vc[idx] = make_float2(i == j ? 1.0f : 0.0f, 0.0f);
  }
  for (int j = blockIdx.x * CPT + threadIdx.x; j < n; j += gridDim.x * CPT) {
    const int pos = rr_position(j, 0, m);
    const int pj = rr_index(m - 1 - pos, 0, m);
    const double a = 0.5 * (P.A_in[(long)j * n + j] + P.A_in[(long)j * n + j]);
    const dd djj = dd_from_double(a);
    dd off = dd_make(0.0f);
    if (pj < n) off = dd_from_double(0.5 * (P.A_in[(long)pj * n + j] + P.A_in[(long)j * n + pj]));
    P.pub[j] = make_float2(djj.hi, djj.lo);
    P.pub[m + j] = make_float2(off.hi, off.lo);
  }
  if (!grid_barrier_at(P.bar, P.status)) return;
  const double tol = fmax(1e-30, ((double)n * 4e-15) * ((double)n * 4e-15));
  double prev = -1.0;
  int converged = 0, sweeps_done = 0, cur = 0;
  for (int sweep = 0; sweep <= P.max_sweeps; ++sweep) {
    sweeps_done = sweep;
    // ---- convergence: off-diagonal and total squared norms (fixed order)
    {
      __shared__ double s_o[CPT], s_t[CPT];
      double o = 0.0, t = 0.0;
      for (long idx = blockIdx.x * (long)CPT + threadIdx.x; idx < n2; idx += (long)gridDim.x * CPT) {
        const float2 v = __ldcg(P.Ac + idx);
        const double a = (double)v.x + (double)v.y;
        t += a * a;
        if (idx / n != idx % n) o += a * a;
      }
      s_o[threadIdx.x] = o;
      s_t[threadIdx.x] = t;
      __syncthreads();
      for (int w = CPT / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
          s_o[threadIdx.x] += s_o[threadIdx.x + w];
          s_t[threadIdx.x] += s_t[threadIdx.x + w];
        }
        __syncthreads();
      }
      if (threadIdx.x == 0) {
        __stcg(P.red + 2 * blockIdx.x, s_o[0]);
        __stcg(P.red + 2 * blockIdx.x + 1, s_t[0]);
      }
      if (!grid_barrier_at(P.bar, P.status)) return;
      double so = 0.0, st = 0.0;
      for (int b = 0; b < (int)gridDim.x; ++b) {
        so += __ldcg(P.red + 2 * b);
        st += __ldcg(P.red + 2 * b + 1);
      }
      if (st == 0.0 || so <= tol * st || (so <= 1e-22 * st && prev >= 0.0 && so > 0.25 * prev)) {
        converged = 1;
        break;
      }
      prev = so;
      if (sweep == P.max_sweeps) break;
    }
    for (int r = 0; r < m - 1; ++r) {
      const float2* pd = P.pub + (size_t)cur * 2 * m;      // a_jj
      const float2* po = pd + m;                             // a_{partner(j), j}
      // ---- all rotations of this round, from the published entries
      for (int k = threadIdx.x; k < half; k += CPT) {
        const int i1 = rr_index(k, r, m), i2 = rr_index(m - 1 - k, r, m);
        const int p = min(i1, i2), q = max(i1, i2);
        float4 cs = make_float4(1.f, 0.f, 0.f, 0.f);
        if (q < n) {
          const float2 dp = __ldcg(pd + p), dq = __ldcg(pd + q), op = __ldcg(po + p), oq = __ldcg(po + q);
          const dd apq = dd_mul_f(dd_add(dd{op.x, op.y}, dd{oq.x, oq.y}), 0.5f);
          cs = jacobi_rotation(dd{dp.x, dp.y}, dd{dq.x, dq.y}, apq);
        }
        s_rot[k] = cs;
        s_pair[k] = make_int2(p, q);
      }
      __syncthreads();
      float2* nd = P.pub + (size_t)(cur ^ 1) * 2 * m;
      float2* no = nd + m;
      const int rn = next_round(r, m);
      const int k0 = blockIdx.x * P.cp;
      const int kend = min(k0 + P.cp, half);
      // this block's pairs, P.cpc at a time (as many as shared memory holds)
      for (int kb = k0; kb < kend; kb += P.cpc) {
        const int nk = min(P.cpc, kend - kb);
        // M = A J on columns p, q of each pair (colP / colQ rows of length n)
        for (int idx = threadIdx.x; idx < nk * n; idx += CPT) {
          const int kk = idx / n, i = idx - kk * n;
          const int2 pq = s_pair[kb + kk];
          const float4 cc = s_rot[kb + kk];
          const dd c = {cc.x, cc.y}, sn = {cc.z, cc.w};
          const float2 a = __ldcg(P.Ac + (long)pq.x * n + i);
          float2* cP = colP + (size_t)kk * 2 * n;
          if (pq.y < n) {
            const float2 b = __ldcg(P.Ac + (long)pq.y * n + i);
            const dd ap = {a.x, a.y}, aq = {b.x, b.y};
            const dd mp = rot_combine(c, ap, sn, aq, true), mq = rot_combine(sn, ap, c, aq, false);
            cP[i] = make_float2(mp.hi, mp.lo);
            cP[n + i] = make_float2(mq.hi, mq.lo);
            // V J on the same columns (rows are independent)
            const float2 va = __ldcg(P.Vc + (long)pq.x * n + i), vb = __ldcg(P.Vc + (long)pq.y * n + i);
            const dd vp = {va.x, va.y}, vq = {vb.x, vb.y};
            const dd wp = rot_combine(c, vp, sn, vq, true), wq = rot_combine(sn, vp, c, vq, false);
            __stcg(P.Vc + (long)pq.x * n + i, make_float2(wp.hi, wp.lo));
            __stcg(P.Vc + (long)pq.y * n + i, make_float2(wq.hi, wq.lo));
          } else {
            cP[i] = a;
          }
        }
        __syncthreads();
        // A' = J^T M: every row pair of the round, on every loaded column, in place
        for (int idx = threadIdx.x; idx < nk * 2 * half; idx += CPT) {
          const int col = idx / half, k2 = idx - col * half;   // col: 2 kk + (0: p, 1: q)
          const int kk = col >> 1;
          if ((col & 1) && s_pair[kb + kk].y >= n) continue;
          const int2 rq = s_pair[k2];
          if (rq.y >= n) continue;
          const float4 rc = s_rot[k2];
          const dd cr = {rc.x, rc.y}, sr = {rc.z, rc.w};
          float2* cc = colP + (size_t)col * n;
          const float2 x = cc[rq.x], y = cc[rq.y];
          const dd xp = {x.x, x.y}, yq = {y.x, y.y};
          const dd u = rot_combine(cr, xp, sr, yq, true), v = rot_combine(sr, xp, cr, yq, false);
          cc[rq.x] = make_float2(u.hi, u.lo);
          cc[rq.y] = make_float2(v.hi, v.lo);
        }
        __syncthreads();
        for (int idx = threadIdx.x; idx < nk * 2 * n; idx += CPT) {
          const int col = idx / n, i = idx - col * n;
          const int2 pq = s_pair[kb + (col >> 1)];
          const int j = (col & 1) ? pq.y : pq.x;
          if (j < n) __stcg(P.Ac + (long)j * n + i, colP[(size_t)col * n + i]);
        }
        // the next round's inputs of the loaded columns
        for (int col = threadIdx.x; col < 2 * nk; col += CPT) {
          const int2 pq = s_pair[kb + (col >> 1)];
          const int j = (col & 1) ? pq.y : pq.x;
          if (j >= n) continue;
          const float2* cc = colP + (size_t)col * n;
          const int pj = rr_index(m - 1 - rr_position(j, rn, m), rn, m);
          __stcg(nd + j, cc[j]);
          __stcg(no + j, pj < n ? cc[pj] : make_float2(0.f, 0.f));
        }
        __syncthreads();
      }
      if (!grid_barrier_at(P.bar, P.status)) return;
      cur ^= 1;
    }
  }
  // ---- output: Rayleigh quotients and eigenvectors normalised by the
  // column norms of V (they drift from 1 by rounding of the rotations)
  double* nrm2 = P.nrm2;
  for (int j = blockIdx.x; j < n; j += gridDim.x) {
    __shared__ double s_r[CPT];
    double acc = 0.0;
    for (int i = threadIdx.x; i < n; i += CPT) {
      const float2 v = __ldcg(P.Vc + (long)j * n + i);
      const dd vv = dd_mul(dd{v.x, v.y}, dd{v.x, v.y});
      acc += dd_to_double(vv);
    }
    s_r[threadIdx.x] = acc;
    __syncthreads();
    for (int w = CPT / 2; w > 0; w >>= 1) {
      if (threadIdx.x < w) s_r[threadIdx.x] += s_r[threadIdx.x + w];
      __syncthreads();
    }
    if (threadIdx.x == 0) __stcg(nrm2 + j, s_r[0]);
    __syncthreads();
  }
  if (!grid_barrier_at(P.bar, P.status)) return;
  for (long idx = blockIdx.x * (long)CPT + threadIdx.x; idx < n2; idx += (long)gridDim.x * CPT) {
    const int i = (int)(idx / n), j = (int)(idx % n);
    const float2 a = __ldcg(P.Ac + (long)j * n + i), v = __ldcg(P.Vc + (long)j * n + i);
    const double nj = __ldcg(nrm2 + j), ni = __ldcg(nrm2 + i);
    P.A_out[idx] = ((double)a.x + (double)a.y) / (i == j ? nj : sqrt(nj * ni));
    P.V_out[idx] = ((double)v.x + (double)v.y) / sqrt(nj);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    P.status[0] = converged ? 0 : 1;
    P.status[2] = sweeps_done;
  }
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

static thread_local bool t_device_shared = false;

SharedDeviceScope::SharedDeviceScope(bool shared) : prev(t_device_shared) { t_device_shared = shared; }
SharedDeviceScope::~SharedDeviceScope() { t_device_shared = prev; }

// A (n x n, symmetric) is destroyed: on return its diagonal holds the
// eigenvalues; V (n x n) receives the eigenvectors (column j <-> A[j][j]).
// work: eig_work_doubles(n) doubles.  status_dev: four ints of device memory.
// Matrices above the shared-memory size: the column-pair kernel (default) or
// the round-parallel kernel over A in global memory (test hook, comparison).
static std::atomic<int> g_eig_colpair{1};
void set_eig_colpair(bool on) { g_eig_colpair.store(on ? 1 : 0); }

static int eig_colpair(int n, int m, double* A, double* V, double* work, int* status_dev, int max_sweeps,
                       cudaStream_t st) {
  const long n2 = (long)n * n;
  ColPairArgs P;
  P.n = n;
  P.m = m;
  P.half = m / 2;
  P.A_in = A;
  P.A_out = A;
  P.V_out = V;
  P.Ac = reinterpret_cast<float2*>(work);
  P.Vc = reinterpret_cast<float2*>(work + 2 * n2);
  P.pub = reinterpret_cast<float2*>(work + n2);
  P.nrm2 = work + n2 + 4 * (long)m + 16;
  P.red = work + 3 * n2;
  P.bar = reinterpret_cast<unsigned*>(work + 3 * n2 + 2 * JMAX_BLOCKS);
  P.status = status_dev;
  P.max_sweeps = max_sweeps;
  const size_t table = (sizeof(float4) + sizeof(int2)) * (size_t)P.half;
  const size_t per_pair = 2 * sizeof(float2) * (size_t)n;
  const size_t cap = 200 * 1024;
  if (table + per_pair > cap || n2 < 4 * (long)m + 16 + n) return DSRG_FNO_ERR_UNSUPPORTED;
  auto kern = jacobi_colpair_kernel;
  int dev = 0, sms = 0;
  DSRG_CUDA(cudaGetDevice(&dev));
  DSRG_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  // one block per SM: a round ends in a grid barrier whose arrivals are
  // serialised atomics, so more blocks make every round slower; the pairs of
  // a block are rotated together, as many at a time as shared memory holds
  // (half the SMs when batch workers share the device: their solves overlap)
  const int G = std::max(1, std::min(std::min(t_device_shared ? sms / 2 : sms, JMAX_BLOCKS), P.half));
  P.cp = (P.half + G - 1) / G;
  P.cpc = (int)std::max<size_t>(1, std::min<size_t>((size_t)P.cp, (cap - table) / per_pair));
  const size_t smem = table + per_pair * (size_t)P.cpc;
  if (smem > 48 * 1024) DSRG_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cap));
  int occ = 0;
  DSRG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, CPT, smem));
  if (occ < 1) return DSRG_FNO_ERR_UNSUPPORTED;
  const int grid = (P.half + P.cp - 1) / P.cp;
  void* args[] = {&P};
  DSRG_CUDA(cudaLaunchCooperativeKernel((const void*)kern, dim3(grid), dim3(CPT), args, smem, st));
  DSRG_LAUNCH_CHECK();
  int h[3] = {0, 0, 0};
  DSRG_CUDA(cudaMemcpyAsync(h, status_dev, 3 * sizeof(int), cudaMemcpyDeviceToHost, st));
  DSRG_CUDA(cudaStreamSynchronize(st));
  prof_count(n >= 256 ? "eig_sweeps_large" : "eig_sweeps_small", (double)h[2]);
  if (h[1]) return DSRG_FNO_ERR_TIMEOUT;
  return h[0] ? DSRG_FNO_ERR_NOCONV : DSRG_FNO_OK;
}

// Spin limit of the grid barrier on the current device; spins <= 0 restores
// the default (test hook: a tiny limit makes the barrier's wait run out).
int eig_set_barrier_limit(long long spins) {
  const long long v = spins > 0 ? spins : BAR_SPIN_LIMIT;
  DSRG_CUDA(cudaMemcpyToSymbol(g_bar_spin_limit, &v, sizeof(v)));
  return DSRG_FNO_OK;
}

int eig_sym_jacobi(int n, double* A, double* V, double* work, int* status_dev, int max_sweeps,
                   cudaStream_t st) {
  if (n <= 0) return DSRG_FNO_OK;
  const int m = (n % 2 == 0) ? n : n + 1;
  const long n2 = (long)n * n;
  JacobiArgs P;
  P.n = n;
  P.m = m;
  P.A_in = A;
  P.A_out = A;
  P.V_out = V;
  P.A0 = reinterpret_cast<float2*>(work);
  P.A1 = reinterpret_cast<float2*>(work + n2);
  P.V = reinterpret_cast<float2*>(work + 2 * n2);
  P.red = work + 3 * n2;
  P.bar = reinterpret_cast<unsigned*>(work + 3 * n2 + 2 * JMAX_BLOCKS);
  P.status = status_dev;
  P.max_sweeps = max_sweeps;
  DSRG_CUDA(cudaMemsetAsync(P.bar, 0, 2 * sizeof(unsigned), st));
  DSRG_CUDA(cudaMemsetAsync(status_dev, 0, 4 * sizeof(int), st));
  if ((long)n * n >= (1L << 31)) return DSRG_FNO_ERR_UNSUPPORTED;  // 32-bit element offsets
  constexpr int SMEM_CEILING = 200 * 1024;
  // small matrices: one block with A, its copy and V in shared memory
  const bool in_smem = n <= SMEM_JACOBI_N;
  const size_t smem = in_smem ? sizeof(float4) * (size_t)m + 3 * sizeof(float2) * (size_t)n * n
                              : (sizeof(float4) + sizeof(int2)) * (size_t)(m / 2);
  if (smem > (size_t)SMEM_CEILING) return DSRG_FNO_ERR_UNSUPPORTED;
  // (the column-pair kernel stages two columns of n per pair: above n of
  // about 7000 it does not fit, and the round-parallel kernel takes the matrix)
  if (!in_smem && g_eig_colpair.load()) {
    const int rc = eig_colpair(n, m, A, V, work, status_dev, max_sweeps, st);
    if (rc != DSRG_FNO_ERR_UNSUPPORTED) return rc;
  }
  auto kern = in_smem ? jacobi_coop_kernel<true> : jacobi_coop_kernel<false>;
  // one fixed ceiling for every launch: concurrent callers (batch workers)
  // never lower it under one another
  if (smem > 48 * 1024)
    DSRG_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_CEILING));
  int dev = 0, sms = 0, occ = 0;
  DSRG_CUDA(cudaGetDevice(&dev));
  DSRG_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  DSRG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, JNT, smem));
  if (occ < 1) return DSRG_FNO_ERR_UNSUPPORTED;
  // (half + n) items of half column pairs per round, about two per thread
  // on a device of its own: a round's tasks are chains of dependent L2 round
  // trips, so short chains over more blocks beat the extra grid-barrier
  // arrivals (GB300, random spectra: n = 200 31.7 -> 17.8 ms, n = 400 65 ->
  // 43 ms against eight per thread; n >= ~1100 is capped by the co-resident
  // grid either way).  On a shared device, eight per thread: there the extra
  // resident blocks cost the other workers more than they save (64-instance
  // batch 3.30 -> 3.67 s with two per thread).
  const long units = (long)(m / 2 + n) * (m / 2);
  const long per_block = (t_device_shared ? 8 : 2) * (long)JNT;
  int nblk = (int)std::min<long>(std::min(sms * std::min(occ, JACOBI_BLOCKS_PER_SM), JMAX_BLOCKS),
                                 (units + per_block - 1) / per_block);
  nblk = in_smem ? 1 : std::max(nblk, 1);
  if (nblk == 1) {
    // one block: its barrier is __syncthreads, no co-residency to guarantee
    kern<<<1, JNT, smem, st>>>(P);
  } else {
    void* args[] = {&P};
    DSRG_CUDA(cudaLaunchCooperativeKernel((const void*)kern, dim3(nblk), dim3(JNT), args, smem, st));
  }
  DSRG_LAUNCH_CHECK();
  int h[3] = {0, 0, 0};
  DSRG_CUDA(cudaMemcpyAsync(h, status_dev, 3 * sizeof(int), cudaMemcpyDeviceToHost, st));
  DSRG_CUDA(cudaStreamSynchronize(st));
  prof_count(n >= 256 ? "eig_sweeps_large" : "eig_sweeps_small", (double)h[2]);
  if (h[1]) return DSRG_FNO_ERR_TIMEOUT;
  return h[0] ? DSRG_FNO_ERR_NOCONV : DSRG_FNO_OK;
}

int eig_sym_jacobi_batch(int count, const int* n, double* const* A, double* const* V, double* const* work,
                         int* status_dev, int max_sweeps, cudaStream_t st) {
  if (count <= 0) return DSRG_FNO_OK;
  if (count > JBATCH_MAX) return DSRG_FNO_ERR_ARG;
  // matrices above the shared-memory size: one solve each, as eig_sym_jacobi
  for (int e = 0; e < count; ++e)
    if (n[e] > SMEM_JACOBI_N) DSRG_TRY(eig_sym_jacobi(n[e], A[e], V[e], work[e], status_dev + 4 * e, max_sweeps, st));
  JacobiBatch Bt{};
  int idx[JBATCH_MAX];
  int k = 0;
  size_t smem = 0;
  for (int e = 0; e < count; ++e) {
    if (n[e] <= 0 || n[e] > SMEM_JACOBI_N) continue;
    const int m = (n[e] % 2 == 0) ? n[e] : n[e] + 1;
    const long n2 = (long)n[e] * n[e];
    JacobiArgs& P = Bt.a[k];
    P.n = n[e];
    P.m = m;
    P.A_in = A[e];
    P.A_out = A[e];
    P.V_out = V[e];
    P.A0 = P.A1 = P.V = nullptr;  // in shared memory
    P.red = work[e] + 3 * n2;
    P.bar = reinterpret_cast<unsigned*>(work[e] + 3 * n2 + 2 * JMAX_BLOCKS);
    P.status = status_dev + 4 * e;
    P.max_sweeps = max_sweeps;
    smem = std::max(smem, sizeof(float4) * (size_t)m + 3 * sizeof(float2) * (size_t)n2);
    DSRG_CUDA(cudaMemsetAsync(P.status, 0, 4 * sizeof(int), st));
    idx[k++] = e;
  }
  if (k == 0) return DSRG_FNO_OK;
  if (smem > 48 * 1024)
    DSRG_CUDA(cudaFuncSetAttribute(jacobi_smem_batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   200 * 1024));
  jacobi_smem_batch_kernel<<<k, JNT, smem, st>>>(Bt);
  DSRG_LAUNCH_CHECK();
  int h[4 * JBATCH_MAX];
  DSRG_CUDA(cudaMemcpyAsync(h, status_dev, 4 * count * sizeof(int), cudaMemcpyDeviceToHost, st));
  DSRG_CUDA(cudaStreamSynchronize(st));
  int rc = DSRG_FNO_OK;
  for (int q = 0; q < k; ++q) {
    const int e = idx[q];
    prof_count("eig_sweeps_small", (double)h[4 * e + 2]);
    if (h[4 * e]) rc = DSRG_FNO_ERR_NOCONV;
  }
  return rc;
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
