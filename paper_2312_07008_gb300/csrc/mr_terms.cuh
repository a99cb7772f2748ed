// Element bodies of the full multi-reference PT2 energy (energy_mr.cu).
//
// E^(2) = <[H, A]>_0 + 1/2 <[[H0, A], A]>_0 (Eq. A4's H-bar to second order)
// equals 2 <[X, T]>_0, X the de-excitation vertex (upper holes, lower
// particles) X2^{ij}_{ab} = <ab|ij> - 1/2 Delta^{ij}_{ab} t^{ij}_{ab},
// X1^i_a = f^i_a - 1/2 Delta^i_a t^i_a + 1/2 r^i_a, with the amplitudes of
// Eqs. A6, A7.  The doubles whose particles are both virtual give E_vv (the
// pair-contraction path); everything else is computed here in float64 from
// the tensors with one active particle index y:
//   tp[i][j][a][y] = t^{ij}_{ay},  xp[i][j][a][y] = X2^{ij}_{ay}
// (i, j holes, a any particle, y active; t^{ij}_{ya} = tp[j][i][a][y] by the
// pair symmetry, all-active entries zero), and the singles t1, x1 [i][a].
// Each energy term is a dot product of X with a linear image Y of T (the
// generalised Wick contractions: Gamma over holes, Theta over particles, one
// density cumulant); the stages below form the partial images Y needs.
//
// The functions are plain per-element bodies so that every kernel is a
// one-line loop over them.
#pragma once

#include "common.cuh"

namespace dsrg {

struct MRArgs {
  int nc, na, nv, nh, np;
  double s;
  const double* eps;   // [nc + na + nv]: core | active | virtual
  const double* f_hp;  // [nh][np] off-diagonal Fock f^i_a, or null (zero)
  const double* g1;    // [na][na] Gamma1
  const double* l2;    // [na]^4 Lambda^{uv}_{xy} at ((u na + v) na + x) na + y
  const double* l3;    // [na]^6 Lambda^{xyz}_{uvw}, or null (3-cumulant terms dropped)
  const double* nu;    // <ay|ij> from the GEMM, at ((i np + a) nh + j) na + y
  double* tp;          // [nh][nh][np][na]
  double* xp;          // [nh][nh][np][na]
  double* t1;          // [nh][np]
  double* x1;          // [nh][np]
  double* z1;          // [l][k][a][c] = sum_d Theta_{da} tp[l][k][d][c]
  double* tpp;         // [l][k][a][y] = sum_c Theta_{yc} z1[l][k][a][c]
  double* z2;          // [l'][j][a][c] = sum_k Gamma_{jk} z1[nc+l'][k][a][c]
  double* z3;          // [j][k'][a][c] = sum_l Gamma_{jl} z1[l][nc+k'][a][c]
  double* g2t;         // [i][j][c][d] = sum_{kl} Gamma_{il} Gamma_{jk} tp[k][l][c][d]   (c, d active)
  double* w3;          // [j][l'][c][d] = sum_k Gamma_{jk} tp[k][nc+l'][c][d]           (c, d active)
  double* tt1;         // [k][a] = sum_c t1[k][c] Theta_{ca}
  double* gt1;         // [j][c] = sum_k Gamma_{jk} t1[k][c]                            (c active)
};

// sizes of the element loops
__host__ __device__ inline long mr_n4(const MRArgs& A) { return (long)A.nh * A.nh * A.np * A.na; }
__host__ __device__ inline long mr_n4a(const MRArgs& A) { return (long)A.na * A.nh * A.np * A.na; }

__host__ __device__ inline long mr_at(const MRArgs& A, int i, int j, int a, int y) {
  return (((long)i * A.nh + j) * A.np + a) * A.na + y;
}
__host__ __device__ inline double mr_L2(const MRArgs& A, int u, int v, int x, int y) {
  return A.l2[((u * A.na + v) * A.na + x) * A.na + y];
}
__host__ __device__ inline double mr_L3(const MRArgs& A, int x, int y, int z, int u, int v, int w) {
  const long n = A.na;
  return A.l3[((((x * n + y) * n + z) * n + u) * n + v) * n + w];
}
// Theta over the particles: 2 delta - Gamma1 on the active block, 2 delta on the virtual one
__host__ __device__ inline double mr_th(const MRArgs& A, int a, int c) {
  double t = a == c ? 2.0 : 0.0;
  if (a < A.na && c < A.na) t -= A.g1[a * A.na + c];
  return t;
}

// Eq. A7 for the doubles with an active particle y, and the vertex X2.
__host__ __device__ inline void mr_amp_elem(const MRArgs& A, long idx) {
  const int y = (int)(idx % A.na);
  const int a = (int)((idx / A.na) % A.np);
  const int j = (int)((idx / ((long)A.na * A.np)) % A.nh);
  const int i = (int)(idx / ((long)A.na * A.np * A.nh));
  if (i >= A.nc && j >= A.nc && a < A.na) {
    A.tp[idx] = 0.0;
    A.xp[idx] = 0.0;
    return;
  }
  const double nu = A.nu[(((long)i * A.np + a) * A.nh + j) * A.na + y];
  const double d = A.eps[i] + A.eps[j] - A.eps[A.nc + a] - A.eps[A.nc + y];
  const double t = nu * regularizer(d, A.s);
  A.tp[idx] = t;
  A.xp[idx] = fma(-0.5 * d, t, nu);
}

// Eq. A6 for every hole i and particle a (not both active), and the vertex X1:
// t = (f + r) R(Delta^i_a), r = 1/2 sum_{ux} (eps_x - eps_u) Gamma^x_u (2 t^{iu}_{ax} - t^{ui}_{ax}),
// x1 = f - 1/2 Delta t + 1/2 r.
__host__ __device__ inline void mr_t1_elem(const MRArgs& A, long idx) {
  const int a = (int)(idx % A.np);
  const int i = (int)(idx / A.np);
  if (i >= A.nc && a < A.na) {
    A.t1[idx] = 0.0;
    A.x1[idx] = 0.0;
    return;
  }
  const double f = A.f_hp ? A.f_hp[idx] : 0.0;
  double r = 0.0;
  for (int u = 0; u < A.na; ++u) {
    const double eu = A.eps[A.nc + u];
    for (int x = 0; x < A.na; ++x) {
      const double tch = 2.0 * A.tp[mr_at(A, i, A.nc + u, a, x)] - A.tp[mr_at(A, A.nc + u, i, a, x)];
      r = fma((A.eps[A.nc + x] - eu) * A.g1[x * A.na + u], tch, r);
    }
  }
  r *= 0.5;
  const double d = A.eps[i] - A.eps[A.nc + a];
  const double t = (f + r) * regularizer(d, A.s);
  A.t1[idx] = t;
  A.x1[idx] = f - 0.5 * d * t + 0.5 * r;
}

// z1 = Theta applied to the particle index a of tp
__host__ __device__ inline void mr_z1_elem(const MRArgs& A, long idx) {
  const int c = (int)(idx % A.na);
  const int a = (int)((idx / A.na) % A.np);
  const long lk = idx / ((long)A.na * A.np);
  const double* t = A.tp + lk * A.np * A.na;
  double z;
  if (a >= A.na) {
    z = 2.0 * t[(long)a * A.na + c];
  } else {
    z = 0.0;
    for (int d = 0; d < A.na; ++d) z = fma(mr_th(A, d, a), t[(long)d * A.na + c], z);
  }
  A.z1[idx] = z;
}

// tpp = Theta applied to the active index of z1
__host__ __device__ inline void mr_tpp_elem(const MRArgs& A, long idx) {
  const int y = (int)(idx % A.na);
  const long row = idx - y;
  double z = 0.0;
  for (int c = 0; c < A.na; ++c) z = fma(mr_th(A, y, c), A.z1[row + c], z);
  A.tpp[idx] = z;
}

// sum_k Gamma_{jk} F(k) over the holes: 2 F(j) for a core j, Gamma1 on the active ones
#define MR_GAMMA_SUM(A, j, EXPR_OF_K, out)                                  \
  do {                                                                      \
    if ((j) < (A).nc) {                                                     \
      const int k = (j);                                                    \
      out = 2.0 * (EXPR_OF_K);                                              \
    } else {                                                                \
      double acc_ = 0.0;                                                    \
      for (int kk_ = 0; kk_ < (A).na; ++kk_) {                              \
        const int k = (A).nc + kk_;                                         \
        acc_ = fma((A).g1[((j) - (A).nc) * (A).na + kk_], (EXPR_OF_K), acc_); \
      }                                                                     \
      out = acc_;                                                           \
    }                                                                       \
  } while (0)

// z2 [l'][j][a][c] and z3 [j][k'][a][c] (both na nh np na elements)
__host__ __device__ inline void mr_z23_elem(const MRArgs& A, long idx) {
  const int c = (int)(idx % A.na);
  const int a = (int)((idx / A.na) % A.np);
  {
    const int j = (int)((idx / ((long)A.na * A.np)) % A.nh);
    const int l = A.nc + (int)(idx / ((long)A.na * A.np * A.nh));
    double z;
    MR_GAMMA_SUM(A, j, A.z1[mr_at(A, l, k, a, c)], z);
    A.z2[idx] = z;
  }
  {
    const int kp = A.nc + (int)((idx / ((long)A.na * A.np)) % A.na);
    const int j = (int)(idx / ((long)A.na * A.np * A.na));
    double z;
    MR_GAMMA_SUM(A, j, A.z1[mr_at(A, k, kp, a, c)], z);
    A.z3[idx] = z;
  }
}

// g2t [i][j][c][d] (nh nh na na elements)
__host__ __device__ inline void mr_g2t_elem(const MRArgs& A, long idx) {
  const int d = (int)(idx % A.na);
  const int c = (int)((idx / A.na) % A.na);
  const int j = (int)((idx / ((long)A.na * A.na)) % A.nh);
  const int i = (int)(idx / ((long)A.na * A.na * A.nh));
  // sum_l Gamma_{il} [ sum_k Gamma_{jk} tp[k][l][c][d] ]
  double out;
  if (i < A.nc) {
    const int l = i;
    MR_GAMMA_SUM(A, j, A.tp[mr_at(A, k, l, c, d)], out);
    out *= 2.0;
  } else {
    out = 0.0;
    for (int ll = 0; ll < A.na; ++ll) {
      const int l = A.nc + ll;
      double inner;
      MR_GAMMA_SUM(A, j, A.tp[mr_at(A, k, l, c, d)], inner);
      out = fma(A.g1[(i - A.nc) * A.na + ll], inner, out);
    }
  }
  A.g2t[idx] = out;
}

// w3 [j][l'][c][d] (nh na na na elements)
__host__ __device__ inline void mr_w3_elem(const MRArgs& A, long idx) {
  const int d = (int)(idx % A.na);
  const int c = (int)((idx / A.na) % A.na);
  const int l = A.nc + (int)((idx / ((long)A.na * A.na)) % A.na);
  const int j = (int)(idx / ((long)A.na * A.na * A.na));
  double out;
  MR_GAMMA_SUM(A, j, A.tp[mr_at(A, k, l, c, d)], out);
  A.w3[idx] = out;
}

// tt1 [k][a] (nh np elements) and gt1 [j][c] (nh na elements, idx < nh na)
__host__ __device__ inline void mr_t1img_elem(const MRArgs& A, long idx) {
  const int a = (int)(idx % A.np);
  const int k = (int)(idx / A.np);
  double z;
  if (a >= A.na) {
    z = 2.0 * A.t1[idx];
  } else {
    z = 0.0;
    for (int c = 0; c < A.na; ++c) z = fma(A.t1[(long)k * A.np + c], mr_th(A, c, a), z);
  }
  A.tt1[idx] = z;
  if (idx < (long)A.nh * A.na) {
    const int c = (int)(idx % A.na);
    const int j = (int)(idx / A.na);
    double g;
    MR_GAMMA_SUM(A, j, A.t1[(long)k * A.np + c], g);
    A.gt1[idx] = g;
  }
}

// X2 element times its image Y (every term of <[X2, T1 + T2]> that is not E_vv).
__host__ __device__ inline double mr_energy_elem(const MRArgs& A, long idx) {
  const double x = A.xp[idx];
  if (x == 0.0) return 0.0;
  const int y = (int)(idx % A.na);
  const int a = (int)((idx / A.na) % A.np);
  const int j = (int)((idx / ((long)A.na * A.np)) % A.nh);
  const int i = (int)(idx / ((long)A.na * A.np * A.nh));
  const int nc = A.nc, na = A.na;
  // doubles with two Gamma or one 2-cumulant over the holes and Theta on both
  // particles: 1/8 w_a sum_{kl} Gamma2_H[i][j][k][l] tpp[k][l][a][y]
  // (w_a = 2 for a virtual: the av block mirrors the va one)
  double yp;
  if (i < nc && j < nc) {
    yp = 4.0 * A.tpp[mr_at(A, i, j, a, y)] - 2.0 * A.tpp[mr_at(A, j, i, a, y)];
  } else if (i < nc) {
    const int u = j - nc;
    yp = 0.0;
    for (int v = 0; v < na; ++v)
      yp = fma(A.g1[u * na + v], 2.0 * A.tpp[mr_at(A, i, nc + v, a, y)] - A.tpp[mr_at(A, nc + v, i, a, y)], yp);
  } else if (j < nc) {
    const int u = i - nc;
    yp = 0.0;
    for (int v = 0; v < na; ++v)
      yp = fma(A.g1[u * na + v], 2.0 * A.tpp[mr_at(A, nc + v, j, a, y)] - A.tpp[mr_at(A, j, nc + v, a, y)], yp);
  } else {
    const int u = i - nc, v = j - nc;
    yp = 0.0;
    for (int p = 0; p < na; ++p)
      for (int q = 0; q < na; ++q) {
        const double g2 = mr_L2(A, u, v, p, q) + A.g1[u * na + p] * A.g1[v * na + q] -
                          0.5 * A.g1[v * na + p] * A.g1[u * na + q];
        yp = fma(g2, A.tpp[mr_at(A, nc + p, nc + q, a, y)], yp);
      }
  }
  double Y = 0.125 * (a < na ? 1.0 : 2.0) * yp;
  const long n_apc = (long)A.np * na;  // stride of one (.., .) pair in z2 / z3
  if (i >= nc) {  // one 2-cumulant with the active hole i of X
    const int u = i - nc;
    double s4 = 0.0, s5 = 0.0;
    for (int c = 0; c < na; ++c)
      for (int w = 0; w < na; ++w) {
        s4 = fma(mr_L2(A, u, c, w, y), A.z2[((long)w * A.nh + j) * n_apc + (long)a * na + c], s4);
        s5 = fma(mr_L2(A, u, c, y, w), A.z3[((long)j * na + w) * n_apc + (long)a * na + c], s5);
      }
    Y -= 0.25 * (s4 + s5);
  }
  if (j >= nc) {  // the same terms through the pair transpose of X
    const int u = j - nc;
    double s6 = 0.0, s7 = 0.0;
    for (int c = 0; c < na; ++c)
      for (int w = 0; w < na; ++w) {
        const double l = mr_L2(A, u, c, y, w);
        s6 = fma(l, A.z2[((long)w * A.nh + i) * n_apc + (long)a * na + c], s6);
        s7 = fma(l, A.z3[((long)i * na + w) * n_apc + (long)a * na + c], s7);
      }
    Y += -0.25 * s6 + 0.5 * s7;
  }
  if (a < na) {  // both particles of X active, 2-cumulant over the particles
    double s8 = 0.0;
    for (int c = 0; c < na; ++c)
      for (int d = 0; d < na; ++d)
        s8 = fma(mr_L2(A, c, d, y, a), A.g2t[(((long)i * A.nh + j) * na + c) * na + d], s8);
    Y += 0.125 * s8;
  }
  if (i >= nc && j >= nc) {  // singles: 1/2 sum Lambda^{ij}_{kb} (t1 Theta)[k][a]
    double s = 0.0;
    for (int k = 0; k < na; ++k) s = fma(mr_L2(A, i - nc, j - nc, k, y), A.tt1[(long)(nc + k) * A.np + a], s);
    Y += 0.5 * s;
  }
  if (i >= nc && a < na) {  // singles: -1/2 sum Lambda^{ic}_{ab} (Gamma t1)[j][c]
    double s = 0.0;
    for (int c = 0; c < na; ++c) s = fma(mr_L2(A, i - nc, c, a, y), A.gt1[(long)j * na + c], s);
    Y -= 0.5 * s;
  }
  if (A.l3) {  // one 3-cumulant
    if (i >= nc && j >= nc) {
      double s = 0.0;
      for (int c = 0; c < na; ++c)
        for (int l = 0; l < na; ++l)
          for (int k = 0; k < na; ++k)
            s = fma(mr_L3(A, i - nc, j - nc, c, l, y, k), A.z1[mr_at(A, nc + l, nc + k, a, c)], s);
      Y += 0.5 * s;
    }
    if (i >= nc && a < na) {
      double s = 0.0;
      for (int c = 0; c < na; ++c)
        for (int d = 0; d < na; ++d)
          for (int l = 0; l < na; ++l)
            s = fma(mr_L3(A, i - nc, c, d, a, y, l), A.w3[(((long)j * na + l) * na + c) * na + d], s);
      Y -= 0.5 * s;
    }
  }
  return x * Y;
}

// X1 element times its image (<[X1, T1 + T2]>).
__host__ __device__ inline double mr_energy1_elem(const MRArgs& A, long idx) {
  const double x = A.x1[idx];
  if (x == 0.0) return 0.0;
  const int a = (int)(idx % A.np);
  const int i = (int)(idx / A.np);
  const int nc = A.nc, na = A.na;
  double Y;
  MR_GAMMA_SUM(A, i, A.tt1[(long)k * A.np + a], Y);
  Y *= 0.5;
  if (i >= nc) {
    double s = 0.0;
    for (int c = 0; c < na; ++c)
      for (int l = 0; l < na; ++l)
        for (int k = 0; k < na; ++k)
          s = fma(mr_L2(A, i - nc, c, l, k), A.z1[mr_at(A, nc + l, nc + k, a, c)], s);
    Y += 0.5 * s;
  }
  if (a < na) {
    double s = 0.0;
    for (int c = 0; c < na; ++c)
      for (int d = 0; d < na; ++d)
        for (int l = 0; l < na; ++l)
          s = fma(mr_L2(A, c, d, a, l), A.w3[(((long)i * na + l) * na + c) * na + d], s);
    Y -= 0.5 * s;
  }
  return x * Y;
}

}  // namespace dsrg
