// Semi-internal and singles contributions to D_vv (Eq. A12 terms 1-3, 6, 8-12,
// and term 13 when a 3-cumulant is given) and the singles amplitudes of
// Eq. A6, float64.
//
// Every term is written as D_ef += coef * sum_k X[e][k] Y[f][k]: a builder
// kernel contracts the amplitudes with the active-space densities into X and
// gathers Y, and a GEMM accumulates X Y^T into D.
//
// Amplitude layout: ts[((i*nh + j)*nv + e)*na + x] = t^{ij}_{ex} (e virtual,
// x active particle) for every ordered hole pair; t1[i*nv + e] = t^i_e.
// Term 11 carries tcheck on its second amplitude: evaluating Eq. A11 in a
// determinant space requires it (the printed form has a plain t there).
#include "kernels.h"

namespace dsrg {

namespace {

struct SI {
  int nc, na, nv, nh;
  const double* ts;
  const double* t1;
  const double* g1;  // [na][na]
  const double* l2;  // [na]^4
  // partial contractions shared by the builders (theta_kernel, lambda_kernel):
  const double* qaa;  // [u][v][e][w] = sum_z t^{uv}_{ez} Theta^w_z
  const double* pa;   // [m][u][e][x] = sum_y t^{mu}_{ey} Theta^x_y
  const double* pb;   // [m][u][e][x] = sum_y t^{um}_{ey} Theta^x_y
  const double* pla;  // [w][e][x][u] = sum_{vy} t^{wv}_{ey} Lambda^{uv}_{xy}
  const double* plb;  // [w][e][x][u] = sum_{vy} t^{vw}_{ey} Lambda^{uv}_{xy}
  const double* plc;  // [w][e][y][u] = sum_{vx} t^{vw}_{ex} Lambda^{uv}_{xy}
  const double* l3;   // [na]^6 Lambda^{xyz}_{uvw} (term 13), or null
  __device__ double t(int i, int j, int e, int x) const {
    return ts[(((long)i * nh + j) * nv + e) * na + x];
  }
  __device__ double G(int u, int v) const { return g1[u * na + v]; }
  __device__ double Th(int u, int v) const { return (u == v ? 2.0 : 0.0) - g1[u * na + v]; }
  __device__ double L(int u, int v, int x, int y) const { return l2[((u * na + v) * na + x) * na + y]; }
};

// Eq. A6 with the off-diagonal Fock f^i_a (may be null):
// t^i_e = [f^i_e + 1/2 sum_{ux} (eps_x - eps_u) Gamma^x_u tcheck^{iu}_{ex}] R(eps_i - eps_e)
__global__ void t1_kernel(SI S, Geometry g, const double* __restrict__ eps, const double* __restrict__ f_hp,
                          double* __restrict__ t1) {
  long idx = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (idx >= (long)S.nh * S.nv) return;
  const int i = (int)(idx / S.nv), e = (int)(idx % S.nv);
  double f = f_hp ? f_hp[(long)i * g.np + g.na + e] : 0.0;
  double c = 0.0;
  for (int u = 0; u < S.na; ++u) {
    const double eu = eps[S.nc + u];
    for (int x = 0; x < S.na; ++x) {
      const double ex = eps[S.nc + x];
      const double tch = 2.0 * S.t(i, S.nc + u, e, x) - S.t(S.nc + u, i, e, x);
      c = fma((ex - eu) * S.G(x, u), tch, c);
    }
  }
  const double d = eps[i] - eps[S.nc + S.na + e];
  t1[idx] = (f + 0.5 * c) * regularizer(d, g.s);
}

// qaa / pa / pb: out[p][e][w] = sum_z t(i_p, j_p, e, z) Theta^w_z over the hole
// pairs p of one family: 0 = (nc+u, nc+v), p = u na + v; 1 = (m, nc+u) and
// 2 = (nc+u, m), p = m na + u.
__global__ void theta_kernel(SI S, int family, long npairs, double* __restrict__ out) {
  const long idx = blockIdx.x * (long)blockDim.x + threadIdx.x;
  const int na = S.na, nv = S.nv, nc = S.nc;
  if (idx >= npairs * nv * na) return;
  const int w = (int)(idx % na);
  const int e = (int)((idx / na) % nv);
  const long p = idx / ((long)na * nv);
  const int a = (int)(p / na), b = (int)(p % na);
  int i, j;
  if (family == 0) {
    i = nc + a;
    j = nc + b;
  } else if (family == 1) {
    i = a;
    j = nc + b;
  } else {
    i = nc + b;
    j = a;
  }
  double acc = 0.0;
  for (int z = 0; z < na; ++z) acc = fma(S.t(i, j, e, z), S.Th(w, z), acc);
  out[idx] = acc;
}

// pla / plb / plc: out[w][e][x][u] = sum_{v,y} t(., ., e, .) Lambda^{uv}_{..}
// variant 0: t^{wv}_{ey} L^{uv}_{xy}; 1: t^{vw}_{ey} L^{uv}_{xy}; 2: t^{vw}_{ex} L^{uv}_{xy}
// (variant 2 indexes its output [w][e][y][u]).
__global__ void lambda_kernel(SI S, int variant, double* __restrict__ out) {
  const long idx = blockIdx.x * (long)blockDim.x + threadIdx.x;
  const int na = S.na, nv = S.nv, nc = S.nc;
  if (idx >= (long)na * nv * na * na) return;
  const int u = (int)(idx % na);
  const int q = (int)((idx / na) % na);  // x (variants 0, 1) or y (variant 2)
  const int e = (int)((idx / ((long)na * na)) % nv);
  const int w = (int)(idx / ((long)na * na * nv));
  double acc = 0.0;
  for (int v = 0; v < na; ++v)
    for (int r = 0; r < na; ++r) {
      if (variant == 0) acc = fma(S.t(nc + w, nc + v, e, r), S.L(u, v, q, r), acc);
      else if (variant == 1) acc = fma(S.t(nc + v, nc + w, e, r), S.L(u, v, q, r), acc);
      else acc = fma(S.t(nc + v, nc + w, e, r), S.L(u, v, r, q), acc);
    }
  out[idx] = acc;
}

enum TermId {
  T1_CORE = 0, T2_ACT, T3_A, T3_B, T6, T8_A, T8_B, T9_A, T9_B, T9_C, T10, T11, T12_A, T12_B, T12_C, T13,
  NTERMS
};

__device__ __forceinline__ void unflat3(int k, int n1, int n2, int* a, int* b, int* c) {
  *c = k % n2;
  k /= n2;
  *b = k % n1;
  *a = k / n1;
}

// X[e][k], Y[e][k] for one term (rows e, K contiguous)
__global__ void build_kernel(SI S, int term, int K, double* __restrict__ X, double* __restrict__ Y) {
  long idx = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (idx >= (long)S.nv * K) return;
  const int e = (int)(idx / K), k = (int)(idx % K);
  const int nc = S.nc, na = S.na;
  double x = 0.0, y = 0.0;
  switch (term) {
    case T1_CORE: {  // 2 t^m_e t^m_f
      x = S.t1[(long)k * S.nv + e];
      y = x;
      break;
    }
    case T2_ACT: {  // t^u_e t^v_f Gamma^u_v ; k = v
      for (int u = 0; u < na; ++u) x = fma(S.t1[(long)(nc + u) * S.nv + e], S.G(u, k), x);
      y = S.t1[(long)(nc + k) * S.nv + e];
      break;
    }
    case T3_A:    // t^u_e Z[f][u],  Z[f][u] = sum_{vxy} t^{xy}_{fv} Lambda^{uv}_{xy} ; k = u
    case T3_B: {  // Z'[e][x] t^x_f, Z'[e][x] = sum_{uvy} t^{uv}_{ey} Lambda^{uv}_{xy} ; k = x
      double t1v = S.t1[(long)(nc + k) * S.nv + e];
      double z = 0.0;
      if (term == T3_A) {
        for (int v = 0; v < na; ++v)
          for (int xx = 0; xx < na; ++xx)
            for (int yy = 0; yy < na; ++yy) z = fma(S.t(nc + xx, nc + yy, e, v), S.L(k, v, xx, yy), z);
        x = t1v;
        y = z;
      } else {
        for (int u = 0; u < na; ++u)
          for (int v = 0; v < na; ++v)
            for (int yy = 0; yy < na; ++yy) z = fma(S.t(nc + u, nc + v, e, yy), S.L(u, v, k, yy), z);
        x = z;
        y = t1v;
      }
      break;
    }
    case T6: {  // t^{mn}_{ev} tcheck^{mn}_{fu} Theta^u_v ; k = (m, n, u)
      int m, n, u;
      unflat3(k, nc, na, &m, &n, &u);
      for (int v = 0; v < na; ++v) x = fma(S.t(m, n, e, v), S.Th(u, v), x);
      y = 2.0 * S.t(m, n, e, u) - S.t(n, m, e, u);
      break;
    }
    case T8_A:    // t^{mu}_{ey} tcheck^{mv}_{fx} Gamma^u_v Theta^x_y ; k = (m, v, x)
    case T8_B: {  // t^{um}_{ey} tcheck^{vm}_{fx} Gamma^u_v Theta^x_y
      int m, v, xx;
      unflat3(k, na, na, &m, &v, &xx);
      const double* P = term == T8_A ? S.pa : S.pb;
      for (int u = 0; u < na; ++u) x = fma(S.G(u, v), P[(((long)m * na + u) * S.nv + e) * na + xx], x);
      y = term == T8_A ? 2.0 * S.t(m, nc + v, e, xx) - S.t(nc + v, m, e, xx)
                       : 2.0 * S.t(nc + v, m, e, xx) - S.t(m, nc + v, e, xx);
      break;
    }
    case T9_A:    // t^{mv}_{ey} (2 t^{mx}_{fu} - t^{xm}_{fu}) Lambda^{uv}_{xy} ; k = (m, x, u)
    case T9_B: {  // -t^{vm}_{ey} t^{mx}_{fu} Lambda^{uv}_{xy}
      int m, xx, u;
      unflat3(k, na, na, &m, &xx, &u);
      for (int v = 0; v < na; ++v)
        for (int yy = 0; yy < na; ++yy) {
          double tt = term == T9_A ? S.t(m, nc + v, e, yy) : S.t(nc + v, m, e, yy);
          x = fma(tt, S.L(u, v, xx, yy), x);
        }
      y = term == T9_A ? 2.0 * S.t(m, nc + xx, e, u) - S.t(nc + xx, m, e, u) : S.t(m, nc + xx, e, u);
      break;
    }
    case T9_C: {  // -t^{vm}_{ex} t^{ym}_{fu} Lambda^{uv}_{xy} ; k = (m, y, u)
      int m, yy, u;
      unflat3(k, na, na, &m, &yy, &u);
      for (int v = 0; v < na; ++v)
        for (int xx = 0; xx < na; ++xx) x = fma(S.t(nc + v, m, e, xx), S.L(u, v, xx, yy), x);
      y = S.t(nc + yy, m, e, u);
      break;
    }
    case T10: {  // t^{uv}_{ez} t^{xy}_{fw} Theta^w_z Lambda^{uv}_{xy} ; k = (x, y, w)
      int xx, yy, w;
      unflat3(k, na, na, &xx, &yy, &w);
      for (int u = 0; u < na; ++u)
        for (int v = 0; v < na; ++v)
          x = fma(S.qaa[(((long)u * na + v) * S.nv + e) * na + w], S.L(u, v, xx, yy), x);
      y = S.t(nc + xx, nc + yy, e, w);
      break;
    }
    case T11: {  // t^{ux}_{ez} tcheck^{vy}_{fw} Gamma^u_v Gamma^x_y Theta^w_z ; k = (v, y, w)
      int v, yy, w;
      unflat3(k, na, na, &v, &yy, &w);
      for (int u = 0; u < na; ++u) {
        double a = 0.0;
        for (int xx = 0; xx < na; ++xx) a = fma(S.G(xx, yy), S.qaa[(((long)u * na + xx) * S.nv + e) * na + w], a);
        x = fma(S.G(u, v), a, x);
      }
      y = 2.0 * S.t(nc + v, nc + yy, e, w) - S.t(nc + yy, nc + v, e, w);
      break;
    }
    case T12_A:    // t^{wv}_{ey} (2 t^{zx}_{fu} - t^{xz}_{fu}) Gamma^w_z Lambda^{uv}_{xy} ; k = (z, x, u)
    case T12_B: {  // -t^{vw}_{ey} t^{zx}_{fu} Gamma^w_z Lambda^{uv}_{xy}
      int z, xx, u;
      unflat3(k, na, na, &z, &xx, &u);
      const double* P = term == T12_A ? S.pla : S.plb;
      for (int w = 0; w < na; ++w) x = fma(S.G(w, z), P[(((long)w * S.nv + e) * na + xx) * na + u], x);
      y = term == T12_A ? 2.0 * S.t(nc + z, nc + xx, e, u) - S.t(nc + xx, nc + z, e, u)
                        : S.t(nc + z, nc + xx, e, u);
      break;
    }
    case T12_C: {  // -t^{vw}_{ex} t^{yz}_{fu} Gamma^w_z Lambda^{uv}_{xy} ; k = (y, z, u)
      int yy, z, u;
      unflat3(k, na, na, &yy, &z, &u);
      for (int w = 0; w < na; ++w) x = fma(S.G(w, z), S.plc[(((long)w * S.nv + e) * na + yy) * na + u], x);
      y = S.t(nc + yy, nc + z, e, u);
      break;
    }
    case T13: {  // t^{uw}_{ez} t^{xy}_{fv} Lambda^{xyz}_{uvw} ; k = (z, u, w)
      int z, u, w;
      unflat3(k, na, na, &z, &u, &w);
      x = S.t(nc + u, nc + w, e, z);
      const long n2 = (long)na * na, n3 = n2 * na;
      // Lambda^{xyz}_{uvw} at ((((x na + y) na + z) na + u) na + v) na + w
      const double* l = S.l3 + ((long)z * na + u) * n2 + w;
      for (int xx = 0; xx < na; ++xx)
        for (int yy = 0; yy < na; ++yy) {
          const double* lxy = l + ((long)xx * na + yy) * n3 * na;
          for (int v = 0; v < na; ++v) y = fma(S.t(nc + xx, nc + yy, e, v), lxy[(long)v * na], y);
        }
      break;
    }
  }
  X[idx] = x;
  Y[idx] = y;
}

}  // namespace

// K-dimension and coefficient of every term part
static void term_shape(int term, int nc, int na, int* K, double* coef) {
  switch (term) {
    case T1_CORE: *K = nc; *coef = 2.0; break;
    case T2_ACT: *K = na; *coef = 1.0; break;
    case T3_A: case T3_B: *K = na; *coef = 1.0; break;
    case T6: *K = nc * nc * na; *coef = 1.0; break;
    case T8_A: case T8_B: *K = nc * na * na; *coef = 0.5; break;
    case T9_A: *K = nc * na * na; *coef = 1.0; break;
    case T9_B: case T9_C: *K = nc * na * na; *coef = -1.0; break;
    case T10: *K = na * na * na; *coef = 0.5; break;
    case T11: *K = na * na * na; *coef = 0.25; break;
    case T12_A: *K = na * na * na; *coef = 0.5; break;
    case T12_B: case T12_C: *K = na * na * na; *coef = -0.5; break;
    case T13: *K = na * na * na; *coef = 1.0; break;
    default: *K = 0; *coef = 0.0;
  }
}

// partial contractions: qaa na^3 nv, pa and pb nc na^2 nv each, pla/plb/plc na^3 nv each
static size_t partials_doubles(int nc, int na, int nv) {
  return (size_t)nv * na * na * (4 * (size_t)na + 2 * (size_t)nc);
}

size_t small_terms_work_doubles(int nc, int na, int nv) {
  long kmax = 0;
  for (int t = 0; t < NTERMS; ++t) {
    int K;
    double c;
    term_shape(t, nc, na, &K, &c);
    kmax = K > kmax ? K : kmax;
  }
  return 2 * (size_t)nv * (size_t)kmax + partials_doubles(nc, na, nv);
}

int t1_amplitudes(const Geometry& g, const double* ts, const double* eps, const double* f_hp, const double* g1,
                  double* t1, cudaStream_t st) {
  SI S{g.nc, g.na, g.nv, g.nh, ts, nullptr, g1, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr,
       nullptr};
  long n = (long)g.nh * g.nv;
  if (n == 0) return DSRG_FNO_OK;
  t1_kernel<<<ceil_div(n, 256), 256, 0, st>>>(S, g, eps, f_hp, t1);
  DSRG_LAUNCH_CHECK();
  return DSRG_FNO_OK;
}

__global__ void axpy_kernel(long n, double a, const double* __restrict__ x, double* __restrict__ y) {
  long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (i < n) y[i] = fma(a, x[i], y[i]);
}

// Largest K of any term part (the contraction length of its GEMM).
int small_terms_kmax(int nc, int na) {
  int kmax = 0;
  for (int t = 0; t < NTERMS; ++t) {
    int K;
    double c;
    term_shape(t, nc, na, &K, &c);
    kmax = K > kmax ? K : kmax;
  }
  return kmax;
}

// D += terms 1-3, 6, 8-12, and term 13 when l3 is not null.  work:
// small_terms_work_doubles() doubles.  With F.ks > 0, the GEMMs with
// K >= SLICED_MIN_K run on the tensor cores (digit planes of X and Y, exact
// level sums), the rest in float64.
int small_terms_f64(const Geometry& g, const double* ts, const double* t1, const double* g1, const double* l2,
                    const double* l3, double* D, double* work, const SmallFast& F, cudaStream_t st) {
  SI S{g.nc, g.na, g.nv, g.nh, ts, t1, g1, l2, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, l3};
  if (g.na > 0) {
    // partial contractions after the X / Y area of the largest term
    const int kmax = small_terms_kmax(g.nc, g.na);
    double* q = work + 2 * (size_t)g.nv * kmax;
    const long na = g.na, nv = g.nv, nc = g.nc;
    double* qaa = q;
    double* pa = qaa + na * na * nv * na;
    double* pb = pa + nc * na * nv * na;
    double* pla = pb + nc * na * nv * na;
    double* plb = pla + na * nv * na * na;
    double* plc = plb + na * nv * na * na;
    const long nq = na * na * nv * na, np_ = nc * na * nv * na, nl = na * nv * na * na;
    theta_kernel<<<ceil_div(nq, 256), 256, 0, st>>>(S, 0, na * na, qaa);
    DSRG_LAUNCH_CHECK();
    if (np_ > 0) {
      theta_kernel<<<ceil_div(np_, 256), 256, 0, st>>>(S, 1, nc * na, pa);
      DSRG_LAUNCH_CHECK();
      theta_kernel<<<ceil_div(np_, 256), 256, 0, st>>>(S, 2, nc * na, pb);
      DSRG_LAUNCH_CHECK();
    }
    for (int v = 0; v < 3; ++v) {
      lambda_kernel<<<ceil_div(nl, 256), 256, 0, st>>>(S, v, v == 0 ? pla : (v == 1 ? plb : plc));
      DSRG_LAUNCH_CHECK();
    }
    S.qaa = qaa;
    S.pa = pa;
    S.pb = pb;
    S.pla = pla;
    S.plb = plb;
    S.plc = plc;
  }
  for (int term = 0; term < NTERMS; ++term) {
    if (g.na == 0 && term != T1_CORE) continue;
    if (term == T13 && !l3) continue;
    int K;
    double coef;
    term_shape(term, g.nc, g.na, &K, &coef);
    if (K == 0) continue;
    double* X = work;
    double* Y = work + (long)g.nv * K;
    long n = (long)g.nv * K;
    build_kernel<<<ceil_div(n, 256), 256, 0, st>>>(S, term, K, X, Y);
    DSRG_LAUNCH_CHECK();
    if (F.ks > 0 && K >= SLICED_MIN_K) {
      const int kp = pad64(K);
      __nv_bfloat16* px = F.planes;
      __nv_bfloat16* py = F.planes + (size_t)F.ks * g.nv * kp;
      DSRG_TRY(slice_rows(F.ks, X, g.nv, K, K, 1, kp, px, F.exps, st));
      DSRG_TRY(slice_rows(F.ks, Y, g.nv, K, K, 1, kp, py, F.exps + g.nv, st));
      DSRG_TRY(sliced_plain_gemm(F.ks, g.nv, g.nv, px, F.exps, py, F.exps + g.nv, kp, F.cbuf, g.nv, F.err, st));
      const long n2 = (long)g.nv * g.nv;
      axpy_kernel<<<ceil_div(n2, 256), 256, 0, st>>>(n2, coef, F.cbuf, D);
      DSRG_LAUNCH_CHECK();
    } else {
      DSRG_TRY(gemm_f64(g.nv, g.nv, K, coef, X, K, true, Y, K, true, 1.0, D, g.nv, 1, 0, 0, 0, st));
    }
  }
  return DSRG_FNO_OK;
}

}  // namespace dsrg
