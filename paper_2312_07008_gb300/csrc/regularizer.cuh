// The Eq. A7 regulariser in double-float arithmetic, shared by the
// elementwise epilogue kernel and the fused epilogue of the contraction
// kernel.
//
// With x = s Delta^2 >= 0, y = exp(-x):
//   tau = nu (1 - y) / Delta,  kappa = 2 nu - Delta tau = nu (1 + y).
// exp(-x) follows the table method of Tang (ACM TOMS 15, 1989): t = x log2(e)
// = n/64 + r with |r| <= 1/128, u = r ln 2, exp(-x) = 2^-q 2^-j/64 exp(-u),
// n = 64 q + j, and exp(-u) from its Taylor series (to the cubic term in
// double-float).  1 - y is formed without cancellation: with C_j = 1 -
// 2^-j/64 and 1 - exp(-u) = u - u^2/2 + ...,
//   1 - y = C_j + (1 - e^-u) - C_j (1 - e^-u)     (q = 0),
// so that the small-Delta branch of Eq. A7 (R -> s Delta) keeps its relative
// accuracy without a separate series.  For x > 40, y < 5e-18 is dropped.
#pragma once
#include "dd.cuh"

namespace dsrg {

struct RegTables {
  dd T[64];  // 2^-j/64
  dd C[64];  // 1 - 2^-j/64
  dd log2e, ln2, sixth;
};

// R1 = (1 - exp(-s Delta^2)) / Delta and y = exp(-s Delta^2), double-float.
__device__ __forceinline__ void regularize(dd delta, dd s, const RegTables& R, dd* r1, dd* y) {
  if (delta.hi == 0.0f) {
    *r1 = dd_make(0.0f);
    *y = dd_make(1.0f);
    return;
  }
  const dd x = dd_mul(s, dd_mul(delta, delta));
  if (x.hi < 1e-20f) {  // R1 = s Delta (1 - x/2 + ...), y = 1 - x: the x terms are below the precision
    *r1 = dd_mul(s, delta);
    *y = dd_make(1.0f);
    return;
  }
  if (x.hi > 40.0f) {
    *y = dd_make(0.0f);
    *r1 = dd_recip(delta);
    return;
  }
  const dd t = dd_mul(x, R.log2e);
  const int n = __float2int_rn(t.hi * 64.0f);
  const dd r = dd_sub(t, dd_make((float)n * 0.015625f));
  const dd u = dd_mul(r, R.ln2);
  const float uh = u.hi;
  // 1 - e^-u = u - u^2/2 + u^3/6 - (u^4/24 - u^5/120 + u^6/720)   (|u| <= 0.0055)
  // up to the cubic term in double-float; the rest (< 4e-11) in float
  const dd u2 = dd_mul(u, u);
  const dd c3 = dd_mul(dd_mul(u2, u), R.sixth);
  const float tail = uh * uh * uh * uh * (1.0f / 24.0f - uh * (1.0f / 120.0f - uh * (1.0f / 720.0f)));
  const dd omp = dd_add_f(dd_add_fast(dd_sub_fast(u, dd_mul_f(u2, 0.5f)), c3), -tail);
  const dd p = dd_sub_fast(dd_make(1.0f), omp);
  const int q = n >> 6, j = n & 63;
  *y = dd_ldexp(dd_mul(R.T[j], p), -q);
  dd omy;
  if (q == 0) omy = dd_add_fast(R.C[j], dd_sub_fast(omp, dd_mul(R.C[j], omp)));
  else omy = dd_sub_fast(dd_make(1.0f), *y);
  *r1 = dd_mul(omy, dd_recip(delta));
}


}  // namespace dsrg
