// Staging of the fast form's operands: rows -> exact bfloat16 digit planes
// (and the literal split-bf16 / tf32 parts of the precision study).
//
// Each float64 row v[k] (k = contraction index) gets a power-of-two
// scale 2^e_row with max_k |v| < 2^e_row, and the scaled value x = v 2^-e_row
// is rounded to X = round(x 2^F), F = 7 + 8 (KS - 1), then written in balanced
// radix 256:  X = sum_s d_s 256^(KS-1-s),  d_s integer in [-128, 128], exact in
// bfloat16 (8 significant bits).  Hence x = 2^-7 sum_s d_s 2^-8s up to 2^-(F+1).
//
#include <type_traits>

#include "kernels.h"

namespace dsrg {

namespace {

// ---------------------------------------------------------------- staging
// Row exponent e with max |v| < 2^e (frexp exponent of the row maximum).
__device__ __forceinline__ int row_exponent(double maxabs) {
  long long b = __double_as_longlong(maxabs);
  int E = (int)((b >> 52) & 0x7FF);
  return E == 0 ? -1022 : E - 1022;
}

template <int KS>
__device__ __forceinline__ void digits_of(double v, int e_row, int* d) {
  constexpr int F = 7 + 8 * (KS - 1);
  long long b = __double_as_longlong(v);
  int E = (int)((b >> 52) & 0x7FF);
  long long X = 0;
  if (E != 0) {
    long long m = (b & 0xFFFFFFFFFFFFFLL) | (1LL << 52);
    int sh = 1075 - E - F + e_row;  // >= 53 - F >= 6 for KS <= 6 because |v| < 2^e_row
    if (sh < 63) X = (m + (1LL << (sh - 1))) >> sh;
    if (b < 0) X = -X;
  }
#pragma unroll
  for (int s = KS - 1; s >= 1; --s) {
    long long r = ((X + 128) & 255) - 128;
    d[s] = (int)r;
    X = (X - r) >> 8;
  }
  d[0] = (int)X;
}

// Digits of a double-float value hi + lo with the same rule: X = round((hi +
// lo) 2^(F - e_row)), formed exactly in 64-bit fixed point with 16 guard bits.
__device__ __forceinline__ long long fixed_of_float(float v, int e_row, int F, int G) {
  const int b = __float_as_int(v);
  const int E = (b >> 23) & 0xFF;
  if (E == 0) return 0;
  const long long m = (long long)((b & 0x7FFFFF) | 0x800000);
  // v = m 2^(E-150); scaled by 2^(F - e_row + G)
  const int sh = E - 150 + F - e_row + G;
  long long x;
  if (sh >= 0) x = sh < 39 ? (m << sh) : 0;  // sh < 39 always holds for |v| < 2^e_row
  else x = (-sh < 63) ? (m >> (-sh)) : 0;
  return b < 0 ? -x : x;
}

template <int KS>
__device__ __forceinline__ void digits_of(float2 v, int e_row, int* d) {
  constexpr int F = 7 + 8 * (KS - 1);
  constexpr int G = 16;
  long long Xg = fixed_of_float(v.x, e_row, F, G) + fixed_of_float(v.y, e_row, F, G);
  long long X = Xg >= 0 ? ((Xg + (1LL << (G - 1))) >> G) : -((-Xg + (1LL << (G - 1))) >> G);
#pragma unroll
  for (int s = KS - 1; s >= 1; --s) {
    long long r = ((X + 128) & 255) - 128;
    d[s] = (int)r;
    X = (X - r) >> 8;
  }
  d[0] = (int)X;
}

__device__ __forceinline__ double magnitude(double v) { return fabs(v); }
__device__ __forceinline__ double magnitude(float2 v) { return (double)fabsf(v.x); }
__device__ __forceinline__ int row_exponent_of(double mx, double) { return row_exponent(mx); }
__device__ __forceinline__ int row_exponent_of(double mx, float2) {
  // from the float hi parts: max |hi| < 2^e implies |hi + lo| < 2^e
  const int b = __float_as_int((float)mx);
  const int E = (b >> 23) & 0xFF;
  return E == 0 ? -126 : E - 126;
}
__device__ __forceinline__ double zero_of(double) { return 0.0; }
__device__ __forceinline__ float2 zero_of(float2) { return make_float2(0.f, 0.f); }

// planes[s][row][k] (bf16, k padded to Kpad with zeros), exps[row].
// Source element (row, k) at src[row * rs + k * ks]; one of rs, ks is 1.
// T is double (float64 rows) or float2 (double-float rows).
// rowmax (optional, double-float rows): max |hi| of each row as float bits,
// gathered by the producer; the first pass over the row is then skipped.
template <int KS, typename T>
__global__ void __launch_bounds__(256) slice_rows_kernel(const T* __restrict__ src, long R, int K, long rs,
                                                         long ks, int Kpad, __nv_bfloat16* __restrict__ planes,
                                                         int* __restrict__ exps, const unsigned* __restrict__ rowmax) {
  __shared__ T tile[32][33];
  __shared__ int s_exp[32];
  const long row0 = (long)blockIdx.x * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const bool kfast = (ks == 1);
  const int myrow = threadIdx.x >> 3, part = threadIdx.x & 7;  // 32 rows x 8 parts
  if (kfast) {
    // rows contiguous in k: the 8 threads of a row read it directly (4
    // consecutive elements each, 256 contiguous bytes of float2 per row and
    // step), no staging and no block barrier
    const long row = row0 + myrow;
    double m = 0.0;
    if (rowmax) {
      if (part == 0 && row < R) m = (double)__uint_as_float(rowmax[row]);
    } else if (row < R) {
      for (int k = part; k < K; k += 8) m = fmax(m, magnitude(src[row * rs + k]));
    }
#pragma unroll
    for (int o = 4; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (row >= R) return;
    const int e_row = row_exponent_of(m, T());
    if (part == 0) exps[row] = e_row;
    const T* p = src + row * rs;
#pragma unroll 2
    for (int k0 = part * 4; k0 < Kpad; k0 += 32) {
      T v[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) v[j] = (k0 + j < K) ? p[k0 + j] : zero_of(T());
      int dg[4][KS];
#pragma unroll
      for (int j = 0; j < 4; ++j) digits_of<KS>(v[j], e_row, dg[j]);
#pragma unroll
      for (int s = 0; s < KS; ++s) {
        __nv_bfloat16 h[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) h[j] = __float2bfloat16_rn((float)dg[j][s]);
        uint2 pk;
        pk.x = (uint32_t)__bfloat16_as_ushort(h[0]) | ((uint32_t)__bfloat16_as_ushort(h[1]) << 16);
        pk.y = (uint32_t)__bfloat16_as_ushort(h[2]) | ((uint32_t)__bfloat16_as_ushort(h[3]) << 16);
        *reinterpret_cast<uint2*>(planes + ((long)s * R + row) * Kpad + k0) = pk;
      }
    }
    return;
  }
  double mx = 0.0;
  if (rowmax) {
    if (part == 0 && row0 + myrow < R) mx = (double)__uint_as_float(rowmax[row0 + myrow]);
  }
  // rows strided in k (ks > 1): 32 x 32 tiles staged transposed
  for (int k0 = 0; k0 < K && !rowmax; k0 += 32) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      int r = tx;
      int k = ty + 8 * i;
      long row = row0 + r;
      T v = zero_of(T());
      if (row < R && k0 + k < K) v = src[row * rs + (long)(k0 + k) * ks];
      tile[r][k] = v;
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < 4; ++j) mx = fmax(mx, magnitude(tile[myrow][part * 4 + j]));
    __syncthreads();
  }
#pragma unroll
  for (int o = 4; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if (part == 0) {
    int e = row_exponent_of(mx, T());
    s_exp[myrow] = e;
    if (row0 + myrow < R) exps[row0 + myrow] = e;
  }
  __syncthreads();
  const int e_row = s_exp[myrow];
  const long row = row0 + myrow;
  for (int k0 = 0; k0 < Kpad; k0 += 32) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      int r = tx;
      int k = ty + 8 * i;
      long rr = row0 + r;
      T v = zero_of(T());
      if (rr < R && k0 + k < K) v = src[rr * rs + (long)(k0 + k) * ks];
      tile[r][k] = v;
    }
    __syncthreads();
    if (row < R) {
      int dg[4][KS];
#pragma unroll
      for (int j = 0; j < 4; ++j) digits_of<KS>(tile[myrow][part * 4 + j], e_row, dg[j]);
#pragma unroll
      for (int s = 0; s < KS; ++s) {
        __nv_bfloat16 h[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) h[j] = __float2bfloat16_rn((float)dg[j][s]);
        uint2 pk;
        pk.x = (uint32_t)__bfloat16_as_ushort(h[0]) | ((uint32_t)__bfloat16_as_ushort(h[1]) << 16);
        pk.y = (uint32_t)__bfloat16_as_ushort(h[2]) | ((uint32_t)__bfloat16_as_ushort(h[3]) << 16);
        *reinterpret_cast<uint2*>(planes + ((long)s * R + row) * Kpad + k0 + part * 4) = pk;
      }
    }
    __syncthreads();
  }
}

// tf32 value of x (round to nearest, ties away from zero): 10 fraction bits
// kept, the low 13 bits of the float32 container zero
__device__ __forceinline__ float tf32_round(float x) {
  return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);
}

// Parts of a literal form: planes[s][row][k] (k padded with zeros to Kpad),
// exps[row] = 0.  Source element (row, k) at src[row * rs + k * ks].
template <int FORM, int KS>
__global__ void __launch_bounds__(256) split_rows_kernel(const double* __restrict__ src, long R, int K, long rs,
                                                         long ks, int Kpad, void* __restrict__ planes,
                                                         int* __restrict__ exps) {
  __shared__ double tile[32][33];
  const long row0 = (long)blockIdx.x * 32;
  const int k0 = blockIdx.y * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const bool kfast = (ks == 1);
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int r = kfast ? ty + 8 * i : tx;
    const int k = kfast ? tx : ty + 8 * i;
    const long row = row0 + r;
    tile[r][k] = (row < R && k0 + k < K) ? src[row * rs + (long)(k0 + k) * ks] : 0.0;
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int r = ty + 8 * i;
    const long row = row0 + r;
    if (row >= R) continue;
    const double v = tile[r][tx];
    const long o = row * Kpad + k0 + tx;
    if constexpr (FORM == FORM_BF16X3) {
      __nv_bfloat16* pl = reinterpret_cast<__nv_bfloat16*>(planes);
      const __nv_bfloat16 hi = __double2bfloat16(v);
      pl[o] = hi;
      pl[R * Kpad + o] = __double2bfloat16(v - (double)__bfloat162float(hi));
    } else {
      float* pl = reinterpret_cast<float*>(planes);
      const float big = tf32_round((float)v);
      pl[o] = big;
      if (KS == 2) pl[R * Kpad + o] = tf32_round((float)(v - (double)big));
    }
  }
  if (blockIdx.y == 0 && threadIdx.x < 32 && row0 + threadIdx.x < R) exps[row0 + threadIdx.x] = 0;
}

}  // namespace

template <typename T>
static int slice_rows_t(int KS, const T* src, long R, int K, long rs, long ks, int Kpad, __nv_bfloat16* planes,
                        int* exps, const unsigned* rowmax, cudaStream_t st) {
  if (R <= 0) return DSRG_FNO_OK;
  if (Kpad % 32 != 0 || Kpad < K) return DSRG_FNO_ERR_ARG;  // rows are written in steps of 32
  const int grid = (int)((R + 31) / 32);
  switch (KS) {
    case 3: slice_rows_kernel<3, T><<<grid, 256, 0, st>>>(src, R, K, rs, ks, Kpad, planes, exps, rowmax); break;
    case 4: slice_rows_kernel<4, T><<<grid, 256, 0, st>>>(src, R, K, rs, ks, Kpad, planes, exps, rowmax); break;
    case 5: slice_rows_kernel<5, T><<<grid, 256, 0, st>>>(src, R, K, rs, ks, Kpad, planes, exps, rowmax); break;
    case 6:  // float64 rows only (47 fraction bits; the double-float path keeps <= 5 planes)
      if constexpr (std::is_same<T, double>::value) {
        slice_rows_kernel<6, T><<<grid, 256, 0, st>>>(src, R, K, rs, ks, Kpad, planes, exps, rowmax);
        break;
      } else {
        return DSRG_FNO_ERR_ARG;
      }
    default: return DSRG_FNO_ERR_ARG;
  }
  DSRG_LAUNCH_CHECK();
  return DSRG_FNO_OK;
}

int stage_literal(int form, int KS, const double* src, long R, int K, long rs, long ks, int Kpad, void* planes,
                  int* exps, cudaStream_t st) {
  if (R <= 0) return DSRG_FNO_OK;
  if (Kpad % 32 != 0) return DSRG_FNO_ERR_ARG;
  dim3 grid((unsigned)((R + 31) / 32), (unsigned)(Kpad / 32));
  if (form == FORM_BF16X3 && KS == 2) split_rows_kernel<FORM_BF16X3, 2><<<grid, 256, 0, st>>>(src, R, K, rs, ks, Kpad, planes, exps);
  else if (form == FORM_TF32 && KS == 1) split_rows_kernel<FORM_TF32, 1><<<grid, 256, 0, st>>>(src, R, K, rs, ks, Kpad, planes, exps);
  else if (form == FORM_TF32 && KS == 2) split_rows_kernel<FORM_TF32, 2><<<grid, 256, 0, st>>>(src, R, K, rs, ks, Kpad, planes, exps);
  else return DSRG_FNO_ERR_ARG;
  DSRG_LAUNCH_CHECK();
  return DSRG_FNO_OK;
}

int slice_rows(int KS, const double* src, long R, int K, long rs, long ks, int Kpad, __nv_bfloat16* planes,
               int* exps, cudaStream_t st) {
  return slice_rows_t(KS, src, R, K, rs, ks, Kpad, planes, exps, nullptr, st);
}

int slice_rows_dd(int KS, const float2* src, long R, int K, long rs, long ks, int Kpad, __nv_bfloat16* planes,
                  int* exps, const unsigned* rowmax, cudaStream_t st) {
  return slice_rows_t(KS, src, R, K, rs, ks, Kpad, planes, exps, rowmax, st);
}

}  // namespace dsrg
