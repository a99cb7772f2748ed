// Fast form of the contractions: exact bfloat16 digit planes on the tcgen05
// tensor cores (the planes are staged by stage.cu).
//
// Products.  For two rows a, b:  x_a . x_b = 2^-14 sum_L 2^-8L S_L with the
// level sums S_L = sum_{s+t=L} sum_k d_s(a,k) d_t(b,k).  Only levels
// L <= KS-1 are formed (triangular truncation, KS(KS+1)/2 digit products).
// Every digit product is an integer of magnitude <= 2^14, so the level sums
// S_0, S_1, S_2 over a chunk of 320 k-values stay below 3 * 320 * 2^14 < 2^24
// in magnitude and the float32 accumulator of the tensor core holds them
// exactly.  The levels L >= 3 carry weights 2^-38 and smaller, so their
// float32 rounding (about 2^-24 of the level, 2^-48 of the product) stays far
// below the digit truncation (2^-40).  Every level is merged after every
// chunk, so the KS level accumulators of a chunk lie side by side in TMEM.
//
// Kernel.  Persistent, warp-specialised: warp 0 issues TMA loads of all KS
// planes of a 64-wide k block (128-byte swizzle) into a 2-3 stage ring, warp 1
// issues tcgen05.mma into per-level TMEM accumulators (double buffered per
// chunk; one MMA per A plane covers all its levels, the B planes being
// stacked), warps 2-5 drain them with tcgen05.ld and add 2^-14-8L S_L into a
// float32-pair (double-float) accumulator per element.  At the
// end of a tile the float64 result is written out.  Every mbarrier wait is
// bounded; on expiry the kernel records the failure and leaves.
#include <cuda.h>

#include "kernels.h"
#include "mma_schedule.cuh"
#include "regularizer.cuh"
#include "tc_ptx.cuh"

namespace dsrg {

namespace {

constexpr int BM = 128;
constexpr int BKE = 64;            // k elements per block (128 bytes of bf16, 128-byte swizzle)
constexpr int ROW_BYTES = 2 * BKE;
constexpr int KCHUNK_BLOCKS = 320 / BKE;  // 320 k-values per exact sum of levels 0, 1, 2
constexpr long long WAIT_LIMIT = 4000000000LL;  // ~2 s of clock cycles

enum { MODE_PAIR = 0, MODE_SYRK = 1, MODE_PLAIN = 2 };
constexpr int PLAIN_BAND = 8;  // row tiles per band of the plain mode's job order

// exact 2^e in float32 (0 below the normal range)
__device__ __forceinline__ float pow2f(int e) {
  if (e < -126) return 0.0f;
  if (e > 127) e = 127;
  return __int_as_float((e + 127) << 23);
}

// ------------------------------------------------------- double-float helpers
__device__ __forceinline__ void df_add(float& hi, float& lo, float x) {
  float s = __fadd_rn(hi, x);
  float bb = __fsub_rn(s, hi);
  float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(x, bb));
  err = __fadd_rn(err, lo);
  float s2 = __fadd_rn(s, err);
  lo = __fsub_rn(err, __fsub_rn(s2, s));
  hi = s2;
}

// ------------------------------------------------------------- GEMM kernel
struct GemmParams {
  int mode;
  int nkb;          // k blocks per segment (Kpad / 64)
  int ntm, ntn;     // tiles along rows / columns
  int njobs;
  const int* exps;  // row exponents of the planes
  // pair mode: output tiles of the (nh np) x (nh np) matrix of all hole-
  // particle rows; element (i a, j b) goes to nu_out[slot_of[i nh + j]][a][b]
  const int2* tiles;  // [njobs] (row tile, column tile)
  const int* slot_of; // [nh nh], -1 for a pair outside the batch
  int np, na, nh, rows;
  float2* nu_out;   // [slot][np][np], double-float (when not fused)
  // fused Eq. A7 epilogue (pair mode): tau and kappa of the vv elements
  // (double-float, [slot][nv][nv]) and the semi-internal amplitudes
  // ts[i][j][e][x] (float64) straight from the accumulators; nu is not stored
  PairEpilogue epi;
  int fused;
  // plain mode: C[m][n] = A[m] . B[n] (rows M x N), exps of A and B separately
  int M, N;
  const int* exps_b;
  double* c_out;
  long ldc;
  // syrk mode
  int nv, nr, nsplit;
  const double* seg_sign;  // [nr]
  double* dpart;           // [nsplit][nv][nv]
  int* err;
};

template <int BN>
__device__ __forceinline__ bool decode_job(const GemmParams& P, int job, int* slot, int* mt, int* nt) {
  if (P.mode == MODE_PAIR) {
    const int2 t = P.tiles[job];
    *slot = 0;
    *mt = t.x;
    *nt = t.y;
    return true;
  }
  if (P.mode == MODE_PLAIN) {
    // bands of PLAIN_BAND row tiles, column tile by column tile inside a
    // band: the CTAs running at one time share their A tiles and each B tile
    // is read once per band instead of once per row tile
    *slot = 0;
    const int full = P.ntm / PLAIN_BAND;
    const int per = PLAIN_BAND * P.ntn;
    const int b = job / per;
    if (b < full) {
      const int r = job - b * per;
      *nt = r / PLAIN_BAND;
      *mt = b * PLAIN_BAND + r % PLAIN_BAND;
    } else {
      const int left = P.ntm - full * PLAIN_BAND;
      const int r = job - full * per;
      *nt = r / left;
      *mt = full * PLAIN_BAND + r % left;
    }
    return true;
  }
  // syrk: upper tiles only (some f >= e inside), all splits
  int per = 0;
  for (int m = 0; m < P.ntm; ++m) per += P.ntn - (m * BM) / BN;
  *slot = job / per;  // split
  int rem = job % per, m = 0;
  while (rem >= P.ntn - (m * BM) / BN) {
    rem -= P.ntn - (m * BM) / BN;
    ++m;
  }
  *mt = m;
  *nt = (m * BM) / BN + rem;
  return true;
}

__device__ __forceinline__ void seg_range(const GemmParams& P, int split, int* r0, int* r1) {
  if (P.mode != MODE_SYRK) {
    *r0 = 0;
    *r1 = 1;
  } else {
    *r0 = (int)((long)P.nr * split / P.nsplit);
    *r1 = (int)((long)P.nr * (split + 1) / P.nsplit);
  }
}

// Arithmetic forms of the kernel.  DIGITS: exact bf16 digit planes (above).
// The literal forms, for the precision study of the B.B contraction: a value
// is split into KS floating-point parts whose products the tensor core sums
// into ONE float32 accumulator over the whole contraction (no chunk merges):
//   BF16X3: x = hi + lo, hi = bf16(x), lo = bf16(x - hi); hi.hi + hi.lo + lo.hi
//   TF32:   KS = 1: tf32(x) . tf32(y); KS = 2: big = tf32(x), small =
//           tf32(x - big), big.big + big.small + small.big  (kind::tf32)
template <int KS, int BN, int STAGES, int FORM>
struct Cfg {
  static constexpr bool DIG = FORM == FORM_DIGITS || FORM == FORM_DIGITS_T;  // digit planes
  static constexpr int EB = FORM == FORM_TF32 ? 4 : 2;      // bytes per element
  static constexpr int BKE_E = ROW_BYTES / EB;              // elements per 128-byte k block
  static constexpr int NPROD = DIG ? KS * (KS + 1) / 2 : (KS == 1 ? 1 : 3);
  static constexpr int A_SLICE = BM * ROW_BYTES;
  static constexpr int B_SLICE = BN * ROW_BYTES;
  static_assert(A_SLICE % 1024 == 0 && B_SLICE % 1024 == 0, "plane tiles keep the 1024-byte swizzle atoms aligned");
  static constexpr int A_BYTES = KS * A_SLICE;
  static constexpr int B_BYTES = KS * B_SLICE;
  static constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
  static constexpr int SMEM = STAGES * STAGE_BYTES + 1024 + 256;
  static_assert(SMEM <= 232448, "dynamic shared memory per block");
  static_assert((2 * STAGES + 9) * 8 + 8 <= 256, "barrier area");
  static constexpr int TMEM_COLS = 512;
  // every level is accumulated per chunk and merged after it (levels 0-2
  // exactly, see above), so one set of KS consecutive level accumulators,
  // double buffered, and each A plane needs one MMA per k step
  static constexpr int NEXACT = FORM == FORM_DIGITS ? KS : (FORM == FORM_DIGITS_T ? (KS < 3 ? KS : 3) : 1);
  static constexpr int SET_COLS = NEXACT * BN;              // levels of one chunk
  static constexpr int TAIL_BASE = 2 * SET_COLS;             // lower levels of one segment
  // levels accumulated per segment and merged once (none in the current
  // configurations: the digit form merges every level per chunk, a literal
  // form has a single accumulator)
  static constexpr int TAIL_COLS = DIG ? (KS - NEXACT) * BN : 0;
  static_assert(2 * SET_COLS + 2 * (TAIL_COLS > 0 ? TAIL_COLS : 0) <= TMEM_COLS, "TMEM budget");
  static_assert(!DIG || stacked_n_valid(KS, BN, NEXACT), "stacked MMA widths");
  static_assert(DIG || KS == 1 || KS == 2, "literal forms: one or two parts");
};

template <int KS, int BN, int STAGES, int FORM>
__global__ void __launch_bounds__(192, 1) sliced_gemm_kernel(const __grid_constant__ CUtensorMap mapA,
                                                             const __grid_constant__ CUtensorMap mapB,
                                                             GemmParams P) {
  using C = Cfg<KS, BN, STAGES, FORM>;
  // k blocks per chunk: the digit form merges exact level sums every 320 k;
  // a literal form accumulates the whole contraction in float32
  const int kchunk = C::DIG ? KCHUNK_BLOCKS : P.nkb;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + STAGES * C::STAGE_BYTES);
  uint64_t* empty = full + STAGES;
  uint64_t* tfull = empty + STAGES;
  uint64_t* tempty = tfull + 2;
  uint64_t* lfull = tempty + 2;   // low-order levels of a segment ready
  uint64_t* lempty = lfull + 2;   // ... drained
  uint64_t* done_bar = lempty + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done_bar + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      tc::mbar_init(&full[s], 1);
      tc::mbar_init(&empty[s], 1);
    }
    for (int q = 0; q < 2; ++q) {
      tc::mbar_init(&tfull[q], 1);
      tc::mbar_init(&tempty[q], 4);
      tc::mbar_init(&lfull[q], 1);
      tc::mbar_init(&lempty[q], 4);
    }
    tc::mbar_init(done_bar, 1);
    *abort_flag = 0;
    tc::fence_barrier_init();
  }
  if (warp == 0 && lane == 0) {
    tc::prefetch_tmap(&mapA);
    tc::prefetch_tmap(&mapB);
  }
  if (warp == 1) tc::tmem_alloc(tmem_slot, C::TMEM_COLS);
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    // ---------------------------------------------------------- TMA producer
    if (lane == 0) {
      uint32_t it = 0;
      for (int job = blockIdx.x; job < P.njobs && !*abort_flag; job += gridDim.x) {
        int slot, mt, nt;
        if (!decode_job<BN>(P, job, &slot, &mt, &nt)) continue;
        int r0, r1;
        seg_range(P, slot, &r0, &r1);
        for (int r = r0; r < r1; ++r) {
          int arow, brow;
          if (P.mode == MODE_PAIR || P.mode == MODE_PLAIN) {
            arow = mt * BM;
            brow = nt * BN;
          } else {
            arow = r * P.nv + mt * BM;
            brow = r * P.nv + nt * BN;
          }
          for (int kb = 0; kb < P.nkb; ++kb, ++it) {
            const int s = it % STAGES;
            const uint32_t ph = (it / STAGES) & 1;
            if (!tc::mbar_wait(&empty[s], ph ^ 1, WAIT_LIMIT)) {
              *abort_flag = 1;
              atomicExch(P.err, 1);
              break;
            }
            uint8_t* sa = smem + s * C::STAGE_BYTES;
            tc::mbar_arrive_expect_tx(&full[s], C::STAGE_BYTES);
            tc::tma_load_3d(sa, &mapA, kb * C::BKE_E, arow, 0, &full[s]);
            tc::tma_load_3d(sa + C::A_BYTES, &mapB, kb * C::BKE_E, brow, 0, &full[s]);
          }
          if (*abort_flag) break;
        }
      }
      // After an abort the MMA warp may not have consumed the last loads: no
      // CTA leaves with bulk copies in flight, so wait (bounded) until the
      // last load issued into every stage has landed.  Without an abort every
      // load was consumed and this is skipped.
      if (*abort_flag) {
        for (uint32_t k = it > (uint32_t)STAGES ? it - STAGES : 0; k < it; ++k)
          tc::mbar_wait(&full[k % STAGES], (k / STAGES) & 1, WAIT_LIMIT);
      }
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    uint32_t it = 0, chunk = 0, segc = 0;
    if (lane == 0) {
      for (int job = blockIdx.x; job < P.njobs && !*abort_flag; job += gridDim.x) {
        int slot, mt, nt;
        if (!decode_job<BN>(P, job, &slot, &mt, &nt)) continue;
        int r0, r1;
        seg_range(P, slot, &r0, &r1);
        for (int r = r0; r < r1 && !*abort_flag; ++r) {
          // low-order levels of this segment accumulate in tail set `lt`
          const uint32_t lt = segc & 1;
          if (C::TAIL_COLS > 0) {
            if (!tc::mbar_wait(&lempty[lt], ((segc >> 1) & 1) ^ 1, WAIT_LIMIT)) {
              *abort_flag = 1;
              atomicExch(P.err, 5);
              break;
            }
            tc::tc_fence_after();
          }
          uint32_t set = 0;
          for (int kb = 0; kb < P.nkb; ++kb, ++it) {
            const int kc = kb % kchunk;
            if (kc == 0) {
              set = chunk & 1;
              if (!tc::mbar_wait(&tempty[set], ((chunk >> 1) & 1) ^ 1, WAIT_LIMIT)) {
                *abort_flag = 1;
                atomicExch(P.err, 2);
                break;
              }
              tc::tc_fence_after();
            }
            const int s = it % STAGES;
            const uint32_t ph = (it / STAGES) & 1;
            if (!tc::mbar_wait(&full[s], ph, WAIT_LIMIT)) {
              *abort_flag = 1;
              atomicExch(P.err, 3);
              break;
            }
            tc::tc_fence_after();
            const uint32_t a_base = tc::smem_u32(smem + s * C::STAGE_BYTES);
            const uint32_t b_base = a_base + C::A_BYTES;
            const uint64_t a_desc0 = tc::make_sdesc_sw128(a_base);
            const uint64_t b_desc0 = tc::make_sdesc_sw128(b_base);
            // Stacked-B schedule: the products of A plane m.a with the
            // consecutive B planes m.b0 .. m.b0 + m.nb - 1 belong to the
            // consecutive levels m.level .. m.level + m.nb - 1, which lie one
            // after another in TMEM, and the B planes lie one after another in
            // shared memory: one MMA with N = m.nb BN does them all.
            if constexpr (C::DIG) {
#pragma unroll
            for (int i = 0; i < stacked_mma_count(KS, C::NEXACT); ++i) {
              const StackedMma m = stacked_mma(KS, i, C::NEXACT);
              // exact levels: per chunk (restart at the chunk's first block);
              // lower levels: per segment (restart at the segment's first block)
              const bool exact = m.level < C::NEXACT;
              const uint32_t d = exact ? tmem + set * C::SET_COLS + m.level * BN
                                       : tmem + C::TAIL_BASE + lt * C::TAIL_COLS + (m.level - C::NEXACT) * BN;
              const bool first_block = exact ? (kc == 0) : (kb == 0);
              const uint32_t idesc = tc::make_idesc_bf16(BM, m.nb * BN);
#pragma unroll
              for (int kk = 0; kk < 4; ++kk) {  // 16 bf16 of k per MMA
                // start-address field += byte offset / 16 (no carry: shared addresses < 2^18)
                const uint64_t ad = a_desc0 + (uint64_t)((m.a * C::A_SLICE + kk * 32) >> 4);
                const uint64_t bd = b_desc0 + (uint64_t)((m.b0 * C::B_SLICE + kk * 32) >> 4);
                // the MMA of A plane 0 covers every level of its set and comes
                // first: it alone starts a fresh accumulation
                const uint32_t acc = (first_block && kk == 0 && m.a == 0) ? 0u : 1u;
                tc::mma_bf16(d, ad, bd, idesc, acc);
              }
            }
            } else {
              // literal form: every product into one float32 accumulator
              const uint32_t d = tmem + set * C::SET_COLS;
#pragma unroll
              for (int pi = 0; pi < C::NPROD; ++pi) {
                const int pa = pi == 2 ? 1 : 0, pb = pi == 1 ? 1 : 0;
#pragma unroll
                for (int kk = 0; kk < 4; ++kk) {  // 32 bytes of k per MMA (16 bf16 or 8 tf32)
                  const uint64_t ad = a_desc0 + (uint64_t)((pa * C::A_SLICE + kk * 32) >> 4);
                  const uint64_t bd = b_desc0 + (uint64_t)((pb * C::B_SLICE + kk * 32) >> 4);
                  const uint32_t acc = (kc == 0 && kk == 0 && pi == 0) ? 0u : 1u;
                  if constexpr (FORM == FORM_TF32) tc::mma_tf32(d, ad, bd, tc::make_idesc_tf32(BM, BN), acc);
                  else tc::mma_bf16(d, ad, bd, tc::make_idesc_bf16(BM, BN), acc);
                }
              }
            }
            tc::mma_commit(&empty[s]);
            if (kc == kchunk - 1 || kb == P.nkb - 1) {
              tc::mma_commit(&tfull[set]);
              ++chunk;
            }
          }
          if (*abort_flag) break;
          if (C::TAIL_COLS > 0) tc::mma_commit(&lfull[lt]);
          ++segc;
        }
      }
      // all MMAs retired before TMEM is released
      tc::mma_commit(done_bar);
      tc::mbar_wait(done_bar, 0, WAIT_LIMIT);
    }
    __syncwarp();
  } else {
    // ------------------------------------------------- merge / output warps
    const int q = warp & 3;  // TMEM lane quadrant of this warp
    const int row = q * 32 + lane;
    uint32_t chunk = 0, segc = 0;
    // Fused Eq. A7 epilogue (pair mode): the finished accumulators of a tile
    // wait in local memory and are regularised a few columns at a time after
    // each chunk merge of the next tile, so that the MMA warp is not left
    // without a drained accumulator set while 48 regulariser evaluations run.
    float2 prev[BN];
    int prev_mt = 0, prev_nt = 0, prev_pos = BN;  // prev_pos == BN: nothing pending
    auto epi_range = [&](int c_end) {
      const int R = prev_mt * BM + row;
      if (R < P.rows) {
        const int i = R / P.np, a = R - i * P.np;
        const int ea = P.exps[R];
        const int* srow = P.slot_of + (long)i * P.nh;
        const float2 hr = P.epi.hp[R];
        const dd rowhp = {hr.x, hr.y}, sdd = {P.epi.s_hi, P.epi.s_lo};
        const int nv = P.epi.nv, na = P.na;
        const bool av = a >= na;
#pragma unroll 1
        for (int c = prev_pos; c < c_end; ++c) {
          const int C = prev_nt * BN + c;
          const int j = C / P.np, b = C - j * P.np;
          if (j >= P.nh) break;
          const int slot = srow[j];
          const bool bv = b >= na;
          // as the separate epilogue: vv -> tau, kappa; va -> ts[i][j];
          // av -> ts[j][i] unless i == j (the va element of that pair writes it)
          const bool want = slot >= 0 && (av || bv) && (av && bv ? true : (P.epi.ts != nullptr && (av || i != j)));
          if (!want) continue;
          const int sc = ea + P.exps[C];
          const dd n = {ldexpf(prev[c].x, sc), ldexpf(prev[c].y, sc)};
          const float2 hc = P.epi.hp[C];
          const dd delta = dd_add(rowhp, dd{hc.x, hc.y});
          dd r1, y;
          regularize(delta, sdd, *P.epi.reg, &r1, &y);
          const dd t = dd_mul(n, r1);
          if (av && bv) {
            const dd k = dd_mul(n, dd_add_f(y, 1.0f));
            const long o = ((long)slot * nv + (a - na)) * nv + (b - na);
            P.epi.tau[o] = make_float2(t.hi, t.lo);
            P.epi.kap[o] = make_float2(k.hi, k.lo);
          } else if (av) {
            P.epi.ts[(((long)i * P.nh + j) * nv + (a - na)) * na + b] = dd_to_double(t);
          } else {
            P.epi.ts[(((long)j * P.nh + i) * nv + (b - na)) * na + a] = dd_to_double(t);
          }
        }
      }
      prev_pos = c_end;
    };
    const bool spread = P.mode == MODE_PAIR && P.fused;
    for (int job = blockIdx.x; job < P.njobs; job += gridDim.x) {
      int slot, mt, nt;
      if (!decode_job<BN>(P, job, &slot, &mt, &nt)) continue;
      int r0, r1;
      seg_range(P, slot, &r0, &r1);
      float hi[BN], lo[BN];
#pragma unroll
      for (int c = 0; c < BN; ++c) {
        hi[c] = 0.f;
        lo[c] = 0.f;
      }
      bool failed = false;
      for (int r = r0; r < r1 && !failed; ++r) {
        // per-merge scale of this segment (syrk); pair/plain modes scale at the end
        float rowscale = 1.0f;
        const int* ecol = nullptr;
        if (P.mode == MODE_SYRK) {
          const int e = mt * BM + row;
          const int ea = (e < P.nv) ? P.exps[(long)r * P.nv + e] : -200;
          rowscale = (float)P.seg_sign[r] * pow2f(ea);
          ecol = P.exps + (long)r * P.nv + nt * BN;
        }
        // adds 2^(-14-8L) x level L (TMEM columns at col0) into the accumulators
        auto merge = [&](int L, uint32_t col0) {
          const float lscale = (C::DIG ? pow2f(-14 - 8 * L) : 1.0f) * rowscale;
#pragma unroll
          for (int c0 = 0; c0 < BN; c0 += 16) {
            float v[16];
            tc::tmem_ld16(tmem + ((uint32_t)(q * 32) << 16) + col0 + c0, v);
#pragma unroll
            for (int j = 0; j < 16; ++j) {
              float sc = lscale;
              if (P.mode == MODE_SYRK) {
                const int f = nt * BN + c0 + j;
                sc *= pow2f((f < P.nv) ? ecol[c0 + j] : -200);
              }
              df_add(hi[c0 + j], lo[c0 + j], v[j] * sc);
            }
          }
        };
        const int nchunks = (P.nkb + kchunk - 1) / kchunk;
        for (int c = 0; c < nchunks; ++c) {
          const uint32_t set = chunk & 1;
          if (!tc::mbar_wait(&tfull[set], (chunk >> 1) & 1, WAIT_LIMIT)) {
            *abort_flag = 1;
            atomicExch(P.err, 4);
            failed = true;
            break;
          }
          tc::tc_fence_after();
#pragma unroll 1
          for (int L = 0; L < C::NEXACT && L < KS; ++L) merge(L, set * C::SET_COLS + L * BN);
          tc::tc_fence_before();
          __syncwarp();
          if (lane == 0) tc::mbar_arrive(&tempty[set]);
          ++chunk;
          if (spread && prev_pos < BN) epi_range(min(BN, prev_pos + (BN + nchunks - 1) / nchunks));
        }
        if (failed) break;
        if (C::TAIL_COLS > 0) {
          const uint32_t lt = segc & 1;
          if (!tc::mbar_wait(&lfull[lt], (segc >> 1) & 1, WAIT_LIMIT)) {
            *abort_flag = 1;
            atomicExch(P.err, 6);
            failed = true;
            break;
          }
          tc::tc_fence_after();
#pragma unroll 1
          for (int L = C::NEXACT; L < KS; ++L) merge(L, C::TAIL_BASE + lt * C::TAIL_COLS + (L - C::NEXACT) * BN);
          tc::tc_fence_before();
          __syncwarp();
          if (lane == 0) tc::mbar_arrive(&lempty[lt]);
        }
        ++segc;
      }
      if (failed) break;
      // ------------------------------------------------------ tile output
      if (spread) {
        if (prev_pos < BN) epi_range(BN);  // a previous tile with fewer chunks than columns
#pragma unroll
        for (int c = 0; c < BN; ++c) prev[c] = make_float2(hi[c], lo[c]);
        prev_mt = mt;
        prev_nt = nt;
        prev_pos = 0;
      } else if (P.mode == MODE_PAIR) {
        const int R = mt * BM + row;
        if (R < P.rows) {
          const int i = R / P.np, a = R - i * P.np;
          const int ea = P.exps[R];
          const int* srow = P.slot_of + (long)i * P.nh;
          int j = (nt * BN) / P.np, b = nt * BN - j * P.np;
#pragma unroll
          for (int c = 0; c < BN; ++c) {
            if (j < P.nh) {
              const int slot = srow[j];
              if (slot >= 0 && !(a < P.na && b < P.na)) {
                const int sc = ea + P.exps[nt * BN + c];
                P.nu_out[((long)slot * P.np + a) * P.np + b] =
                    make_float2(ldexpf(hi[c], sc), ldexpf(lo[c], sc));  // double-float nu
              }
            }
            if (++b == P.np) {
              b = 0;
              ++j;
            }
          }
        }
      } else if (P.mode == MODE_PLAIN) {
        const int m = mt * BM + row;
        if (m < P.M) {
          const int ea = P.exps[m];
          double* out = P.c_out + (long)m * P.ldc;
#pragma unroll
          for (int c = 0; c < BN; ++c) {
            const int n = nt * BN + c;
            if (n < P.N) out[n] = ldexp((double)hi[c] + (double)lo[c], ea + P.exps_b[n]);
          }
        }
      } else {
        const int e = mt * BM + row;
        if (e < P.nv) {
          double* out = P.dpart + ((long)slot * P.nv + e) * P.nv;
#pragma unroll
          for (int c = 0; c < BN; ++c) {
            const int f = nt * BN + c;
            if (f < P.nv) out[f] = (double)hi[c] + (double)lo[c];
          }
        }
      }
    }
    // the last tile's epilogue (the job loop ends without a next tile)
    if (spread && prev_pos < BN && !*abort_flag) epi_range(BN);
  }
  __syncwarp();
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  if (warp == 1) tc::tmem_dealloc(tmem, C::TMEM_COLS);
}

// D[e][f] += sum_split dpart[split][min(e,f)][max(e,f)]
__global__ void syrk_tc_reduce_kernel(int nv, int nsplit, const double* __restrict__ dpart, double* D) {
  long idx = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (idx >= (long)nv * nv) return;
  int e = (int)(idx / nv), f = (int)(idx % nv);
  long src = e <= f ? (long)e * nv + f : (long)f * nv + e;
  double s = 0.0;
  for (int k = 0; k < nsplit; ++k) s += dpart[(long)k * nv * nv + src];
  D[idx] += s;
}

// ------------------------------------------------------- host side helpers
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  // initialised once, thread-safe (function-local static)
  static const EncodeTiledFn fn = []() -> EncodeTiledFn {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPoint("cuTensorMapEncodeTiled", &p, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      return reinterpret_cast<EncodeTiledFn>(p);
    return nullptr;
  }();
  return fn;
}

// 3-D map over planes [KS][rows][Kpad] (bf16, or float32 for tf32), box
// {128 bytes of k, box_rows, box_planes}, 128-byte swizzle.
int make_plane_map(CUtensorMap* map, const void* planes, int KS, long rows, int Kpad, int box_rows,
                   int box_planes, int eb) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return DSRG_FNO_ERR_CUDA;
  cuuint64_t dims[3] = {(cuuint64_t)Kpad, (cuuint64_t)rows, (cuuint64_t)KS};
  cuuint64_t strides[2] = {(cuuint64_t)Kpad * eb, (cuuint64_t)rows * Kpad * eb};
  cuuint32_t box[3] = {(cuuint32_t)(ROW_BYTES / eb), (cuuint32_t)box_rows, (cuuint32_t)box_planes};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = fn(map, eb == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(planes), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? DSRG_FNO_OK : DSRG_FNO_ERR_CUDA;
}

int num_sms() {
  int dev = 0, n = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
  return n > 0 ? n : 148;
}

template <int KS, int BN, int STAGES, int FORM = FORM_DIGITS>
int launch_gemm(const void* pa, long rows_a, const void* pb, long rows_b, int Kpad, GemmParams P,
                cudaStream_t st) {
  using C = Cfg<KS, BN, STAGES, FORM>;
  if (P.njobs <= 0) return DSRG_FNO_OK;
  if (Kpad % C::BKE_E != 0) return DSRG_FNO_ERR_ARG;
  P.nkb = Kpad / C::BKE_E;
  CUtensorMap ma, mb;
  DSRG_TRY(make_plane_map(&ma, pa, KS, rows_a, Kpad, BM, KS, C::EB));
  DSRG_TRY(make_plane_map(&mb, pb, KS, rows_b, Kpad, BN, KS, C::EB));
  auto kern = sliced_gemm_kernel<KS, BN, STAGES, FORM>;
  // the same value on every launch (per device, idempotent, thread-safe)
  DSRG_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM));
  const int grid = std::min(num_sms(), P.njobs);
  void* tok = nullptr;
  if (profiling()) {
    // executed tensor-core flops of the output tiles: tiles x 2 BM BN Kpad x digit products
    long tiles = 0;
    if (P.mode == MODE_PAIR) {
      tiles = P.njobs;
    } else if (P.mode == MODE_SYRK) {
      tiles = (long)P.njobs / P.nsplit * P.nr;  // every segment of every upper tile
    } else {
      tiles = P.njobs;
    }
    const double fl = 2.0 * BM * BN * (double)Kpad * C::NPROD * (double)tiles;
    const char* nm = P.mode == MODE_PAIR ? "sliced_gemm_pair" : (P.mode == MODE_SYRK ? "sliced_gemm_syrk"
                                                                                      : "sliced_gemm_plain");
    prof_begin(nm, fl, st, &tok);
  }
  kern<<<grid, 192, C::SMEM, st>>>(ma, mb, P);
  DSRG_LAUNCH_CHECK();
  prof_end(tok, st);
  return DSRG_FNO_OK;
}

int dispatch_gemm(int KS, const void* pa, long rows_a, const void* pb, long rows_b, int Kpad, GemmParams P,
                  cudaStream_t st, int form = FORM_DIGITS) {
  if (form == FORM_BF16X3) return launch_gemm<2, 64, 4, FORM_BF16X3>(pa, rows_a, pb, rows_b, Kpad, P, st);
  if (form == FORM_TF32)
    return KS == 1 ? launch_gemm<1, 64, 4, FORM_TF32>(pa, rows_a, pb, rows_b, Kpad, P, st)
                   : launch_gemm<2, 64, 4, FORM_TF32>(pa, rows_a, pb, rows_b, Kpad, P, st);
  if (P.mode == MODE_SYRK) {
    switch (KS) {
      case 3: return launch_gemm<3, 64, 3, FORM_DIGITS_T>(pa, rows_a, pb, rows_b, Kpad, P, st);
      case 4: return launch_gemm<4, 64, 2, FORM_DIGITS_T>(pa, rows_a, pb, rows_b, Kpad, P, st);
      case 5: return launch_gemm<5, 48, 2, FORM_DIGITS_T>(pa, rows_a, pb, rows_b, Kpad, P, st);
      default: return DSRG_FNO_ERR_ARG;
    }
  }
  switch (KS) {
    case 3: return launch_gemm<3, 64, 3>(pa, rows_a, pb, rows_b, Kpad, P, st);
    case 4: return launch_gemm<4, 64, 2>(pa, rows_a, pb, rows_b, Kpad, P, st);
    case 5: return launch_gemm<5, 48, 2>(pa, rows_a, pb, rows_b, Kpad, P, st);
    // 6 planes (21 products): TMEM allows N = 32, shared memory one stage
    case 6: return P.mode == MODE_PLAIN ? launch_gemm<6, 32, 1>(pa, rows_a, pb, rows_b, Kpad, P, st)
                                        : DSRG_FNO_ERR_ARG;
    default: return DSRG_FNO_ERR_ARG;
  }
}

int tile_n_for(int KS) { return KS == 6 ? 32 : (KS == 5 ? 48 : 64); }

}  // namespace

// ------------------------------------------------------------ public (lib)
// Output tiles of the pair contraction for one batch of hole pairs (i <= j).
// The rows of all holes form one (nh np)-row operand, so tiles run across the
// borders of the pairs' np x np blocks and no tile is padded to a block edge.
// A tile is listed when it meets a block of the batch outside that block's
// active x active corner (and, energy only, inside its virtual x virtual
// part).  Order: bands of ROW_BAND row tiles; within a band, column tile
// by column tile, the band's row tiles in turn, so that the CTAs running at
// one time share their A tiles (the band) and each B tile serves the band.
static constexpr int ROW_BAND = 8;

int pair_tile_n(int form, int KS) { return form == FORM_DIGITS ? tile_n_for(KS) : 64; }

int pair_tile_bound(int BN, const Geometry& g, int npairs) {
  return npairs * (ceil_div(g.np, BM) + 1) * (ceil_div(g.np, BN) + 1);
}

int pair_tiles(int BN, const Geometry& g, const int2* pairs, int npairs, bool energy_only, std::vector<int2>& out) {
  out.clear();
  if (npairs <= 0) return DSRG_FNO_OK;
  const long np = g.np, na = g.na;
  const int lo = energy_only ? (int)na : 0;
  int mt0 = 1 << 30, mt1 = -1;
  for (int k = 0; k < npairs; ++k) {
    mt0 = std::min<int>(mt0, (int)((pairs[k].x * np + lo) / BM));
    mt1 = std::max<int>(mt1, (int)((pairs[k].x * np + np - 1) / BM));
  }
  const int ntt = ceil_div((long)g.nh * np, BN);
  const int words = (ntt + 63) / 64;
  std::vector<uint64_t> bits((size_t)(mt1 - mt0 + 1) * words, 0);
  auto set_range = [&](int mt, int n0, int n1) {  // [n0, n1]
    uint64_t* row = bits.data() + (size_t)(mt - mt0) * words;
    for (int n = n0; n <= n1; ++n) row[n >> 6] |= (uint64_t)1 << (n & 63);
  };
  for (int k = 0; k < npairs; ++k) {
    const long i = pairs[k].x, j = pairs[k].y;
    const long r0 = i * np + lo, r1 = i * np + np, c0 = j * np + lo, c1 = j * np + np;
    for (int mt = (int)(r0 / BM); mt <= (int)((r1 - 1) / BM); ++mt) {
      // rows of this tile inside the block all active: skip the column
      // tiles that stay inside the active columns
      const bool rows_active = std::min<long>((long)mt * BM + BM, r1) - i * np <= na;
      long cs = c0;
      if (rows_active) {
        const long first = (j * np + na) / BN;  // first column tile reaching a virtual column
        cs = std::max<long>(c0, first * BN);
      }
      if (cs >= c1) continue;
      set_range(mt, (int)(cs / BN), (int)((c1 - 1) / BN));
    }
  }
  std::vector<uint64_t> band(words);
  for (int b0 = mt0; b0 <= mt1; b0 += ROW_BAND) {
    const int b1 = std::min(mt1, b0 + ROW_BAND - 1);
    std::fill(band.begin(), band.end(), 0);
    for (int mt = b0; mt <= b1; ++mt)
      for (int w = 0; w < words; ++w) band[w] |= bits[(size_t)(mt - mt0) * words + w];
    for (int w = 0; w < words; ++w) {
      uint64_t m = band[w];
      while (m) {
        const int n = w * 64 + __builtin_ctzll(m);
        m &= m - 1;
        for (int mt = b0; mt <= b1; ++mt)
          if ((bits[(size_t)(mt - mt0) * words + (n >> 6)] >> (n & 63)) & 1) out.push_back(make_int2(mt, n));
      }
    }
  }
  return DSRG_FNO_OK;
}

// nu[slot][a][b] of a batch of pairs from B planes ([KS][nh*np][Kpad]) over
// the output tiles of pair_tiles (device copy) and the batch's slot table.
int sliced_pair_gemm(int KS, int form, const Geometry& g, const void* planes, const int* exps, int Kpad,
                     const int2* tiles, int ntiles, const int* slot_of, float2* nu, const PairEpilogue* epi, int* err,
                     cudaStream_t st) {
  GemmParams P{};
  P.mode = MODE_PAIR;
  P.nkb = Kpad / BKE;
  P.njobs = ntiles;
  P.exps = exps;
  P.tiles = tiles;
  P.slot_of = slot_of;
  P.np = g.np;
  P.na = g.na;
  P.nh = g.nh;
  P.rows = g.nh * g.np;
  P.nu_out = nu;
  if (epi) {
    P.epi = *epi;
    P.fused = 1;
  }
  P.err = err;
  const long rows = (long)g.nh * g.np;
  return dispatch_gemm(KS, planes, rows, planes, rows, Kpad, P, st, form);
}

// D += sum_r sign_r Sig_r Sig_r^T from Sig planes ([KS][nr*nv][Kpad]).
int sliced_syrk(int KS, int nv, int nr, const __nv_bfloat16* planes, const int* exps, int Kpad, const double* sign,
                double* dpart, int nsplit, double* D, int* err, cudaStream_t st) {
  if (nr <= 0) return DSRG_FNO_OK;
  GemmParams P{};
  P.mode = MODE_SYRK;
  P.nkb = Kpad / BKE;
  const int BN = tile_n_for(KS);
  P.ntm = ceil_div(nv, BM);
  P.ntn = ceil_div(nv, BN);
  int per = 0;
  for (int m = 0; m < P.ntm; ++m) per += P.ntn - (m * BM) / BN;
  P.njobs = per * nsplit;
  P.exps = exps;
  P.nv = nv;
  P.nr = nr;
  P.nsplit = nsplit;
  P.seg_sign = sign;
  P.dpart = dpart;
  P.err = err;
  const long rows = (long)nr * nv;
  DSRG_TRY(dispatch_gemm(KS, planes, rows, planes, rows, Kpad, P, st));
  syrk_tc_reduce_kernel<<<ceil_div((long)nv * nv, 256), 256, 0, st>>>(nv, nsplit, dpart, D);
  DSRG_LAUNCH_CHECK();
  return DSRG_FNO_OK;
}

// C[m][n] (ldc) = A[m] . B[n] from planes of A ([KS][M][Kpad]) and B ([KS][N][Kpad]).
int sliced_plain_gemm(int KS, int M, int N, const void* pa, const int* ea, const void* pb,
                      const int* eb, int Kpad, double* C, long ldc, int* err, cudaStream_t st, int form) {
  if (M <= 0 || N <= 0) return DSRG_FNO_OK;
  GemmParams P{};
  P.mode = MODE_PLAIN;
  P.nkb = Kpad / BKE;
  const int BN = form == FORM_DIGITS ? tile_n_for(KS) : 64;
  P.ntm = ceil_div(M, BM);
  P.ntn = ceil_div(N, BN);
  P.njobs = P.ntm * P.ntn;
  P.exps = ea;
  P.exps_b = eb;
  P.M = M;
  P.N = N;
  P.c_out = C;
  P.ldc = ldc;
  P.err = err;
  return dispatch_gemm(KS, pa, M, pb, N, Kpad, P, st, form);
}

}  // namespace dsrg
