// Issue schedule of the digit-plane MMAs with a stacked B operand.
//
// One 16-wide k step of an output tile needs the products A_a B_b^T of the
// digit planes with a + b <= KS - 1, each added to the accumulator of level
// L = a + b.  The B planes of a tile lie one after another in shared memory
// (BN rows each, the plane index outermost in the TMA box) and the level
// accumulators of one set lie one after another in TMEM (BN columns each).
// So the products of A plane a with B planes b0 .. b0 + nb - 1 land in the
// consecutive levels a + b0 .. a + b0 + nb - 1, and ONE tcgen05.mma with
// N = nb * BN computes all of them.  Levels below the exact-level count live
// in the per-chunk set and the others in the per-segment tail set, so an A
// plane needs at most two MMAs, one per set: 8 MMAs per k step instead of 15
// for 5 planes, each A plane read from shared memory once per set instead of
// once per product.  In each set the MMA of A plane 0 covers every level of
// the set and is issued first, so it alone starts a fresh accumulation
// (accumulate flag 0) at the first k step of a chunk or segment.
#pragma once

namespace dsrg {

struct StackedMma {
  int a;      // A plane
  int b0;     // first B plane
  int nb;     // B planes (consecutive), = levels written
  int level;  // first level written (a + b0)
};

// Levels whose chunk sums the tensor core keeps exact (fp32) per chunk.
constexpr int kExactLevels = 3;

// N of the 128 x N tile in the configuration of each plane count (the
// TMEM budget of two exact sets and two tail sets sets it).
__host__ __device__ constexpr int plane_tile_n(int ks) { return ks == 5 ? 48 : (ks == 6 ? 32 : 64); }

__host__ __device__ constexpr int stacked_mma_count(int ks, int nexact = kExactLevels) {
  return (ks < nexact ? ks : nexact) + (ks > nexact ? ks : 0);
}

// The i-th MMA of a k step, in issue order: for each A plane its exact-set
// MMA, then its tail-set MMA.
__host__ __device__ constexpr StackedMma stacked_mma(int ks, int i, int nexact = kExactLevels) {
  const int top = ks < nexact ? ks : nexact;  // exact levels that exist
  for (int a = 0; a < ks; ++a) {
    if (a < top) {
      if (i == 0) return StackedMma{a, 0, top - a, a};
      --i;
    }
    if (ks > nexact) {
      const int l = a > nexact ? a : nexact;
      if (i == 0) return StackedMma{a, l - a, ks - l, l};
      --i;
    }
  }
  return StackedMma{-1, 0, 0, 0};
}

// Every MMA of the schedule has a valid N for M = 128 (a multiple of 16,
// 16 .. 256) when the level width is bn.
__host__ __device__ constexpr bool stacked_n_valid(int ks, int bn, int nexact = kExactLevels) {
  for (int i = 0; i < stacked_mma_count(ks, nexact); ++i) {
    const int n = stacked_mma(ks, i, nexact).nb * bn;
    if (n % 16 != 0 || n < 16 || n > 256) return false;
  }
  return true;
}

}  // namespace dsrg
