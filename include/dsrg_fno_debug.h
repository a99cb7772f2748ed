/*
 * dsrg_fno_debug.h - test hooks of libdsrg_fno.so (not part of the method).
 *
 * These entry points expose single building blocks of the fast form so that
 * tests can check them in isolation.  They allocate their own device buffers
 * (cudaMalloc/cudaFree), synchronise the device, and are not meant for
 * production use.  Return values follow dsrg_fno_status.
 */
#ifndef DSRG_FNO_DEBUG_H
#define DSRG_FNO_DEBUG_H
#include <stdint.h>
#ifdef __cplusplus
extern "C" {
#endif

/* C[M][N] = A[M][K] B[N][K]^T with the exact bf16 digit-plane GEMM on the
 * tensor cores (nslices planes, 3..6; 6 is the configuration the library
 * uses for the rotation of B to the frozen natural orbitals).  All arrays are host float64,
 * row-major.  This is the contraction kernel of the fast form by itself. */
int dsrg_fno_debug_sliced_gemm(int32_t nslices, int32_t M, int32_t N, int32_t K, const double* A,
                               const double* B, double* C);

/* C[M][N] = A[M][K] B[N][K]^T in a literal form of the precision study
 * (precision DSRG_FNO_BF16X3, nterms 0 or 3; DSRG_FNO_TF32, nterms 1 or 3,
 * 0 = 3): split parts on the tensor cores, one float32 accumulator over K.
 * Host float64 arrays, row-major. */
int dsrg_fno_debug_literal_gemm(int32_t precision, int32_t nterms, int32_t M, int32_t N, int32_t K,
                                const double* A, const double* B, double* C);

/* Digit planes of rows[R][K] (host float64): planes[s][r][Kpad] as float
 * values (host, R*Kpad*nslices) and the row exponents exps[R] (host). */
int dsrg_fno_debug_slice_rows(int32_t nslices, int32_t R, int32_t K, const double* rows, float* planes,
                              int32_t* exps);

/* Digit planes of double-float rows: rows[R][K][2] holds hi, lo float32
 * pairs (value hi + lo).  Output layout as dsrg_fno_debug_slice_rows. */
int dsrg_fno_debug_slice_rows_dd(int32_t nslices, int32_t R, int32_t K, const float* rows, float* planes,
                                 int32_t* exps);

/* The Eq. A7 regulariser as the fast form evaluates it (double-float):
 * r1[k] = (1 - exp(-s delta[k]^2)) / delta[k] (0 at delta = 0) and
 * y[k] = exp(-s delta[k]^2), for n host float64 inputs; outputs are host
 * float64 (the double-float value rounded). */
int dsrg_fno_debug_regularizer(int32_t n, const double* delta, double s, double* r1, double* y);

/* The stacked-B issue schedule of the digit-plane MMAs for nslices planes
 * (3..6), host only: entries[5*i ..] = {A plane, first B plane, B planes,
 * first level, N columns} of the i-th MMA of a 16-wide k step, in issue
 * order.  Returns the number of MMAs (>= 0), or DSRG_FNO_ERR_ARG for a bad
 * nslices, a null pointer or max_entries below that number. */
int dsrg_fno_debug_mma_schedule(int32_t nslices, int32_t* entries, int32_t max_entries);

/* Output tiles of the pair contraction for one batch of hole pairs, host
 * only: pairs[2k], pairs[2k+1] = (i, j), i <= j < ncore + nact; the tiles are
 * 128-row x N-column blocks (N = 48 for 5 planes, 64 for 3 or 4) of the
 * (nh np) x (nh np) matrix of all hole-particle rows; energy_only restricts
 * the needed elements to virtual x virtual.  tiles[2t], tiles[2t+1] = (row
 * tile, column tile) in the kernel's order.  Returns the tile count, or
 * DSRG_FNO_ERR_ARG for bad arguments or max_tiles too small. */
int dsrg_fno_debug_pair_tiles(int32_t nslices, int32_t ncore, int32_t nact, int32_t nvir, const int32_t* pairs,
                              int32_t npairs, int32_t energy_only, int32_t* tiles, int32_t max_tiles);

/* Spin limit (iterations of ~100 ns) of the eigensolver's grid barrier on
 * the current device; spins <= 0 restores the default (about 2 s).  A tiny
 * limit makes a multi-block solve's barrier wait run out, so that the
 * solver returns DSRG_FNO_ERR_TIMEOUT (fault injection on the device without
 * a hang: the expired block sets the status word and every block leaves). */
int dsrg_fno_debug_set_barrier_limit(int64_t spins);

/* on != 0: the fast form's Eq. A7 regulariser runs in the output stage of
 * the pair-contraction kernel; 0 (the default, faster on GB300): in a
 * separate kernel over the stored contraction tiles.  Affects later calls of
 * this process. */
int dsrg_fno_debug_set_fused_epilogue(int32_t on);

/* Digit planes of the dressed matrices in the fast form's rank-K update of
 * D_vv: 0 (default) = the problem's count; 3..5 = that many (at most the
 * problem's count).  Affects later calls of this process. */
int dsrg_fno_debug_set_syrk_planes(int32_t nslices);

/* on != 0 (the default): symmetric eigensolves above 80 x 80 run on the
 * column-pair Jacobi kernel; 0: on the round-parallel kernel over A in
 * global memory (for comparison).  Affects later calls of this process. */
int dsrg_fno_debug_set_eig_colpair(int32_t on);

/* Symmetric eigensolves of `count` (1..4) matrices at once, as the density
 * step of every pass does: n[e] x n[e] row-major float64 matrices A[e] (host,
 * overwritten: eigenvalues on the diagonal, unsorted), eigenvectors into the
 * columns of V[e] (host, n[e] x n[e]).  Matrices up to 80 x 80 share one
 * launch (one block each), larger ones are solved one after another first.
 * Allocates device memory; DSRG_FNO_ERR_NOCONV if a solve did not converge. */
int dsrg_fno_debug_eig_batch(int32_t count, const int32_t* n, double* const* A, double* const* V);

/* Bytes of device workspace the single-instance calls hold on the current
 * device (grow-only; 0 before the first call and after dsrg_fno_release()).
 * Host only: reads the library's bookkeeping, launches nothing. */
int64_t dsrg_fno_debug_workspace_bytes(void);

#ifdef __cplusplus
}
#endif
#endif
