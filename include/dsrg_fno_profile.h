/*
 * dsrg_fno_profile.h - launch accounting of libdsrg_fno.so.
 *
 * While profiling is enabled, the library brackets every launch of its
 * tensor-core contraction kernel and of its float64 pair-contraction kernel
 * with CUDA events on the launching stream, and counts every kernel it
 * launches.  Queries synchronise on the recorded events.  Records of
 * concurrent calls (the batch runner's workers) are summed: phase totals are
 * then stream time, not wall time.
 */
#ifndef DSRG_FNO_PROFILE_H
#define DSRG_FNO_PROFILE_H
#include <stdint.h>
#ifdef __cplusplus
extern "C" {
#endif

/* enable != 0 starts recording (and clears earlier records); 0 stops. */
void dsrg_fno_profile_enable(int32_t enable);

/* Totals over the recorded launches of kernel `name` ("sliced_gemm_pair",
 * "sliced_gemm_syrk", "sliced_gemm_plain", "pair_gemm_f64", or a phase
 * "phase_*"): summed event time (ms), number of launches, and summed executed
 * flops.  Counters without timing ("eig_sweeps_large" / "eig_sweeps_small":
 * Jacobi sweeps of matrices with n >= 256 / n < 256) report calls in
 * `launches` and the summed count in `flops`.  Returns 0. */
int dsrg_fno_profile_query(const char* name, double* total_ms, int64_t* launches, double* flops);

/* Number of kernels the library launched since the last reset; `reset`
 * != 0 zeroes the counter after reading it. */
int64_t dsrg_fno_launch_count(int32_t reset);

/* Worker count the last dsrg_fno_batch_run used (0 before any). */
int32_t dsrg_fno_batch_last_workers(void);

#ifdef __cplusplus
}
#endif
#endif
