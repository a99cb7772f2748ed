/*
 * dsrg_fno.h - C ABI of the GB300 (sm_103a) FNO SA-DSRG-PT2 hot path.
 *
 * Method: frozen natural orbitals for state-averaged DSRG, arXiv:2312.07008.
 * The library forms the regularised first-order amplitudes of SA-DSRG-PT2
 * from density-fitted integrals (Eqs. A6, A7), contracts them into the
 * virtual-virtual block of the unrelaxed second-order 1-RDM (Eq. A12) and the
 * vv-class second-order energy (scalar of Eq. A4), diagonalises that block
 * into natural orbitals (Eq. 8), truncates the virtual NOs (Eqs. 9, 10 and
 * the near-degeneracy rule of Sec. 2), and forms the second-order correction
 * for the discarded virtuals (scalar part of Eq. 11).  The full second-order
 * energy over every amplitude class, and its correction, are available too
 * (dsrg_fno_pt2_energy_mr, dsrg_fno_discarded_correction_mr).
 *
 * Conventions shared by every entry point
 *   - nh = ncore + nact holes (core first), np = nact + nvir particles
 *     (active first).  Orbitals are semicanonical.
 *   - Arrays are row-major, float64, caller-owned.  "device" pointers are
 *     CUDA device memory of the current device, 8-byte aligned; "host"
 *     pointers are ordinary host memory.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Work is enqueued on it; scalars returned through host
 *     pointers are valid when the call returns (the call synchronises the
 *     stream for them).
 *   - Return value: DSRG_FNO_OK (0) or a negative dsrg_fno_status.  On error
 *     the outputs are unspecified.  No C++ exception crosses the ABI.
 *   - The library keeps a grow-only device workspace per device; it is freed
 *     by dsrg_fno_release().  Calls on one device are serialised by the
 *     library's workspace lock; one problem per call.
 */
#ifndef DSRG_FNO_H
#define DSRG_FNO_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  DSRG_FNO_OK = 0,
  DSRG_FNO_ERR_ARG = -1,        /* invalid argument (null pointer, size, mode) */
  DSRG_FNO_ERR_CUDA = -2,       /* a CUDA runtime call failed */
  DSRG_FNO_ERR_NOMEM = -3,      /* device workspace could not be allocated */
  DSRG_FNO_ERR_NOCONV = -4,     /* the eigensolver did not converge */
  DSRG_FNO_ERR_TIMEOUT = -5,    /* a bounded device wait expired */
  DSRG_FNO_ERR_NONFINITE = -6,  /* an input or result is NaN/Inf */
  DSRG_FNO_ERR_UNSUPPORTED = -7 /* valid request this build does not serve */
} dsrg_fno_status;

/* Arithmetic of the integral contractions.  FP64: plain float64 on the CUDA
 * cores.  SLICED_BF16: each float64 row is split into `nslices` exact bfloat16
 * digit planes with a per-row power-of-two scale; digit products run on the
 * tensor cores (tcgen05) with exact float32 level sums, merged into
 * double-float accumulators (float32 hi + lo pairs, about 48 bits); the
 * regulariser and the dressing of this form run in double-float, the energy
 * and D_vv sums in float64.  In both forms the NO eigensolve runs in
 * double-float.  On the workloads here the two forms agree to a few 1e-9 E_h
 * in energies; ONs are tested to agree within 1e-8. */
/* BF16X3 and TF32 are the literal forms of the precision study: only the
 * contractions of B with B (nu^{ij}_{ab} = sum_Q B^Q_{ia} B^Q_{jb}, Eq. A7, of
 * the D_vv pass and of the energy passes of the correction) run as tensor-
 * core products with one float32 accumulator over the whole auxiliary index;
 * everything else runs as in SLICED_BF16 with 5 planes.
 *   BF16X3: x = hi + lo (hi = bf16(x), lo = bf16(x - hi)), products
 *           hi.hi + hi.lo + lo.hi (3 terms).
 *   TF32:   nslices 1: tf32(x).tf32(y); nslices 0 or 3: x = big + small
 *           (tf32 parts), big.big + big.small + small.big (3 terms).
 * Their errors against float64 are far above 1e-7 E_h on the workloads here
 * (they exist to measure that); SLICED_BF16 is the fast form. */
typedef enum { DSRG_FNO_FP64 = 0, DSRG_FNO_SLICED_BF16 = 1, DSRG_FNO_BF16X3 = 2, DSRG_FNO_TF32 = 3 }
    dsrg_fno_precision;

typedef struct {
  int32_t ncore, nact, nvir, naux;
  /* device [naux][nh][np]: B^Q_{ip}, hole i, particle p (DF factors, Sec. 3);
   * the active(hole) x active(particle) sub-block must be symmetric in (i,p). */
  const double* B_hp;
  /* device [ncore+nact+nvir]: semicanonical orbital energies eps_p, ordered
   * core | active | virtual (the Delta denominators below Eq. A7). */
  const double* eps;
  /* device [nact][nact]: state-averaged spin-free 1-RDM Gamma^u_v (Eq. A1);
   * NULL iff nact == 0. */
  const double* gamma1;
  /* device [nact]^4: state-averaged spin-free 2-cumulant Lambda^{uv}_{xy},
   * with Gamma^{uv}_{xy} = Lambda + Gamma^u_x Gamma^v_y - 1/2 Gamma^v_x Gamma^u_y
   * (definitions after Eq. A12); NULL iff nact == 0. */
  const double* lambda2;
  /* device [nh][np] off-diagonal Fock f^i_a of Eq. A6, or NULL (= 0). */
  const double* f_hp;
  /* host [nstates] state weights w_alpha of Eq. A1: each >= 0, sum 1 (1e-12).
   * Metadata: the densities above already carry them. */
  int32_t nstates;
  const double* weights;
  /* flow parameter s (E_h^-2), s >= 0 (Eq. A7). */
  double s;
  int32_t precision;  /* dsrg_fno_precision */
  int32_t nslices;    /* SLICED_BF16 digit planes: 3, 4 or 5; 0 = library default (5);
                       * TF32 terms: 1 or 3 (0 = 3); BF16X3: 0 or 3;
                       * other values give DSRG_FNO_ERR_UNSUPPORTED */
} dsrg_fno_problem;

/* vv-class SA-DSRG-PT2 energy E_vv (doubles whose particles are both
 * virtual; Eq. A4 scalar restricted to them; in the single-reference limit
 * the whole DSRG-PT2 energy).  e2_out: host scalar. */
int dsrg_fno_pt2_energy(const dsrg_fno_problem* prob, double* e2_out, void* stream);

/* Full second-order SA-DSRG energy E^(2) = <[H, A]>_0 + 1/2 <[[H0, A], A]>_0,
 * the correlation part of <H-bar^[2]> (the second-order Hamiltonian stated
 * with Eq. A4), over every first-order amplitude class of Eqs. A6, A7: the
 * doubles with active or virtual particles and core or active holes (the
 * all-active block excluded) and the singles, with the off-diagonal Fock
 * f^i_a of f_hp (NULL: zero).  The scalar is evaluated by the generalised
 * Wick theorem in the Mukherjee-Kutzelnigg normal order of the ensemble:
 * Gamma1 and Lambda2 always, the 3-cumulant when `lambda3` is given.
 *   lambda3  device [nact]^6 (layout as in dsrg_fno_vv_opdm_lambda3), or NULL:
 *            the terms with one 3-cumulant are then dropped, which Sec. 2
 *            allows when the 1-RDM drops them too (dsrg_fno_vv_opdm); read only.
 *   e2_out   host: E^(2).
 *   evv_out  host, may be NULL: its vv-class part E_vv (dsrg_fno_pt2_energy).
 * E_vv runs on the path that prob->precision selects; the rest (the doubles
 * with an active particle, the singles, their cumulant couplings) in float64,
 * except that outside the FP64 form its integrals <ay|ij> (one contraction
 * over the auxiliary index, rows (i, a) against (j, y), y active) run on the
 * digit-plane tensor-core path when naux >= 256.
 * In the single-reference limit (nact = 0) E^(2) = E_vv plus the singles of
 * f_hp.  Errors as for dsrg_fno_pt2_energy; a host lambda3 gives
 * DSRG_FNO_ERR_ARG, a non-finite one DSRG_FNO_ERR_NONFINITE.  Device
 * workspace: about 32 nh^2 np nact bytes beyond the E_vv pass, plus the digit
 * planes of B (2 nslices nh np naux bytes) on the tensor-core path (grow-only,
 * freed by dsrg_fno_release).  Synchronises `stream`. */
int dsrg_fno_pt2_energy_mr(const dsrg_fno_problem* prob, const double* lambda3, double* e2_out,
                           double* evv_out, void* stream);

/* D_vv = virtual-virtual block of the unrelaxed PT2 1-RDM correction, Eq. A12
 * terms 1-12 (the Lambda3 term 13 is not formed, as Sec. 2 allows when the
 * energy drops Lambda3), symmetrised.  dvv_out: device [nvir][nvir].
 * e2_out: host, may be NULL; when given, receives E_vv of the same pass. */
int dsrg_fno_vv_opdm(const dsrg_fno_problem* prob, double* dvv_out, double* e2_out,
                     void* stream);

/* D_vv of dsrg_fno_vv_opdm plus Eq. A12 term 13,
 *   t^{uw}_{ez} t^{xy}_{fv} Lambda^{xyz}_{uvw},
 * the contraction with the state-averaged 3-cumulant that Sec. 2 drops
 * whenever the final energy drops Lambda3 (for an energy that keeps it, or to
 * measure what dropping it does to the ONs and N').
 *   lambda3  device [nact]^6, Lambda^{xyz}_{uvw} at
 *            ((((x*nact + y)*nact + z)*nact + u)*nact + v)*nact + w, as written
 *            by dsrg_fno_sa_lambda3; required when nact > 0 (NULL gives
 *            DSRG_FNO_ERR_ARG), ignored when nact == 0; read only.
 *   Other arguments, outputs and errors as for dsrg_fno_vv_opdm; a non-finite
 *   lambda3 gives DSRG_FNO_ERR_NONFINITE.  The term is formed in float64 in
 *   both precisions; with SLICED_BF16 its final contraction (length nact^3,
 *   when >= 256) runs on the digit-plane tensor-core path like terms 10-12. */
int dsrg_fno_vv_opdm_lambda3(const dsrg_fno_problem* prob, const double* lambda3, double* dvv_out,
                             double* e2_out, void* stream);

/* State-averaged spin-free 3-cumulant Lambda^{xyz}_{uvw} on the device (the
 * 3-body density cumulant named after Eq. A12), from the ensemble's Gamma1
 * and 2-cumulant and the per-state spin-free 3-RDMs.
 *   weights        host [nstates], each >= 0, summing to 1 (1e-12); nstates <= 32.
 *   gamma1         device [nact][nact], ensemble Gamma^u_v (as in dsrg_fno_problem).
 *   lambda2        device [nact]^4, ensemble Lambda^{uv}_{xy} (as in dsrg_fno_problem).
 *   gamma3_states  device [nstates][nact]^6, state a's
 *                  Gamma3_a[x][y][z][u][v][w] = sum_{s,t,r} <a+_{xs} a+_{yt} a+_{zr} a_{wr} a_{vt} a_{us}>.
 *   lambda3_out    device [nact]^6 (layout as in dsrg_fno_vv_opdm_lambda3).
 * The ensemble Gamma3 = sum_a w_a Gamma3_a; the cumulant is the spin sum of
 * the spin-orbital cumulant over the pairs (x,u), (y,v), (z,w) with the
 * spin-orbital 1-RDM Gamma1/2 per spin (exact for spin-adapted ensembles, a
 * definition otherwise, like Lambda2):
 *   Lambda3 = Gamma3 - [G^x_u L^{yz}_{vw} + G^y_v L^{xz}_{uw} + G^z_w L^{xy}_{uv}]
 *           + 1/2 [G^x_v L^{yz}_{uw} + G^x_w L^{yz}_{vu} + G^y_u L^{xz}_{vw}
 *                  + G^y_w L^{xz}_{uv} + G^z_u L^{xy}_{wv} + G^z_v L^{xy}_{uw}]
 *           - G^x_u G^y_v G^z_w + 1/2 [G^x_v G^y_u G^z_w + G^x_w G^y_v G^z_u + G^x_u G^y_w G^z_v]
 *           - 1/4 [G^x_v G^y_w G^z_u + G^x_w G^y_u G^z_v].
 * Errors: DSRG_FNO_ERR_ARG for nact outside 1..16, nstates outside 1..32, a
 * null or host pointer where a device one is due, or bad weights;
 * DSRG_FNO_ERR_NONFINITE for a non-finite result.  Synchronises `stream`. */
int dsrg_fno_sa_lambda3(int32_t nact, int32_t nstates, const double* weights, const double* gamma1,
                        const double* lambda2, const double* gamma3_states, double* lambda3_out,
                        void* stream);

/* Natural orbitals of D_vv (Eq. 8) and the truncation of Sec. 2.
 *   dvv       device [nvir][nvir], symmetric, read only.
 *   mode      0: p_o (Eq. 10, threshold in percent of the summed ONs);
 *             1: p_v (Eq. 9, threshold in percent of nvir, rounded up);
 *             2: n_kappa (keep ONs >= threshold);
 *             3: a fixed N' = threshold (rounded, clamped to [0, nvir]): the
 *                same number of virtuals at every geometry of a potential
 *                energy surface, which Sec. 4 suggests against the jumps a
 *                cumulative cut makes (pass degen_ratio 0 to keep N' exact).
 *   degen_ratio  near-degeneracy widening: while the next ON differs from the
 *             last kept one by less than degen_ratio times the larger, keep it
 *             (0.01 in the paper); 0 disables.
 *   on_out    device [nvir]: ONs, descending.
 *   no_out    device [nvir][nvir]: column k is the NO of on_out[k] in the
 *             semicanonical virtual basis; sign: largest |component| > 0.
 *   nkept_out host: N'.  */
int dsrg_fno_truncate(int32_t nvir, const double* dvv, int32_t mode, double threshold,
                      double degen_ratio, double* on_out, double* no_out,
                      int32_t* nkept_out, void* stream);

/* The truncation of dsrg_fno_truncate applied to ONs already computed (for
 * further cuts of the same NOs, e.g. p_o = 98 % and 99 %).
 *   ons  device [nvir], descending (as written by dsrg_fno_truncate).
 *   mode, threshold, degen_ratio, nkept_out: as in dsrg_fno_truncate. */
int dsrg_fno_cut(int32_t nvir, const double* ons, int32_t mode, double threshold, double degen_ratio,
                 int32_t* nkept_out, void* stream);

/* dsrg_fno_truncate without any device allocation (the paper has no
 * counterpart; this is a service for callers that cannot allocate).  Some
 * callers cannot call cudaMalloc: a framework that owns all device memory
 * through its own pool, or a latency-critical loop where an allocation, which
 * may synchronise the device, is not acceptable.  This call does the same
 * eigensolve and cut as dsrg_fno_truncate with the same arguments, but its
 * scratch is one fixed file-scope device array of the library (5 nvir^2
 * doubles and a few KB for nvir up to 512, about 10.5 MB), held by every device that loads
 * the library until the process exits.
 *   - nvir > 512 returns DSRG_FNO_ERR_ARG, with the limit named in a message
 *     to the log callback (dsrg_fno_set_log_callback).  dvv, on_out and
 *     no_out must be device memory (else DSRG_FNO_ERR_ARG, before any work).
 *   - Every call looks up the array's device address on the current device
 *     (cudaGetSymbolAddress, which allocates nothing); the first call on a
 *     device also loads the library's device code there (set-up), so make
 *     that first call before any stream capture.
 *   - Every call on a device shares the array, which keeps the last call's
 *     contents; each call writes every scratch word before reading it.  Calls
 *     whose GPU work overlaps (other streams or threads) race on the array:
 *     serialise them.
 *   - No cudaMalloc, cudaFree or allocating library routine is called. */
int dsrg_fno_truncate_noalloc(int32_t nvir, const double* dvv, int32_t mode, double threshold,
                              double degen_ratio, double* on_out, double* no_out,
                              int32_t* nkept_out, void* stream);

/* Particle-particle ladder of Eq. 6 in a (truncated) virtual basis: of the
 * two-body commutator C2 = [O2, T2]_2, the term with four virtual indices,
 * which sets its O(N_C^2 N_V^4) cost and which the FNO truncation cuts by
 * (N_V'/N_V)^4 (Sec. 2):
 *   C^{ij}_{ab} = sum_{cd} <ab|cd> T^{ij}_{cd},  <ab|cd> = sum_Q B^Q_{ac} B^Q_{bd}
 * with the bare DF integrals as the four-virtual block of O2.
 *   nv, naux   virtual orbitals of the basis (N_V or N_V') and DF functions.
 *   B_vv       device [naux][nv][nv]: B^Q_{ab}, virtual-virtual DF factors in
 *              that basis (e.g. rotated to the recanonicalised kept NOs).
 *   T          device [npairs][nv][nv]: T[p][c][d] = T^{ij}_{cd} of hole pair p.
 *   precision  DSRG_FNO_FP64 or DSRG_FNO_SLICED_BF16 (5 digit planes).
 *   C_out      device [npairs][nv][nv].
 * The 4-index integrals are formed for 16 values of a at a time and never
 * stored whole.  Errors: DSRG_FNO_ERR_ARG for bad sizes, null or host
 * pointers; DSRG_FNO_ERR_NONFINITE for a NaN/Inf in B_vv or T; sizes with
 * nv^3 * 16 or npairs * nv^2 >= 2^31 and other precisions give
 * DSRG_FNO_ERR_UNSUPPORTED. */
int dsrg_fno_ladder(int32_t nv, int32_t naux, const double* B_vv, int32_t npairs, const double* T,
                    int32_t precision, double* C_out, void* stream);

/* Natural auxiliary functions (the compression of the auxiliary basis that
 * Sec. 4 proposes for the PT2 step): W_PQ = sum_{ia} B^P_{ia} B^Q_{ia} over
 * the hole-particle factors is diagonalised, W = U diag(w) U^T with w
 * descending, and the factors are rotated to the naux' eigenvectors with
 * w_K > threshold: B'^K_{ia} = sum_Q U_QK B^Q_{ia}.  B' gives every integral
 * nu^{ij}_{ab} up to the discarded weight (sum of the dropped w), so a
 * problem with B' and naux' replaces the original one.
 *   nh, np     holes (ncore + nact) and particles (nact + nvir).
 *   B_hp       device [naux][nh][np], as in dsrg_fno_problem.
 *   threshold  absolute eigenvalue threshold (w > threshold kept).
 *   precision  DSRG_FNO_FP64, or DSRG_FNO_SLICED_BF16 (digit-plane
 *              contractions: 5 planes for W, 6 for B'); the eigensolve is the
 *              double-float Jacobi solver in both.
 *   B_out      device [naux][nh][np], caller-allocated: its first naux'
 *              slices receive B' (the rest is left untouched).
 *   w_out      device [naux] or NULL: every eigenvalue of W, descending.
 *   naux_out   host: naux'.
 * Errors: DSRG_FNO_ERR_ARG for bad sizes, null or host pointers;
 * DSRG_FNO_ERR_NONFINITE for a NaN/Inf in B_hp; other precisions give
 * DSRG_FNO_ERR_UNSUPPORTED. */
int dsrg_fno_naf(int32_t nh, int32_t np, int32_t naux, const double* B_hp, double threshold,
                 int32_t precision, double* B_out, double* w_out, int32_t* naux_out, void* stream);

/* Second-order correction for the discarded virtuals (scalar part of
 * Eq. 11): the kept NOs (first nkept columns of `no`, device [nvir][nvir])
 * are recanonicalised (virtual Fock block diagonal, Sec. 2), B is rotated to
 * them, and E_vv is re-evaluated in that basis.
 *   e2_mo_in    host or NULL: E_vv(MO) of the same problem (as returned by
 *               dsrg_fno_vv_opdm); NULL makes the call evaluate it.
 *   de_out      host: E_vv(MO) - E_vv(FNO).
 *   e2_fno_out  host or NULL: E_vv(FNO).
 *   eps_fno_out device [nkept] or NULL: recanonicalised virtual energies, ascending. */
int dsrg_fno_discarded_correction(const dsrg_fno_problem* prob, int32_t nkept,
                                  const double* no, const double* e2_mo_in, double* de_out,
                                  double* e2_fno_out, double* eps_fno_out, void* stream);

/* Eq. 11 with the full second-order energy of dsrg_fno_pt2_energy_mr:
 * E^(2)(MO) - E^(2)(FNO), where the FNO problem keeps the active particles
 * and the recanonicalised kept NOs (B, the virtual orbital energies and the
 * virtual columns of f_hp rotated to them).  Beside the vv part this carries
 * the active-labelled parts of the correction (the doubles with an active
 * particle, the singles and their cumulant couplings; Sec. 2 costs them as
 * O(N_V^2 (N_C^2 + N_A^4))).
 *   lambda3     device [nact]^6 or NULL, as in dsrg_fno_pt2_energy_mr (used in
 *               both bases).
 *   e2_mo_in    host or NULL: the full E^(2)(MO) of the same problem (as
 *               returned by dsrg_fno_pt2_energy_mr with the same lambda3);
 *               NULL makes the call evaluate it.
 *   de_out      host: E^(2)(MO) - E^(2)(FNO).
 *   e2_fno_out  host or NULL: E^(2)(FNO); with nkept = 0 it is the energy of
 *               the active particles alone (not zero).
 *   Other arguments and errors as for dsrg_fno_discarded_correction; both
 *   energies are evaluated as in dsrg_fno_pt2_energy_mr. */
int dsrg_fno_discarded_correction_mr(const dsrg_fno_problem* prob, const double* lambda3, int32_t nkept,
                                     const double* no, const double* e2_mo_in, double* de_out,
                                     double* e2_fno_out, double* eps_fno_out, void* stream);

/* State-averaged densities of Eq. A1 from per-state spin-free densities,
 * host arrays (a helper for preparing dsrg_fno_problem inputs):
 *   w            [nstates] weights, each >= 0, summing to 1 (1e-12);
 *   g1_states    [nstates][nact][nact], Gamma1_a[u][v] = sum_sigma <a+_u a_v>;
 *   g2_states    [nstates][nact]^4, Gamma2_a[u][v][x][y] = sum_{sigma tau}
 *                <a+_{u sigma} a+_{v tau} a_{y tau} a_{x sigma}>;
 *   gamma1_out   [nact][nact]  = sum_a w_a Gamma1_a;
 *   lambda2_out  [nact]^4      = Gamma2 - Gamma1[u][x] Gamma1[v][y]
 *                               + 1/2 Gamma1[u][y] Gamma1[v][x],
 *                with Gamma1, Gamma2 the averaged densities (the cumulant of
 *                the ensemble, not an average of per-state cumulants).
 * Returns DSRG_FNO_ERR_ARG for nact < 1, nstates < 1, a null pointer or bad
 * weights.  No device work. */
int dsrg_fno_sa_densities(int32_t nact, int32_t nstates, const double* w, const double* g1_states,
                          const double* g2_states, double* gamma1_out, double* lambda2_out);

/* One instance of a batched run (dsrg_fno_batch_run). */
typedef struct {
  dsrg_fno_problem problem;  /* inputs, as for the single-instance calls */
  /* device [nvir][nvir]: D_vv (dsrg_fno_vv_opdm); NULL = energy only */
  double* dvv_out;
  /* natural orbitals and cut (dsrg_fno_truncate): cut_mode -1 = none, else
   * 0..3 (the modes of dsrg_fno_truncate) with cut_threshold and
   * cut_degen_ratio; needs dvv_out, on_out
   * (device [nvir]) and no_out (device [nvir][nvir]). */
  int32_t cut_mode;
  double cut_threshold, cut_degen_ratio;
  double* on_out;
  double* no_out;
  /* 1: discarded-virtual correction of the cut (dsrg_fno_discarded_correction) */
  int32_t correction;
  /* outputs, written by the call */
  double e2;      /* E_vv in the MO basis */
  int32_t nkept;  /* N' of the cut (0 without one) */
  double de;      /* E_vv(MO) - E_vv(FNO) (0 without a correction) */
  int32_t status; /* dsrg_fno_status of this instance */
} dsrg_fno_batch_item;

/* Runs n independent instances (ragged sizes, each the pipeline of the
 * single-instance calls it requests) concurrently on the current device:
 * instances are taken largest first by nworkers host workers, each with its
 * own CUDA stream and device workspace (a share of the free memory).  The
 * work is ordered after what `stream` holds at the call; the call returns
 * when every instance is done, and later work on `stream` is ordered after
 * it.  nworkers 0 = autotuned: the first calls with a given batch shape try
 * 2, 4 and 8 workers, later calls use the fastest.  Returns DSRG_FNO_OK
 * when every instance succeeded, else the status of the first failing
 * instance (in index order); each item carries its own status.  One batch
 * at a time per process (calls are serialised). */
int dsrg_fno_batch_run(dsrg_fno_batch_item* items, int32_t n, int32_t nworkers, void* stream);

/* Human-readable text of a status code. */
const char* dsrg_fno_status_string(int status);

/* Frees the device workspace of every device the library touched. */
void dsrg_fno_release(void);

/* Log sink of the library (the paper has no counterpart).  The library
 * writes nothing to stdout or stderr; the text of a failed CUDA call or of a
 * rejected argument goes to `fn` (level 0 error, 1 warning; `message` is
 * valid during the call only), with `user` passed through.  NULL (the
 * default) drops the messages; the status codes are returned either way.
 * The callback may be called from any thread that calls the library, one
 * message at a time. */
typedef void (*dsrg_fno_log_fn)(int level, const char* message, void* user);
void dsrg_fno_set_log_callback(dsrg_fno_log_fn fn, void* user);

#ifdef __cplusplus
}
#endif
#endif /* DSRG_FNO_H */
