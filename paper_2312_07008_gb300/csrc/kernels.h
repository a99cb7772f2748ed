// Internal launch API between the ABI layer and the kernels.
#pragma once
#include <cuda_bf16.h>

#include "common.cuh"

namespace dsrg {

// C[M][N] = alpha * op(A) op(B) + beta * C, float64, batched over blockIdx.z.
//   a_kcontig: op(A)[m][k] = A[m*lda + k]   else A[k*lda + m]
//   b_kcontig: op(B)[k][n] = B[n*ldb + k]   else B[k*ldb + n]
int gemm_f64(int M, int N, int K, double alpha, const double* A, long lda, bool a_kcontig,
             const double* B, long ldb, bool b_kcontig, double beta, double* C, long ldc,
             int batch, long sa, long sb, long sc, cudaStream_t st);

// Pair contraction nu^{ij}_{ab} = sum_Q B[Q][i][a] B[Q][j][b] for the listed
// unordered hole pairs (i <= j), with the Eq. A7 epilogue:
//   vv (a, b virtual): tau = nu R1(Delta), kappa = 2 nu - Delta tau -> tau/kap[slot][e][f]
//   va / av (one active particle): t^{ij}_{ex} -> ts[i][j][e][x], t^{ji}_{ex}
// ts may be null (energy-only passes).
int pair_gemm_f64(const Geometry& g, const double* B, const double* eps, const int2* pairs,
                  int npairs, double* tau, double* kap, double* ts, cudaStream_t st);

// Dressing work items of one batch (see dress.cu): outputs o_begin ..
// o_begin + o_count - 1 of one hole-pair group whose slots are slot ..
// slot + nslots - 1 and whose dressed matrices start at `out`.
struct DressDesc {
  int kind;     // DressKind
  int slot, nslots;
  int out;      // first dressed matrix of the group in the batch
  int o_begin, o_count;
  int m, pad;
};

enum DressKind {
  GROUP_CC_DIAG = 0,  // core pair (m, m): tau^{mm}, lambda 2
  GROUP_CC_PAIR = 1,  // core pair m < n: (tau +- tau^T)/sqrt2, lambda 2 and 6
  GROUP_CA = 2,       // core m with every active u: sum_u W[u][k] (tau^{mu} +- tau^{mu T})/sqrt2, g_k and 3 g_k
  GROUP_AA = 3        // all active pairs: eigenvectors of the two swap blocks of the aa hole 2-RDM
};

// outputs per work item; blocks per work item (they stride over upper tiles)
#ifndef DRESS_OUTPUTS
#define DRESS_OUTPUTS 8
#endif
#ifndef DRESS_BLOCKS
#define DRESS_BLOCKS 48
#endif
constexpr int DRESS_OC = DRESS_OUTPUTS;          // outputs of one dressing work item
constexpr int DRESS_TILE_BLOCKS = DRESS_BLOCKS;  // blocks sharing the tiles of one work item

struct DressAux {
  const double* g1_evec;   // [na][na] (column k)
  const double* g1_eval;   // [na]
  const double* aas_evec;  // [ns][ns]  ns = na(na+1)/2
  const double* aas_eval;
  const double* aaa_evec;  // [nd][nd]  nd = na(na-1)/2
  const double* aaa_eval;
  const int* aa_slot;      // [na][na] -> slot offset of unordered pair (min,max) within aa group
};

// sigma_r from tau (and kappa): energy partials and Sig_r = sqrt|lambda_r| sigma_r[tau].
int dress_f64(const Geometry& g, const DressDesc* d_desc, int ndesc, int ncc, const DressAux& aux,
              const double* tau, const double* kap, double* sig, double* sig_sign,
              double* e_part, bool want_sig, cudaStream_t st);

// D(upper tiles) += sum_r sign_r Sig_r Sig_r^T  (split-K partials, then reduction)
int syrk_dressed_f64(int nv, int nr, const double* sig, const double* sig_sign, double* dpart,
                     int nsplit, double* D, cudaStream_t st);

// Symmetric-eigen helpers (eig.cu)
constexpr int EIG_MAX_BLOCKS = 1024;  // grid bound of the eigensolver (reduction scratch)
constexpr size_t eig_work_doubles(int n) { return 3 * (size_t)n * n + 2 * EIG_MAX_BLOCKS + 16; }
int eig_set_barrier_limit(long long spins);
void set_eig_colpair(bool on);
int eig_sym_jacobi(int n, double* A, double* V, double* work, int* status_dev, int max_sweeps,
                   cudaStream_t st);
// eig_sym_jacobi on up to 4 matrices at once: those with n <= 80 in one
// launch, one block each; status_dev: 4 ints per matrix.
int eig_sym_jacobi_batch(int count, const int* n, double* const* A, double* const* V, double* const* work,
                         int* status_dev, int max_sweeps, cudaStream_t st);
// Marks the calling thread, for the scope's lifetime, as one of several host
// threads that share the device (batch workers): the eigensolver then keeps
// its cooperative grid small, since its blocks stay resident through every
// grid barrier and would crowd out the other workers' kernels.
struct SharedDeviceScope {
  bool prev;
  explicit SharedDeviceScope(bool shared);
  ~SharedDeviceScope();
};
int eig_sort(int n, const double* A, const double* V, double* evals, double* evecs, int* rank,
             bool descending, bool fix_sign, cudaStream_t st);

// aa block of the hole 2-RDM in the swap-(anti)symmetric pair bases (dress.cu)
int aa_blocks(int na, const double* g1, const double* lam2, double* Ms, double* Ma, cudaStream_t st);
// out = (accumulate ? out : 0) + sum x, fixed summation order (dress.cu)
int ordered_sum(const double* x, long n, double* out, bool accumulate, cudaStream_t st);

// Singles and semi-internal terms (small_terms.cu)
int t1_amplitudes(const Geometry& g, const double* ts, const double* eps, const double* f_hp,
                  const double* g1, double* t1, cudaStream_t st);
size_t small_terms_work_doubles(int nc, int na, int nv);
int small_terms_kmax(int nc, int na);
// Buffers of the tensor-core path of the small terms (ks = 0: float64 only).
struct SmallFast {
  int ks;
  __nv_bfloat16* planes;  // 2 * ks * nv * pad64(kmax)
  int* exps;              // 2 * nv
  double* cbuf;           // nv * nv
  int* err;
};
constexpr int SLICED_MIN_K = 256;
int small_terms_f64(const Geometry& g, const double* ts, const double* t1, const double* g1,
                    const double* l2, const double* l3, double* D, double* work, const SmallFast& F,
                    cudaStream_t st);

// Fast form: exact bf16 digit planes on tcgen05 (sliced.cu)
int slice_rows(int KS, const double* src, long R, int K, long rs, long ks, int Kpad, __nv_bfloat16* planes,
               int* exps, cudaStream_t st);
// rowmax: NULL, or max |hi| per row as float bits (from dress_dd)
int slice_rows_dd(int KS, const float2* src, long R, int K, long rs, long ks, int Kpad, __nv_bfloat16* planes,
                  int* exps, const unsigned* rowmax, cudaStream_t st);
// Arithmetic forms of the contraction kernel: exact digit planes, or the
// literal split-bf16 (3 terms) / tf32 (1 or 3 terms) products with float32
// accumulation of the precision study.
// FORM_DIGITS_T: the digit form with levels >= 3 accumulated per segment
// (fewer merges; the dressed rank-K update, whose merges scale every
// element by its segment's exponents, uses it).
enum { FORM_DIGITS = 0, FORM_BF16X3 = 1, FORM_TF32 = 2, FORM_DIGITS_T = 3 };
// N of the 128 x N output tiles of a form (KS: digit planes or literal parts)
int pair_tile_n(int form, int KS);
int pair_tile_bound(int BN, const Geometry& g, int npairs);
int pair_tiles(int BN, const Geometry& g, const int2* pairs, int npairs, bool energy_only, std::vector<int2>& out);
struct RegTables;
// Eq. A7 epilogue fused into the pair contraction (see sliced.cu)
struct PairEpilogue {
  const float2* hp;       // [nh np] eps_i - eps_a, double-float
  const RegTables* reg;   // regulariser tables of the device
  float s_hi, s_lo;       // flow parameter s, double-float
  float2* tau;            // [slot][nv][nv]
  float2* kap;            // [slot][nv][nv]
  double* ts;             // [nh][nh][nv][na] or null (energy only)
  int nv;
};
// nu (double-float [slot][np][np]) of a batch, or with `epi` its tau, kappa
// and ts directly (nu unused)
int sliced_pair_gemm(int KS, int form, const Geometry& g, const void* planes, const int* exps, int Kpad,
                     const int2* tiles, int ntiles, const int* slot_of, float2* nu, const PairEpilogue* epi, int* err,
                     cudaStream_t st);
// planes of a literal form: KS parts [KS][R][Kpad] (bf16 for FORM_BF16X3,
// float32 holding tf32 values for FORM_TF32), exps[R] = 0
int stage_literal(int form, int KS, const double* src, long R, int K, long rs, long ks, int Kpad, void* planes,
                  int* exps, cudaStream_t st);
// double-float elementwise stages (dd_stages.cu)
int eps_to_dd(int n, const double* eps, float2* out, cudaStream_t st);
int reg_tables_device(const RegTables** out);
bool fused_epilogue_enabled();
void set_syrk_planes(int k);
void set_fused_epilogue(bool on);
int hole_particle_dd(const Geometry& g, const double* eps, float2* out, cudaStream_t st);
int pair_epilogue_dd(const Geometry& g, const double* eps, const float2* eps_dd, const int2* pairs, int npairs,
                     const float2* nu, float2* tau, float2* kap, double* ts, cudaStream_t st);
// rowmax: NULL, or [nout][nv] zeroed words receiving max |hi| of each row of
// the dressed matrices written (float bits, atomicMax)
int dress_dd(const Geometry& g, const DressDesc* d_desc, int ndesc, int ncc, const DressAux& aux,
             const float2* tau, const float2* kap, float2* sig, double* sig_sign, double* e_part, bool want_sig,
             unsigned* rowmax, cudaStream_t st);
int regularize_test(int n, const double* delta, double s, double* r1, double* y, cudaStream_t st);
int sliced_syrk(int KS, int nv, int nr, const __nv_bfloat16* planes, const int* exps, int Kpad,
                const double* sign, double* dpart, int nsplit, double* D, int* err, cudaStream_t st);
int sliced_plain_gemm(int KS, int M, int N, const void* pa, const int* ea, const void* pb,
                      const int* eb, int Kpad, double* C, long ldc, int* err, cudaStream_t st, int form = FORM_DIGITS);
inline int pad64(int k) { return (k + 63) / 64 * 64; }

// Truncation and correction helpers (fno.cu)
int truncate_ons(int nv, const double* ons, int mode, double thr, double ratio, int* nkept,
                 cudaStream_t st);
int symmetrize(int n, double* D, cudaStream_t st);
int scale_rows(int nv, int ncol, long ld, const double* ev, const double* V, double* W,
               cudaStream_t st);
int copy_active(long rows, int na, int np, int npf, const double* B, double* Bf, cudaStream_t st);
int check_finite(const double* x, long n, int* flag, cudaStream_t st);
// Whether p is device (or managed) memory; cudaPointerGetAttributes allocates nothing.
bool is_device_ptr(const void* p);

// Full multi-reference PT2 energy beyond E_vv, float64 (energy_mr.cu).
// ks > 0: the integral GEMM on the digit-plane tensor-core path with ks planes (naux >= SLICED_MIN_K).
size_t mr_energy_work_doubles(const Geometry& g, int ks);
int mr_energy_rest(const Geometry& g, int ks, const double* B, const double* eps, const double* f_hp,
                   const double* g1, const double* l2, const double* l3, double* work, double* e_out,
                   cudaStream_t st);

// Single-instance pipeline stages on an explicit workspace (abi.cu); the C
// entry points call them on the per-device workspace, the batch runner on
// its workers' workspaces.  `budget`: device bytes a pass may plan for.
size_t device_budget(size_t held);
void release_batch_pools();  // batch.cu
int impl_pt2_energy(Workspace& ws, size_t budget, const dsrg_fno_problem* prob, double* e2_out, cudaStream_t st);
// E^(2) over every class: E_vv on the selected path plus mr_energy_rest; l3 may be null
int impl_pt2_energy_mr(Workspace& ws, size_t budget, const dsrg_fno_problem* prob, const double* l3, double* e2_out,
                       double* evv_out, cudaStream_t st);
// l3: device [nact]^6 3-cumulant for Eq. A12 term 13, or null (terms 1-12 only)
int impl_vv_opdm(Workspace& ws, size_t budget, const dsrg_fno_problem* prob, double* dvv_out, double* e2_out,
                 cudaStream_t st, const double* l3 = nullptr);
int impl_truncate(Workspace& ws, int32_t nvir, const double* dvv, int32_t mode, double threshold, double degen_ratio,
                  double* on_out, double* no_out, int32_t* nkept_out, cudaStream_t st);
// Full-energy form of the correction (dsrg_fno_discarded_correction_mr): l3 may be null.
struct CorrectionMR {
  const double* l3;
};
int impl_correction(Workspace& ws, size_t budget, const dsrg_fno_problem* prob, int32_t nkept, const double* no,
                    const double* e2_mo_in, double* de_out, double* e2_fno_out, double* eps_fno_out,
                    cudaStream_t st, const CorrectionMR* mr = nullptr);

}  // namespace dsrg
