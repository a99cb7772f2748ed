// C ABI of the FNO SA-DSRG-PT2 library: argument checks, the batch plan over
// hole-pair groups, workspace management and the order of the kernels.
#include <math.h>

#include <algorithm>
#include <atomic>
#include <vector>

#include "kernels.h"

namespace dsrg {

// ---------------------------------------------------------------------------
// Workspace
// ---------------------------------------------------------------------------
static std::mutex g_ws_mutex;
static Workspace g_ws[64];

std::mutex& workspace_mutex() { return g_ws_mutex; }

Workspace& workspace_for_current_device() {
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) dev = 0;
  g_ws[dev].device = dev;
  return g_ws[dev];
}

int ws_reserve(Workspace& ws, size_t bytes) {
  ws.off = 0;
  if (bytes <= ws.cap) return DSRG_FNO_OK;
  if (ws.base) {
    DSRG_CUDA(cudaDeviceSynchronize());
    DSRG_CUDA(cudaFree(ws.base));
    ws.base = nullptr;
    ws.cap = 0;
  }
  if (cudaMalloc(&ws.base, bytes) != cudaSuccess) {
    cudaGetLastError();
    ws.base = nullptr;
    return DSRG_FNO_ERR_NOMEM;
  }
  ws.cap = bytes;
  return DSRG_FNO_OK;
}

// ---------------------------------------------------------------------------
// Batch plan: hole-pair groups closed under the coupling of the hole 2-RDM
// ---------------------------------------------------------------------------
struct Batch {
  int pair_begin, npairs, desc_begin, ndesc;
  int nout;  // dressed matrices written (a core-core pair writes two)
  int ncc;   // leading work items that are core-core groups
};

struct Plan {
  std::vector<int2> pairs;
  std::vector<DressDesc> desc;
  std::vector<Batch> batches;
  int max_pairs = 0, max_desc = 0, max_out = 0;
};

static void build_plan(int nc, int na, long cap_pairs, Plan& P) {
  struct Group {
    std::vector<int2> pairs;
    int kind, nout;
  };
  std::vector<Group> groups;
  for (int m = 0; m < nc; ++m)
    for (int n = m; n < nc; ++n) {
      Group G;
      G.pairs.push_back(make_int2(m, n));
      G.kind = (m == n) ? GROUP_CC_DIAG : GROUP_CC_PAIR;
      G.nout = (m == n) ? 1 : 2;
      groups.push_back(G);
    }
  if (na > 0) {
    for (int m = 0; m < nc; ++m) {
      Group G;
      for (int u = 0; u < na; ++u) G.pairs.push_back(make_int2(m, nc + u));
      G.kind = GROUP_CA;
      G.nout = 2 * na;
      groups.push_back(G);
    }
    Group G;
    for (int u = 0; u < na; ++u)
      for (int v = u; v < na; ++v) G.pairs.push_back(make_int2(nc + u, nc + v));
    G.kind = GROUP_AA;
    G.nout = na * na;  // na (na + 1) / 2 symmetric + na (na - 1) / 2 antisymmetric
    groups.push_back(G);
  }
  long largest = 0;
  for (auto& G : groups) largest = std::max<long>(largest, (long)G.pairs.size());
  cap_pairs = std::max(cap_pairs, largest);
  Batch cur{0, 0, 0, 0, 0, 0};
  for (auto& G : groups) {
    if (cur.npairs > 0 && cur.npairs + (long)G.pairs.size() > cap_pairs) {
      P.batches.push_back(cur);
      cur = Batch{(int)P.pairs.size(), 0, (int)P.desc.size(), 0, 0, 0};
    }
    for (int o0 = 0; o0 < G.nout; o0 += DRESS_OC) {
      DressDesc d{};
      d.kind = G.kind;
      d.slot = cur.npairs;
      d.nslots = (int)G.pairs.size();
      d.out = cur.nout;
      d.o_begin = o0;
      d.o_count = std::min(DRESS_OC, G.nout - o0);
      d.m = G.pairs[0].x;
      P.desc.push_back(d);
      ++cur.ndesc;
      if (G.kind == GROUP_CC_DIAG || G.kind == GROUP_CC_PAIR) ++cur.ncc;
    }
    cur.nout += G.nout;
    for (auto p : G.pairs) P.pairs.push_back(p);
    cur.npairs += (int)G.pairs.size();
  }
  if (cur.npairs > 0) P.batches.push_back(cur);
  for (auto& b : P.batches) {
    P.max_pairs = std::max(P.max_pairs, b.npairs);
    P.max_desc = std::max(P.max_desc, b.ndesc);
    P.max_out = std::max(P.max_out, b.nout);
  }
}

// ---------------------------------------------------------------------------
// Argument checks
// ---------------------------------------------------------------------------
bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

static int validate(const dsrg_fno_problem* p) {
  if (!p) return DSRG_FNO_ERR_ARG;
  if (p->ncore < 0 || p->nact < 0 || p->nvir < 0 || p->naux < 0) return DSRG_FNO_ERR_ARG;
  if (p->nact > 16) return DSRG_FNO_ERR_UNSUPPORTED;
  if (p->ncore + p->nact == 0 || p->nvir == 0) return DSRG_FNO_ERR_ARG;
  if (!(p->s >= 0.0) || !isfinite(p->s)) return DSRG_FNO_ERR_ARG;
  if (p->precision < DSRG_FNO_FP64 || p->precision > DSRG_FNO_TF32) return DSRG_FNO_ERR_ARG;
  if (p->precision == DSRG_FNO_SLICED_BF16 && p->nslices != 0 && (p->nslices < 3 || p->nslices > 5))
    return DSRG_FNO_ERR_UNSUPPORTED;
  if (p->precision == DSRG_FNO_BF16X3 && p->nslices != 0 && p->nslices != 3) return DSRG_FNO_ERR_UNSUPPORTED;
  if (p->precision == DSRG_FNO_TF32 && p->nslices != 0 && p->nslices != 1 && p->nslices != 3)
    return DSRG_FNO_ERR_UNSUPPORTED;
  if (p->naux > 0 && !is_device_ptr(p->B_hp)) return DSRG_FNO_ERR_ARG;
  if (!is_device_ptr(p->eps)) return DSRG_FNO_ERR_ARG;
  if (p->nact > 0 && (!is_device_ptr(p->gamma1) || !is_device_ptr(p->lambda2))) return DSRG_FNO_ERR_ARG;
  if (p->f_hp && !is_device_ptr(p->f_hp)) return DSRG_FNO_ERR_ARG;
  if (p->nstates > 0) {
    if (!p->weights) return DSRG_FNO_ERR_ARG;
    double s = 0.0;
    for (int k = 0; k < p->nstates; ++k) {
      if (!(p->weights[k] >= 0.0)) return DSRG_FNO_ERR_ARG;
      s += p->weights[k];
    }
    if (fabs(s - 1.0) > 1e-12) return DSRG_FNO_ERR_ARG;
  }
  return DSRG_FNO_OK;
}

static int check_inputs_finite(const dsrg_fno_problem* p, int* flag, cudaStream_t st) {
  const long nh = p->ncore + p->nact, np = p->nact + p->nvir;
  DSRG_CUDA(cudaMemsetAsync(flag, 0, sizeof(int), st));
  DSRG_TRY(check_finite(p->B_hp, (long)p->naux * nh * np, flag, st));
  DSRG_TRY(check_finite(p->eps, nh + p->nvir, flag, st));
  if (p->nact) {
    DSRG_TRY(check_finite(p->gamma1, (long)p->nact * p->nact, flag, st));
    DSRG_TRY(check_finite(p->lambda2, (long)p->nact * p->nact * p->nact * p->nact, flag, st));
  }
  if (p->f_hp) DSRG_TRY(check_finite(p->f_hp, nh * np, flag, st));
  int h = 0;
  DSRG_CUDA(cudaMemcpyAsync(&h, flag, sizeof(int), cudaMemcpyDeviceToHost, st));
  DSRG_CUDA(cudaStreamSynchronize(st));
  return h ? DSRG_FNO_ERR_NONFINITE : DSRG_FNO_OK;
}

// ---------------------------------------------------------------------------
// One pass over the hole pairs: E_vv and, with want_d, the vv classes of D.
// ---------------------------------------------------------------------------
struct PassBuffers {
  int2* pairs;
  DressDesc* desc;
  double *tau, *kap, *sig, *sig_sign, *e_part, *dpart, *ts, *e_acc;
  double *g1A, *g1V, *g1W, *MsA, *MsV, *MsW, *MaA, *MaV, *MaW;
  int* status;
  int nsplit;
  // fast form
  int ks;             // digit planes (0 = float64 form)
  int ks_d;           // digit planes of the dressed matrices (rank-K update)
  int2 pform;         // form and parts of the B.B contraction
  int kpad_q, kpad_v; // padded contraction lengths (naux, nvir)
  __nv_bfloat16 *planes_b, *planes_s;
  int *exps_b, *exps_s, *err;
  float2* nu;        // double-float contraction tiles
  float2* eps_dd;    // orbital energies as double-float
  unsigned* rowmax;  // max |hi| per row of the dressed matrices (float bits)
  float2* hp;        // [nh np] eps_i - eps_a, double-float (fused epilogue)
  const RegTables* reg;
  bool fused;        // Eq. A7 epilogue inside the contraction kernel
  int2* tiles;       // output tiles of the pair contraction, all batches
  int* slot_of;      // [batch][nh][nh] slot of pair (i, j) in the batch, -1 outside
  std::vector<long> tile_begin;
  std::vector<int> tile_count;
};

// In the fast form tau, kappa and the dressed matrices are double-float
// (float2, the same 8 bytes per element as the float64 form's buffers).
static float2* as_dd(double* p) { return reinterpret_cast<float2*>(p); }

static const int DEFAULT_SLICES = 5;

// The Eq. A7 epilogue runs as its own kernel after the contraction (the
// default: on GB300 the regulariser's 48 evaluations per thread at the end of
// every tile, on the contraction kernel's four merge warps, stall the MMAs:
// pair contraction 335 -> 554 ms per C2 solve, against 41 ms for the
// separate kernel), or inside the contraction kernel's output stage.
static std::atomic<int> g_fused_epilogue{0};
bool fused_epilogue_enabled() { return g_fused_epilogue.load() != 0; }
void set_fused_epilogue(bool on) { g_fused_epilogue.store(on ? 1 : 0); }

// Digit planes of the fast-form stages (0 = float64 form).  The literal
// forms of the precision study run every stage but the B.B contraction as
// the default fast form.
static int slices_of(const dsrg_fno_problem* p) {
  if (p->precision == DSRG_FNO_FP64) return 0;
  if (p->precision != DSRG_FNO_SLICED_BF16) return DEFAULT_SLICES;
  return p->nslices ? p->nslices : DEFAULT_SLICES;
}

// Digit planes of the dressed matrices in the rank-K update of D_vv: those
// of the problem, unless a test hook sets fewer.  (4 planes, which would save
// a third of the update's digit products, were measured to miss the 1e-8
// tolerance on the occupation numbers: 1.8e-8 on the single-reference nvir 90
// workload, whose dressed rows hold elements far below their row maximum.)
static std::atomic<int> g_syrk_planes{0};
void set_syrk_planes(int k) { g_syrk_planes.store(k); }
static int syrk_slices(int ks) {
  const int f = g_syrk_planes.load();
  if (f >= 3 && f <= 5) return std::min(f, ks);
  return ks;
}

// Form and parts of the B.B contraction: {FORM_DIGITS, ks}, {FORM_BF16X3, 2},
// {FORM_TF32, 1 or 2}.
static int2 pair_form_of(const dsrg_fno_problem* p, int ks) {
  if (p->precision == DSRG_FNO_BF16X3) return make_int2(FORM_BF16X3, 2);
  if (p->precision == DSRG_FNO_TF32) return make_int2(FORM_TF32, p->nslices == 1 ? 1 : 2);
  return make_int2(FORM_DIGITS, ks);
}

static size_t doubles(size_t n) { return ws_bytes(n, sizeof(double)); }

static long pair_cap_for_budget(int nv, int np, int ks, size_t budget) {
  // tau + kappa + two dressed matrices per pair (+ nu and the dressed planes in the fast form)
  double per_pair = 4.0 * (double)nv * nv * 8.0 + 1024.0;
  if (ks) per_pair += (double)np * np * 8.0 + 2.0 * ks * 2.0 * (double)nv * (nv + 64);
  long cap = (long)(budget / per_pair);
  return std::max<long>(cap, 1);
}

// 45 % of the free device memory, counting `held` bytes that the caller's
// own workspaces already occupy as free (capped at 96 GB): the plan of a pass
// then does not depend on what earlier calls allocated.
size_t device_budget(size_t held) {
  size_t fr = 0, tot = 0;
  if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
    cudaGetLastError();
    return (size_t)4 << 30;
  }
  size_t b = (size_t)(0.45 * (double)(fr + held));
  return std::min(b, (size_t)96 << 30);
}

static size_t plan_budget(const Workspace& ws) { return device_budget(ws.cap); }

static int run_pass(const Geometry& g, const double* B, const double* eps, const double* gamma1,
                    const double* lambda2, const Plan& P, PassBuffers& W, bool want_d, double* D,
                    cudaStream_t st) {
  const int na = g.na;
  DressAux aux{};
  if (na > 0) {
    DSRG_PHASE("phase_density_eigen", st);
    const int ns = na * (na + 1) / 2, nd = na * (na - 1) / 2;
    DSRG_CUDA(cudaMemcpyAsync(W.g1A, gamma1, sizeof(double) * na * na, cudaMemcpyDeviceToDevice, st));
    DSRG_TRY(aa_blocks(na, gamma1, lambda2, W.MsA, W.MaA, st));
    // Gamma1 and the two aa blocks of the hole 2-RDM, solved together
    const int nn[3] = {na, ns, nd};
    double* const AA[3] = {W.g1A, W.MsA, W.MaA};
    double* const VV[3] = {W.g1V, W.MsV, W.MaV};
    double* const WW[3] = {W.g1W, W.MsW, W.MaW};
    DSRG_TRY(eig_sym_jacobi_batch(3, nn, AA, VV, WW, W.status, 60, st));
    aux.g1_evec = W.g1V;
    aux.g1_eval = W.g1A;
    aux.aas_evec = W.MsV;
    aux.aas_eval = W.MsA;
    aux.aaa_evec = W.MaV;
    aux.aaa_eval = W.MaA;
  }
  const int ntd = ceil_div(g.nv, 32);
  if (W.ks) {
    // digit planes of B: rows (hole, particle), contraction over Q
    const long rows = (long)g.nh * g.np;
    DSRG_PHASE("phase_stage_b", st);
    if (W.pform.x == FORM_DIGITS)
      DSRG_TRY(slice_rows(W.ks, B, rows, g.nq, 1, rows, W.kpad_q, W.planes_b, W.exps_b, st));
    else
      DSRG_TRY(stage_literal(W.pform.x, W.pform.y, B, rows, g.nq, 1, rows, W.kpad_q, W.planes_b, W.exps_b, st));
    DSRG_TRY(eps_to_dd(g.nh + g.nv, eps, W.eps_dd, st));
    if (W.fused) DSRG_TRY(hole_particle_dd(g, eps, W.hp, st));
  }
  for (size_t bi = 0; bi < P.batches.size(); ++bi) {
    const Batch& b = P.batches[bi];
    double* ts = want_d ? W.ts : nullptr;
    if (W.ks && W.fused) {
      PairEpilogue epi{};
      epi.hp = W.hp;
      epi.reg = W.reg;
      const float sh = (float)g.s;
      epi.s_hi = sh;
      epi.s_lo = (float)(g.s - (double)sh);
      epi.tau = as_dd(W.tau);
      epi.kap = as_dd(W.kap);
      epi.ts = ts;
      epi.nv = g.nv;
      DSRG_TRY(sliced_pair_gemm(W.pform.y, W.pform.x, g, W.planes_b, W.exps_b, W.kpad_q, W.tiles + W.tile_begin[bi],
                                W.tile_count[bi], W.slot_of + bi * (size_t)g.nh * g.nh, nullptr, &epi, W.err, st));
    } else if (W.ks) {
      DSRG_TRY(sliced_pair_gemm(W.pform.y, W.pform.x, g, W.planes_b, W.exps_b, W.kpad_q, W.tiles + W.tile_begin[bi],
                                W.tile_count[bi], W.slot_of + bi * (size_t)g.nh * g.nh, W.nu, nullptr, W.err, st));
      DSRG_PHASE("phase_pair_epilogue", st);
      DSRG_TRY(pair_epilogue_dd(g, eps, W.eps_dd, W.pairs + b.pair_begin, b.npairs, W.nu, as_dd(W.tau),
                                as_dd(W.kap), ts, st));
    } else {
      DSRG_TRY(pair_gemm_f64(g, B, eps, W.pairs + b.pair_begin, b.npairs, W.tau, W.kap, ts, st));
    }
    {
      DSRG_PHASE("phase_dress", st);
      if (W.ks) {
        unsigned* rm = want_d ? W.rowmax : nullptr;
        if (rm) DSRG_CUDA(cudaMemsetAsync(rm, 0, sizeof(unsigned) * (size_t)b.nout * g.nv, st));
        DSRG_TRY(dress_dd(g, W.desc + b.desc_begin, b.ndesc, b.ncc, aux, as_dd(W.tau), as_dd(W.kap), as_dd(W.sig),
                          W.sig_sign, W.e_part, want_d, rm, st));
      } else {
        DSRG_TRY(dress_f64(g, W.desc + b.desc_begin, b.ndesc, b.ncc, aux, W.tau, W.kap, W.sig, W.sig_sign,
                           W.e_part, want_d, st));
      }
    }
    DSRG_TRY(ordered_sum(W.e_part, (long)b.ndesc * DRESS_TILE_BLOCKS, W.e_acc, bi > 0, st));
    if (want_d) {
      if (W.ks) {
        const long rows = (long)b.nout * g.nv;
        {
          DSRG_PHASE("phase_stage_sig", st);
          DSRG_TRY(slice_rows_dd(W.ks_d, as_dd(W.sig), rows, g.nv, g.nv, 1, W.kpad_v, W.planes_s, W.exps_s, W.rowmax,
                                 st));
        }
        DSRG_TRY(sliced_syrk(W.ks_d, g.nv, b.nout, W.planes_s, W.exps_s, W.kpad_v, W.sig_sign, W.dpart, W.nsplit, D,
                             W.err, st));
      } else {
        DSRG_TRY(syrk_dressed_f64(g.nv, b.nout, W.sig, W.sig_sign, W.dpart, W.nsplit, D, st));
      }
    }
  }
  if (P.batches.empty()) DSRG_CUDA(cudaMemsetAsync(W.e_acc, 0, sizeof(double), st));
  return DSRG_FNO_OK;
}

// Split of the dressed rank-K update over the dressed matrices: enough
// upper-triangle tile jobs for two waves of the SMs, and a count that fills
// its last wave (jobs = tiles x splits, the persistent grid has one CTA per SM).
static int nsplit_for(int nv, int ndesc, int ks) {
  int tiles;
  if (ks) {  // 128 x BN tiles of the digit-plane kernel with some f >= e
    const int bm = 128, bn = ks == 5 ? 48 : 64;
    const int ntm = ceil_div(nv, bm), ntn = ceil_div(nv, bn);
    tiles = 0;
    for (int m = 0; m < ntm; ++m) tiles += ntn - (m * bm) / bn;
  } else {   // 64 x 64 upper tiles of the float64 kernel
    const int nt = ceil_div(nv, 64);
    tiles = nt * (nt + 1) / 2;
  }
  const int sms = 152;
  const int cap = std::max(1, std::min(16, ndesc));
  int best = std::min(cap, std::max(1, ceil_div(2L * sms, tiles)));
  double best_eff = 0.0;
  for (int ns = best; ns <= cap; ++ns) {
    const long jobs = (long)tiles * ns;
    const double eff = (double)jobs / ((double)ceil_div(jobs, (long)sms) * sms);
    if (eff > best_eff + 1e-9) {
      best_eff = eff;
      best = ns;
    }
    if (eff >= 0.97) break;
  }
  return best;
}

// Carves the pass buffers out of the workspace (sizes must match pass_bytes).
static size_t pass_bytes(const Geometry& g, const Plan& P, bool want_d, int nsplit, int ks, int2 pform) {
  const size_t nv2 = (size_t)g.nv * g.nv;
  const int na = g.na, ns = na * (na + 1) / 2, nd = na * (na - 1) / 2;
  const int ntd = ceil_div(g.nv, 32);
  size_t b = 0;
  b += ws_bytes(P.pairs.size(), sizeof(int2));
  b += ws_bytes(P.desc.size(), sizeof(DressDesc));
  b += 2 * doubles((size_t)P.max_pairs * nv2);
  b += doubles(want_d ? (size_t)P.max_out * nv2 : 1);
  b += doubles((size_t)P.max_out + 1);
  b += doubles((size_t)P.max_desc * DRESS_TILE_BLOCKS + 1);
  b += doubles(want_d ? (size_t)nsplit * nv2 : 1);
  b += doubles(want_d && na ? (size_t)g.nh * g.nh * g.nv * na : 1);
  b += doubles(8);
  b += 3 * doubles((size_t)na * na + 1) + doubles(eig_work_doubles(na));
  b += 2 * doubles((size_t)ns * ns + 1) + doubles(eig_work_doubles(ns));
  b += 2 * doubles((size_t)nd * nd + 1) + doubles(eig_work_doubles(nd));
  b += ws_bytes(16, sizeof(int));
  if (ks) {
    const size_t rows = (size_t)g.nh * g.np;
    b += ws_bytes((size_t)ks * rows * pad64(g.nq), 2) + ws_bytes(rows, sizeof(int));
    b += doubles((size_t)P.max_pairs * g.np * g.np);
    b += doubles((size_t)g.nh + g.nv);
    b += doubles((size_t)g.nh * g.np);
    if (want_d)
      b += ws_bytes((size_t)ks * P.max_out * g.nv * pad64(g.nv), 2) + 2 * ws_bytes((size_t)P.max_out * g.nv, sizeof(int));
    b += ws_bytes(8, sizeof(int));
    size_t tiles = 0;
    const int bn = pair_tile_n(pform.x, pform.y);
    for (const Batch& bt : P.batches) tiles += (size_t)pair_tile_bound(bn, g, bt.npairs);
    b += ws_bytes(tiles + 1, sizeof(int2)) + ws_bytes(P.batches.size() * (size_t)g.nh * g.nh + 1, sizeof(int));
  }
  return b;
}

static int carve_pass(Workspace& ws, const Geometry& g, const Plan& P, bool want_d, int nsplit, int ks, int2 pform,
                      PassBuffers& W, cudaStream_t st) {
  const size_t nv2 = (size_t)g.nv * g.nv;
  const int na = g.na, ns = na * (na + 1) / 2, nd = na * (na - 1) / 2;
  const int ntd = ceil_div(g.nv, 32);
  W.pairs = ws_take<int2>(ws, P.pairs.size());
  W.desc = ws_take<DressDesc>(ws, P.desc.size());
  W.tau = ws_take<double>(ws, (size_t)P.max_pairs * nv2);
  W.kap = ws_take<double>(ws, (size_t)P.max_pairs * nv2);
  W.sig = ws_take<double>(ws, want_d ? (size_t)P.max_out * nv2 : 1);
  W.sig_sign = ws_take<double>(ws, (size_t)P.max_out + 1);
  W.e_part = ws_take<double>(ws, (size_t)P.max_desc * DRESS_TILE_BLOCKS + 1);
  W.dpart = ws_take<double>(ws, want_d ? (size_t)nsplit * nv2 : 1);
  W.ts = ws_take<double>(ws, want_d && na ? (size_t)g.nh * g.nh * g.nv * na : 1);
  W.e_acc = ws_take<double>(ws, 8);
  W.g1A = ws_take<double>(ws, (size_t)na * na + 1);
  W.g1V = ws_take<double>(ws, (size_t)na * na + 1);
  W.g1W = ws_take<double>(ws, eig_work_doubles(na));
  (void)ws_take<double>(ws, (size_t)na * na + 1);
  W.MsA = ws_take<double>(ws, (size_t)ns * ns + 1);
  W.MsV = ws_take<double>(ws, (size_t)ns * ns + 1);
  W.MsW = ws_take<double>(ws, eig_work_doubles(ns));
  W.MaA = ws_take<double>(ws, (size_t)nd * nd + 1);
  W.MaV = ws_take<double>(ws, (size_t)nd * nd + 1);
  W.MaW = ws_take<double>(ws, eig_work_doubles(nd));
  W.status = ws_take<int>(ws, 16);  // 4 per density eigensolve
  W.nsplit = nsplit;
  if (!W.status) return DSRG_FNO_ERR_NOMEM;
  W.ks = ks;
  W.ks_d = ks ? syrk_slices(ks) : 0;
  W.pform = pform;
  if (ks) {
    const size_t rows = (size_t)g.nh * g.np;
    W.kpad_q = pad64(g.nq);
    W.kpad_v = pad64(g.nv);
    W.planes_b = ws_take<__nv_bfloat16>(ws, (size_t)ks * rows * W.kpad_q);
    W.exps_b = ws_take<int>(ws, rows);
    W.nu = ws_take<float2>(ws, (size_t)P.max_pairs * g.np * g.np);
    W.eps_dd = ws_take<float2>(ws, (size_t)g.nh + g.nv);
    W.hp = ws_take<float2>(ws, (size_t)g.nh * g.np);
    W.fused = fused_epilogue_enabled();
    if (W.fused) DSRG_TRY(reg_tables_device(&W.reg));
    if (want_d) {
      W.planes_s = ws_take<__nv_bfloat16>(ws, (size_t)ks * P.max_out * g.nv * W.kpad_v);
      W.exps_s = ws_take<int>(ws, (size_t)P.max_out * g.nv);
      W.rowmax = ws_take<unsigned>(ws, (size_t)P.max_out * g.nv);
    }
    W.err = ws_take<int>(ws, 8);
    if (!W.err) return DSRG_FNO_ERR_NOMEM;
    DSRG_CUDA(cudaMemsetAsync(W.err, 0, sizeof(int), st));
    // output tiles and slot tables of every batch (host lists, one upload)
    std::vector<int2> all, one;
    std::vector<int> slots(P.batches.size() * (size_t)g.nh * g.nh, -1);
    size_t bound = 0;
    const int bn = pair_tile_n(pform.x, pform.y);
    for (size_t bi = 0; bi < P.batches.size(); ++bi) {
      const Batch& b = P.batches[bi];
      bound += (size_t)pair_tile_bound(bn, g, b.npairs);
      DSRG_TRY(pair_tiles(bn, g, P.pairs.data() + b.pair_begin, b.npairs, !want_d, one));
      W.tile_begin.push_back((long)all.size());
      W.tile_count.push_back((int)one.size());
      all.insert(all.end(), one.begin(), one.end());
      int* sl = slots.data() + bi * (size_t)g.nh * g.nh;
      for (int k = 0; k < b.npairs; ++k) {
        const int2 pr = P.pairs[b.pair_begin + k];
        sl[(size_t)pr.x * g.nh + pr.y] = k;
      }
    }
    W.tiles = ws_take<int2>(ws, bound + 1);
    W.slot_of = ws_take<int>(ws, slots.size() + 1);
    if (!W.slot_of || all.size() > bound) return DSRG_FNO_ERR_NOMEM;
    if (!all.empty())
      DSRG_CUDA(cudaMemcpyAsync(W.tiles, all.data(), all.size() * sizeof(int2), cudaMemcpyHostToDevice, st));
    if (!slots.empty())
      DSRG_CUDA(cudaMemcpyAsync(W.slot_of, slots.data(), slots.size() * sizeof(int), cudaMemcpyHostToDevice, st));
  }
  if (!P.pairs.empty())
    DSRG_CUDA(cudaMemcpyAsync(W.pairs, P.pairs.data(), P.pairs.size() * sizeof(int2), cudaMemcpyHostToDevice, st));
  if (!P.desc.empty())
    DSRG_CUDA(cudaMemcpyAsync(W.desc, P.desc.data(), P.desc.size() * sizeof(DressDesc), cudaMemcpyHostToDevice,
                              st));
  return DSRG_FNO_OK;
}

static Geometry geometry_of(const dsrg_fno_problem* p) {
  Geometry g;
  g.nc = p->ncore;
  g.na = p->nact;
  g.nv = p->nvir;
  g.nq = p->naux;
  g.nh = p->ncore + p->nact;
  g.np = p->nact + p->nvir;
  g.s = p->s;
  return g;
}

static int read_error_flag(const int* err, cudaStream_t st) {
  if (!err) return DSRG_FNO_OK;
  int h = 0;
  DSRG_CUDA(cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, st));
  DSRG_CUDA(cudaStreamSynchronize(st));
  return h ? DSRG_FNO_ERR_TIMEOUT : DSRG_FNO_OK;
}

// Energy-only pass for an arbitrary geometry (used for the MO and FNO bases).
static int energy_pass(const Geometry& g, int ks, int2 pform, const double* B, const double* eps, const double* gamma1,
                       const double* lambda2, Workspace& ws, size_t base_off, size_t budget, double* e_out,
                       cudaStream_t st) {
  Plan P;
  build_plan(g.nc, g.na, pair_cap_for_budget(g.nv, g.np, ks, budget), P);
  ws.off = base_off;
  PassBuffers W{};
  size_t need = base_off + pass_bytes(g, P, false, 1, ks, pform);
  if (need > ws.cap) return DSRG_FNO_ERR_NOMEM;
  DSRG_TRY(carve_pass(ws, g, P, false, 1, ks, pform, W, st));
  DSRG_TRY(run_pass(g, B, eps, gamma1, lambda2, P, W, false, nullptr, st));
  DSRG_CUDA(cudaMemcpyAsync(e_out, W.e_acc, sizeof(double), cudaMemcpyDeviceToHost, st));
  DSRG_CUDA(cudaStreamSynchronize(st));
  return read_error_flag(W.err, st);
}

static size_t energy_pass_bytes(const Geometry& g, int ks, int2 pform, size_t budget) {
  Plan P;
  build_plan(g.nc, g.na, pair_cap_for_budget(g.nv, g.np, ks, budget), P);
  return pass_bytes(g, P, false, 1, ks, pform);
}

int impl_pt2_energy(Workspace& ws, size_t budget, const dsrg_fno_problem* prob, double* e2_out, cudaStream_t st) {
  int s = validate(prob);
  if (s) return s;
  if (!e2_out) return DSRG_FNO_ERR_ARG;
  const Geometry g = geometry_of(prob);
  const int ks = slices_of(prob);
  const int2 pform = pair_form_of(prob, ks);
  DSRG_TRY(ws_reserve(ws, energy_pass_bytes(g, ks, pform, budget) + ws_bytes(8, sizeof(int))));
  int* flag = ws_take<int>(ws, 8);
  DSRG_TRY(check_inputs_finite(prob, flag, st));
  return energy_pass(g, ks, pform, prob->B_hp, prob->eps, prob->gamma1, prob->lambda2, ws, ws.off, budget, e2_out,
                     st);
}

int impl_pt2_energy_mr(Workspace& ws, size_t budget, const dsrg_fno_problem* prob, const double* l3, double* e2_out,
                       double* evv_out, cudaStream_t st) {
  int s = validate(prob);
  if (s) return s;
  if (!e2_out) return DSRG_FNO_ERR_ARG;
  if (prob->nact == 0) l3 = nullptr;
  if (l3 && !is_device_ptr(l3)) return DSRG_FNO_ERR_ARG;
  const Geometry g = geometry_of(prob);
  const int ks = slices_of(prob);
  const int2 pform = pair_form_of(prob, ks);
  const size_t mr = mr_energy_work_doubles(g, ks);
  DSRG_TRY(ws_reserve(ws, ws_bytes(8, sizeof(int)) + std::max(energy_pass_bytes(g, ks, pform, budget), doubles(mr))));
  int* flag = ws_take<int>(ws, 8);
  DSRG_TRY(check_inputs_finite(prob, flag, st));
  if (l3) {
    const long n3 = (long)g.na * g.na * g.na;
    int h = 0;
    DSRG_TRY(check_finite(l3, n3 * n3, flag, st));
    DSRG_CUDA(cudaMemcpyAsync(&h, flag, sizeof(int), cudaMemcpyDeviceToHost, st));
    DSRG_CUDA(cudaStreamSynchronize(st));
    if (h) return DSRG_FNO_ERR_NONFINITE;
  }
  const size_t base = ws.off;
  double evv = 0.0;
  DSRG_TRY(energy_pass(g, ks, pform, prob->B_hp, prob->eps, prob->gamma1, prob->lambda2, ws, base, budget, &evv, st));
  ws.off = base;
  double* work = ws_take<double>(ws, mr);
  if (!work) return DSRG_FNO_ERR_NOMEM;
  double rest = 0.0;
  DSRG_TRY(mr_energy_rest(g, ks, prob->B_hp, prob->eps, prob->f_hp, prob->gamma1, prob->lambda2, l3, work, &rest, st));
  if (!isfinite(evv) || !isfinite(rest)) return DSRG_FNO_ERR_NONFINITE;
  *e2_out = evv + rest;
  if (evv_out) *evv_out = evv;
  return DSRG_FNO_OK;
}

int impl_vv_opdm(Workspace& ws, size_t budget, const dsrg_fno_problem* prob, double* dvv_out, double* e2_out,
                 cudaStream_t st, const double* l3) {
  int s = validate(prob);
  if (s) return s;
  if (!dvv_out || !is_device_ptr(dvv_out)) return DSRG_FNO_ERR_ARG;
  if (prob->nact == 0) l3 = nullptr;
  if (l3 && !is_device_ptr(l3)) return DSRG_FNO_ERR_ARG;
  const Geometry g = geometry_of(prob);
  const int ks = slices_of(prob);
  Plan P;
  build_plan(g.nc, g.na, pair_cap_for_budget(g.nv, g.np, ks, budget), P);
  const int nsplit = nsplit_for(g.nv, P.max_out, ks ? syrk_slices(ks) : 0);
  const size_t small = small_terms_work_doubles(g.nc, g.na, g.nv);
  const int kmax = small_terms_kmax(g.nc, g.na);
  const bool small_fast = ks > 0 && kmax >= SLICED_MIN_K;
  const size_t small_fast_bytes =
      small_fast ? ws_bytes(2 * (size_t)ks * g.nv * pad64(kmax), 2) + ws_bytes(2 * (size_t)g.nv, sizeof(int)) +
                       doubles((size_t)g.nv * g.nv) + ws_bytes(8, sizeof(int))
                 : 0;
  const int2 pform = pair_form_of(prob, ks);
  size_t need = ws_bytes(8, sizeof(int)) + pass_bytes(g, P, true, nsplit, ks, pform) + doubles((size_t)g.nh * g.nv) +
                doubles(small + 1) + small_fast_bytes;
  DSRG_TRY(ws_reserve(ws, need));
  int* flag = ws_take<int>(ws, 8);
  DSRG_TRY(check_inputs_finite(prob, flag, st));
  if (l3) {
    const long n3 = (long)g.na * g.na * g.na;
    int h = 0;
    DSRG_TRY(check_finite(l3, n3 * n3, flag, st));
    DSRG_CUDA(cudaMemcpyAsync(&h, flag, sizeof(int), cudaMemcpyDeviceToHost, st));
    DSRG_CUDA(cudaStreamSynchronize(st));
    if (h) return DSRG_FNO_ERR_NONFINITE;
  }
  PassBuffers W{};
  DSRG_TRY(carve_pass(ws, g, P, true, nsplit, ks, pform, W, st));
  double* t1 = ws_take<double>(ws, (size_t)g.nh * g.nv);
  double* work = ws_take<double>(ws, small + 1);
  SmallFast sf{0, nullptr, nullptr, nullptr, nullptr};
  if (small_fast) {
    sf.ks = ks;
    sf.planes = ws_take<__nv_bfloat16>(ws, 2 * (size_t)ks * g.nv * pad64(kmax));
    sf.exps = ws_take<int>(ws, 2 * (size_t)g.nv);
    sf.cbuf = ws_take<double>(ws, (size_t)g.nv * g.nv);
    sf.err = W.err;
  }
  const size_t nv2 = (size_t)g.nv * g.nv;
  DSRG_CUDA(cudaMemsetAsync(dvv_out, 0, nv2 * sizeof(double), st));
  DSRG_TRY(run_pass(g, prob->B_hp, prob->eps, prob->gamma1, prob->lambda2, P, W, true, dvv_out, st));
  if (g.na > 0 || prob->f_hp) {
    DSRG_PHASE("phase_small_terms", st);
    DSRG_TRY(t1_amplitudes(g, g.na ? W.ts : nullptr, prob->eps, prob->f_hp, prob->gamma1, t1, st));
    DSRG_TRY(small_terms_f64(g, g.na ? W.ts : nullptr, t1, prob->gamma1, prob->lambda2, l3, dvv_out, work, sf, st));
  }
  DSRG_TRY(symmetrize(g.nv, dvv_out, st));
  DSRG_CUDA(cudaMemsetAsync(flag, 0, sizeof(int), st));
  DSRG_TRY(check_finite(dvv_out, (long)nv2, flag, st));
  double e = 0.0;
  int h = 0;
  DSRG_CUDA(cudaMemcpyAsync(&e, W.e_acc, sizeof(double), cudaMemcpyDeviceToHost, st));
  DSRG_CUDA(cudaMemcpyAsync(&h, flag, sizeof(int), cudaMemcpyDeviceToHost, st));
  DSRG_CUDA(cudaStreamSynchronize(st));
  DSRG_TRY(read_error_flag(W.err, st));
  if (h || !isfinite(e)) return DSRG_FNO_ERR_NONFINITE;
  if (e2_out) *e2_out = e;
  return DSRG_FNO_OK;
}

int impl_truncate(Workspace& ws, int32_t nvir, const double* dvv, int32_t mode, double threshold,
                         double degen_ratio, double* on_out, double* no_out, int32_t* nkept_out, cudaStream_t st) {
  if (nvir <= 0 || !dvv || !on_out || !no_out || !nkept_out) return DSRG_FNO_ERR_ARG;
  if (mode < 0 || mode > 3 || !isfinite(threshold) || !(degen_ratio >= 0.0)) return DSRG_FNO_ERR_ARG;
  if (!is_device_ptr(dvv) || !is_device_ptr(on_out) || !is_device_ptr(no_out)) return DSRG_FNO_ERR_ARG;
  const size_t n2 = (size_t)nvir * nvir;
  DSRG_TRY(ws_reserve(ws, 2 * doubles(n2) + doubles(eig_work_doubles(nvir)) + ws_bytes(nvir + 8, sizeof(int))));
  double* A = ws_take<double>(ws, n2);
  double* V = ws_take<double>(ws, n2);
  double* work = ws_take<double>(ws, eig_work_doubles(nvir));
  int* ib = ws_take<int>(ws, nvir + 8);
  int* status = ib;  // four words
  int* nk = ib + 4;
  int* rank = ib + 8;
  DSRG_CUDA(cudaMemcpyAsync(A, dvv, n2 * sizeof(double), cudaMemcpyDeviceToDevice, st));
  DSRG_PHASE("phase_no_eigen", st);
  int s = eig_sym_jacobi(nvir, A, V, work, status, 60, st);
  if (s) return s;
  DSRG_TRY(eig_sort(nvir, A, V, on_out, no_out, rank, true, true, st));
  DSRG_TRY(truncate_ons(nvir, on_out, mode, threshold, degen_ratio, nk, st));
  int h = 0;
  DSRG_CUDA(cudaMemcpyAsync(&h, nk, sizeof(int), cudaMemcpyDeviceToHost, st));
  DSRG_CUDA(cudaStreamSynchronize(st));
  *nkept_out = h;
  return DSRG_FNO_OK;
}

int impl_correction(Workspace& ws, size_t budget, const dsrg_fno_problem* prob, int32_t nkept,
                           const double* no, const double* e2_mo_in, double* de_out, double* e2_fno_out,
                           double* eps_fno_out, cudaStream_t st, const CorrectionMR* mr) {
  int s = validate(prob);
  if (s) return s;
  if (!de_out || !no || nkept < 0 || nkept > prob->nvir || !is_device_ptr(no)) return DSRG_FNO_ERR_ARG;
  if (eps_fno_out && !is_device_ptr(eps_fno_out)) return DSRG_FNO_ERR_ARG;
  const Geometry g = geometry_of(prob);
  Geometry gf = g;
  gf.nv = nkept;
  gf.np = g.na + nkept;
  const int nk = nkept, nv = g.nv;
  const size_t nk2 = (size_t)nk * nk;
  const long rows = (long)g.nq * g.nh;
  size_t fixed = ws_bytes(8, sizeof(int)) + doubles((size_t)nv * nk) * 2 + doubles(nk2) * 3 + doubles(eig_work_doubles(nk)) +
                 ws_bytes(nk + 8, sizeof(int)) + doubles((size_t)rows * gf.np + 1) + doubles(g.nh + nk + 1) +
                 doubles(nk + 1);
  const int ks = slices_of(prob);
  const int2 pform = pair_form_of(prob, ks);
  size_t pass_mo = e2_mo_in ? 0 : energy_pass_bytes(g, ks, pform, budget);
  size_t pass_f = nk > 0 ? energy_pass_bytes(gf, ks, pform, budget) : 0;
  const int kpv = pad64(nv);
  // B' = B U enters E_vv(FNO) element by element and Delta E is a difference
  // of two large energies: the rotation takes 6 digit planes (47 fraction
  // bits) in the fast form, the passes themselves keep ks.
  const int kx = ks ? 6 : 0;
  size_t xform = 0;
  if (kx && nk > 0)
    xform = ws_bytes((size_t)kx * rows * kpv, 2) + ws_bytes(rows, sizeof(int)) + ws_bytes((size_t)kx * nk * kpv, 2) +
            ws_bytes(nk, sizeof(int)) + ws_bytes(8, sizeof(int));
  // full-energy form: the rest terms of both bases (their work overlaps the passes) and f_hp rotated
  const size_t mr_work = mr ? doubles(mr_energy_work_doubles(g, ks)) : 0;
  const size_t ff_bytes = mr ? doubles((size_t)g.nh * gf.np + 1) : 0;
  DSRG_TRY(ws_reserve(ws, fixed + ff_bytes + std::max(std::max(pass_mo, pass_f), std::max(xform, mr_work))));
  int* flag = ws_take<int>(ws, 8);
  DSRG_TRY(check_inputs_finite(prob, flag, st));
  if (mr && mr->l3) {
    const long n3 = (long)g.na * g.na * g.na;
    int h = 0;
    DSRG_TRY(check_finite(mr->l3, n3 * n3, flag, st));
    DSRG_CUDA(cudaMemcpyAsync(&h, flag, sizeof(int), cudaMemcpyDeviceToHost, st));
    DSRG_CUDA(cudaStreamSynchronize(st));
    if (h) return DSRG_FNO_ERR_NONFINITE;
  }
  double* Wt = ws_take<double>(ws, (size_t)nv * nk);
  double* U = ws_take<double>(ws, (size_t)nv * nk);
  double* F = ws_take<double>(ws, nk2);
  double* FV = ws_take<double>(ws, nk2);
  double* Wsort = ws_take<double>(ws, nk2);
  double* work = ws_take<double>(ws, eig_work_doubles(nk));
  int* ib = ws_take<int>(ws, nk + 8);
  double* Bf = ws_take<double>(ws, (size_t)rows * gf.np + 1);
  double* epsf = ws_take<double>(ws, g.nh + nk + 1);
  double* evals = ws_take<double>(ws, nk + 1);
  double* ff = mr ? ws_take<double>(ws, (size_t)g.nh * gf.np + 1) : nullptr;
  const size_t base = ws.off;
  double e_mo = 0.0;
  if (e2_mo_in) e_mo = *e2_mo_in;
  else {
    DSRG_TRY(energy_pass(g, ks, pform, prob->B_hp, prob->eps, prob->gamma1, prob->lambda2, ws, base, budget, &e_mo,
                         st));
    if (mr) {
      ws.off = base;
      double* work = ws_take<double>(ws, mr_energy_work_doubles(g, ks));
      double rest = 0.0;
      if (!work) return DSRG_FNO_ERR_NOMEM;
      DSRG_TRY(mr_energy_rest(g, ks, prob->B_hp, prob->eps, prob->f_hp, prob->gamma1, prob->lambda2, mr->l3, work, &rest,
                              st));
      e_mo += rest;
    }
  }
  double e_f = 0.0;
  if (nk > 0) {
    // F' = Vk^T diag(eps_v) Vk, recanonicalised: F' W = W eps'
    {
    DSRG_PHASE("phase_recanon_and_rotate", st);
    const double* ev = prob->eps + g.nh;
    DSRG_TRY(scale_rows(nv, nk, nv, ev, no, Wt, st));
    DSRG_TRY(gemm_f64(nk, nk, nv, 1.0, no, nv, false, Wt, nk, false, 0.0, F, nk, 1, 0, 0, 0, st));
    DSRG_TRY(eig_sym_jacobi(nk, F, FV, work, ib, 60, st));
    DSRG_TRY(eig_sort(nk, F, FV, evals, Wsort, ib + 8, false, false, st));
    // U = Vk W
    DSRG_TRY(gemm_f64(nv, nk, nk, 1.0, no, nv, true, Wsort, nk, false, 0.0, U, nk, 1, 0, 0, 0, st));
    // B' = [B_active | B_virtual U]
    DSRG_TRY(copy_active(rows, g.na, g.np, gf.np, prob->B_hp, Bf, st));
    if (ks) {
      ws.off = base;
      __nv_bfloat16* pa = ws_take<__nv_bfloat16>(ws, (size_t)kx * rows * kpv);
      int* ea = ws_take<int>(ws, rows);
      __nv_bfloat16* pb = ws_take<__nv_bfloat16>(ws, (size_t)kx * nk * kpv);
      int* eb = ws_take<int>(ws, nk);
      int* err = ws_take<int>(ws, 8);
      if (!err) return DSRG_FNO_ERR_NOMEM;
      DSRG_CUDA(cudaMemsetAsync(err, 0, sizeof(int), st));
      // rows (Q, h) over the virtual index e, and U^T rows l over e
      DSRG_TRY(slice_rows(kx, prob->B_hp + g.na, rows, nv, g.np, 1, kpv, pa, ea, st));
      DSRG_TRY(slice_rows(kx, U, nk, nv, 1, nk, kpv, pb, eb, st));
      DSRG_TRY(sliced_plain_gemm(kx, (int)rows, nk, pa, ea, pb, eb, kpv, Bf + g.na, gf.np, err, st));
      DSRG_TRY(read_error_flag(err, st));
    } else {
      DSRG_TRY(gemm_f64((int)rows, nk, nv, 1.0, prob->B_hp + g.na, g.np, true, U, nk, false, 0.0, Bf + g.na, gf.np,
                        1, 0, 0, 0, st));
    }
    }
    DSRG_CUDA(cudaMemcpyAsync(epsf, prob->eps, sizeof(double) * g.nh, cudaMemcpyDeviceToDevice, st));
    DSRG_CUDA(cudaMemcpyAsync(epsf + g.nh, evals, sizeof(double) * nk, cudaMemcpyDeviceToDevice, st));
    if (eps_fno_out)
      DSRG_CUDA(cudaMemcpyAsync(eps_fno_out, evals, sizeof(double) * nk, cudaMemcpyDeviceToDevice, st));
    DSRG_TRY(energy_pass(gf, ks, pform, Bf, epsf, prob->gamma1, prob->lambda2, ws, base, budget, &e_f, st));
  }
  if (mr) {
    // E^(2)(FNO) beyond its vv part: the active particles stay, the kept
    // virtuals are the recanonicalised NOs (with nkept = 0 only the active
    // particles are left); f_hp's virtual columns rotate with them.
    if (nk == 0) {
      DSRG_TRY(copy_active(rows, g.na, g.np, gf.np, prob->B_hp, Bf, st));
      DSRG_CUDA(cudaMemcpyAsync(epsf, prob->eps, sizeof(double) * g.nh, cudaMemcpyDeviceToDevice, st));
    }
    const double* f_fno = nullptr;
    if (prob->f_hp) {
      DSRG_TRY(copy_active(g.nh, g.na, g.np, gf.np, prob->f_hp, ff, st));
      if (nk > 0)
        DSRG_TRY(gemm_f64(g.nh, nk, nv, 1.0, prob->f_hp + g.na, g.np, true, U, nk, false, 0.0, ff + g.na, gf.np, 1,
                          0, 0, 0, st));
      f_fno = ff;
    }
    ws.off = base;
    double* work = ws_take<double>(ws, mr_energy_work_doubles(gf, ks));
    double rest = 0.0;
    if (!work) return DSRG_FNO_ERR_NOMEM;
    DSRG_TRY(mr_energy_rest(gf, ks, Bf, epsf, f_fno, prob->gamma1, prob->lambda2, mr->l3, work, &rest, st));
    e_f += rest;
  }
  if (!isfinite(e_mo) || !isfinite(e_f)) return DSRG_FNO_ERR_NONFINITE;
  *de_out = e_mo - e_f;
  if (e2_fno_out) *e2_fno_out = e_f;
  return DSRG_FNO_OK;
}

}  // namespace dsrg

using namespace dsrg;

extern "C" {

const char* dsrg_fno_status_string(int s) {
  switch (s) {
    case DSRG_FNO_OK: return "ok";
    case DSRG_FNO_ERR_ARG: return "invalid argument";
    case DSRG_FNO_ERR_CUDA: return "CUDA runtime error";
    case DSRG_FNO_ERR_NOMEM: return "device workspace allocation failed";
    case DSRG_FNO_ERR_NOCONV: return "eigensolver did not converge";
    case DSRG_FNO_ERR_TIMEOUT: return "bounded device wait expired";
    case DSRG_FNO_ERR_NONFINITE: return "non-finite input or result";
    case DSRG_FNO_ERR_UNSUPPORTED: return "unsupported request";
    default: return "unknown status";
  }
}

void dsrg_fno_release(void) {
  release_batch_pools();
  std::lock_guard<std::mutex> lk(workspace_mutex());
  int cur = 0;
  cudaGetDevice(&cur);
  for (int d = 0; d < 64; ++d) {
    if (g_ws[d].base) {
      cudaSetDevice(d);
      cudaDeviceSynchronize();
      cudaFree(g_ws[d].base);
      g_ws[d].base = nullptr;
      g_ws[d].cap = 0;
      g_ws[d].off = 0;
    }
  }
  cudaSetDevice(cur);
}

int dsrg_fno_pt2_energy(const dsrg_fno_problem* prob, double* e2_out, void* stream) {
  std::lock_guard<std::mutex> lk(workspace_mutex());
  Workspace& ws = workspace_for_current_device();
  return impl_pt2_energy(ws, plan_budget(ws), prob, e2_out, (cudaStream_t)stream);
}

int dsrg_fno_pt2_energy_mr(const dsrg_fno_problem* prob, const double* lambda3, double* e2_out, double* evv_out,
                           void* stream) {
  std::lock_guard<std::mutex> lk(workspace_mutex());
  Workspace& ws = workspace_for_current_device();
  return impl_pt2_energy_mr(ws, plan_budget(ws), prob, lambda3, e2_out, evv_out, (cudaStream_t)stream);
}

int dsrg_fno_vv_opdm(const dsrg_fno_problem* prob, double* dvv_out, double* e2_out, void* stream) {
  std::lock_guard<std::mutex> lk(workspace_mutex());
  Workspace& ws = workspace_for_current_device();
  return impl_vv_opdm(ws, plan_budget(ws), prob, dvv_out, e2_out, (cudaStream_t)stream);
}

int dsrg_fno_vv_opdm_lambda3(const dsrg_fno_problem* prob, const double* lambda3, double* dvv_out, double* e2_out,
                             void* stream) {
  if (prob && prob->nact > 0 && !lambda3) return DSRG_FNO_ERR_ARG;
  std::lock_guard<std::mutex> lk(workspace_mutex());
  Workspace& ws = workspace_for_current_device();
  return impl_vv_opdm(ws, plan_budget(ws), prob, dvv_out, e2_out, (cudaStream_t)stream, lambda3);
}

int dsrg_fno_truncate(int32_t nvir, const double* dvv, int32_t mode, double threshold, double degen_ratio,
                      double* on_out, double* no_out, int32_t* nkept_out, void* stream) {
  std::lock_guard<std::mutex> lk(workspace_mutex());
  Workspace& ws = workspace_for_current_device();
  return impl_truncate(ws, nvir, dvv, mode, threshold, degen_ratio, on_out, no_out, nkept_out, (cudaStream_t)stream);
}

int dsrg_fno_cut(int32_t nvir, const double* ons, int32_t mode, double threshold, double degen_ratio,
                 int32_t* nkept_out, void* stream) {
  if (nvir <= 0 || !ons || !nkept_out || !is_device_ptr(ons)) return DSRG_FNO_ERR_ARG;
  if (mode < 0 || mode > 3 || !isfinite(threshold) || !(degen_ratio >= 0.0)) return DSRG_FNO_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  std::lock_guard<std::mutex> lk(workspace_mutex());
  Workspace& ws = workspace_for_current_device();
  DSRG_TRY(ws_reserve(ws, ws_bytes(8, sizeof(int))));
  int* nk = ws_take<int>(ws, 8);
  DSRG_TRY(truncate_ons(nvir, ons, mode, threshold, degen_ratio, nk, st));
  int h = 0;
  DSRG_CUDA(cudaMemcpyAsync(&h, nk, sizeof(int), cudaMemcpyDeviceToHost, st));
  DSRG_CUDA(cudaStreamSynchronize(st));
  *nkept_out = h;
  return DSRG_FNO_OK;
}

int dsrg_fno_discarded_correction(const dsrg_fno_problem* prob, int32_t nkept, const double* no,
                                  const double* e2_mo_in, double* de_out, double* e2_fno_out,
                                  double* eps_fno_out, void* stream) {
  std::lock_guard<std::mutex> lk(workspace_mutex());
  Workspace& ws = workspace_for_current_device();
  return impl_correction(ws, plan_budget(ws), prob, nkept, no, e2_mo_in, de_out, e2_fno_out, eps_fno_out,
                         (cudaStream_t)stream);
}

int dsrg_fno_discarded_correction_mr(const dsrg_fno_problem* prob, const double* lambda3, int32_t nkept,
                                     const double* no, const double* e2_mo_in, double* de_out, double* e2_fno_out,
                                     double* eps_fno_out, void* stream) {
  if (lambda3 && prob && prob->nact > 0 && !is_device_ptr(lambda3)) return DSRG_FNO_ERR_ARG;
  CorrectionMR mr{prob && prob->nact > 0 ? lambda3 : nullptr};
  std::lock_guard<std::mutex> lk(workspace_mutex());
  Workspace& ws = workspace_for_current_device();
  return impl_correction(ws, plan_budget(ws), prob, nkept, no, e2_mo_in, de_out, e2_fno_out, eps_fno_out,
                         (cudaStream_t)stream, &mr);
}

}  // extern "C"
