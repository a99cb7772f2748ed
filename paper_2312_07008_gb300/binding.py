"""ctypes binding of libdsrg_fno.so: argument marshalling only.

The functions carry the names of the C ABI (include/dsrg_fno.h).  Device
arrays are torch tensors (float64, contiguous, on the current CUDA device);
every step of the computation runs in the library's CUDA kernels.  A missing
library raises; there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libdsrg_fno.so")

EXPORTED = (
    "dsrg_fno_pt2_energy",
    "dsrg_fno_pt2_energy_mr",
    "dsrg_fno_discarded_correction_mr",
    "dsrg_fno_vv_opdm",
    "dsrg_fno_vv_opdm_lambda3",
    "dsrg_fno_sa_lambda3",
    "dsrg_fno_truncate",
    "dsrg_fno_truncate_noalloc",
    "dsrg_fno_cut",
    "dsrg_fno_naf",
    "dsrg_fno_ladder",
    "dsrg_fno_discarded_correction",
    "dsrg_fno_sa_densities",
    "dsrg_fno_batch_run",
    "dsrg_fno_status_string",
    "dsrg_fno_release",
    "dsrg_fno_debug_sliced_gemm",
    "dsrg_fno_debug_literal_gemm",
    "dsrg_fno_debug_slice_rows",
    "dsrg_fno_debug_slice_rows_dd",
    "dsrg_fno_debug_regularizer",
    "dsrg_fno_debug_mma_schedule",
    "dsrg_fno_debug_workspace_bytes",
    "dsrg_fno_debug_eig_batch",
    "dsrg_fno_debug_pair_tiles",
    "dsrg_fno_debug_set_barrier_limit",
    "dsrg_fno_debug_set_fused_epilogue",
    "dsrg_fno_debug_set_syrk_planes",
    "dsrg_fno_debug_set_eig_colpair",
    "dsrg_fno_set_log_callback",
    "dsrg_fno_profile_enable",
    "dsrg_fno_profile_query",
    "dsrg_fno_launch_count",
    "dsrg_fno_batch_last_workers",
)

FP64 = 0
SLICED_BF16 = 1
BF16X3 = 2
TF32 = 3
MODE_PO, MODE_PV, MODE_NKAPPA, MODE_FIXED = 0, 1, 2, 3


class DsrgFnoError(RuntimeError):
    def __init__(self, func: str, status: int, text: str):
        super().__init__(f"{func} returned {status}: {text}")
        self.status = status


class CProblem(ctypes.Structure):
    _fields_ = [
        ("ncore", ctypes.c_int32), ("nact", ctypes.c_int32), ("nvir", ctypes.c_int32), ("naux", ctypes.c_int32),
        ("B_hp", ctypes.c_void_p), ("eps", ctypes.c_void_p), ("gamma1", ctypes.c_void_p),
        ("lambda2", ctypes.c_void_p), ("f_hp", ctypes.c_void_p),
        ("nstates", ctypes.c_int32), ("weights", ctypes.POINTER(ctypes.c_double)),
        ("s", ctypes.c_double), ("precision", ctypes.c_int32), ("nslices", ctypes.c_int32),
    ]


class CBatchItem(ctypes.Structure):
    _fields_ = [
        ("problem", CProblem), ("dvv_out", ctypes.c_void_p),
        ("cut_mode", ctypes.c_int32), ("cut_threshold", ctypes.c_double), ("cut_degen_ratio", ctypes.c_double),
        ("on_out", ctypes.c_void_p), ("no_out", ctypes.c_void_p), ("correction", ctypes.c_int32),
        ("e2", ctypes.c_double), ("nkept", ctypes.c_int32), ("de", ctypes.c_double), ("status", ctypes.c_int32),
    ]


_lib = None
# void (*)(int level, const char* message, void* user)
LOG_FN = ctypes.CFUNCTYPE(None, ctypes.c_int, ctypes.c_char_p, ctypes.c_void_p)
_log_keep = None  # the installed ctypes callback, kept alive while installed


def load(path: str = LIB_PATH):
    """Loads the library (once).  Raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: run __graft_entry__.build() (nvcc, sm_103a) first")
    lib = ctypes.CDLL(path)
    vp, d, i32 = ctypes.c_void_p, ctypes.c_double, ctypes.c_int32
    P = ctypes.POINTER(CProblem)
    lib.dsrg_fno_pt2_energy.argtypes = [P, ctypes.POINTER(d), vp]
    lib.dsrg_fno_pt2_energy_mr.argtypes = [P, vp, ctypes.POINTER(d), ctypes.POINTER(d), vp]
    lib.dsrg_fno_discarded_correction_mr.argtypes = [P, vp, i32, vp, ctypes.POINTER(d), ctypes.POINTER(d),
                                                     ctypes.POINTER(d), vp, vp]
    lib.dsrg_fno_vv_opdm.argtypes = [P, vp, ctypes.POINTER(d), vp]
    lib.dsrg_fno_vv_opdm_lambda3.argtypes = [P, vp, vp, ctypes.POINTER(d), vp]
    lib.dsrg_fno_sa_lambda3.argtypes = [i32, i32, ctypes.POINTER(d), vp, vp, vp, vp, vp]
    lib.dsrg_fno_truncate.argtypes = [i32, vp, i32, d, d, vp, vp, ctypes.POINTER(i32), vp]
    lib.dsrg_fno_truncate_noalloc.argtypes = [i32, vp, i32, d, d, vp, vp, ctypes.POINTER(i32), vp]
    lib.dsrg_fno_cut.argtypes = [i32, vp, i32, d, d, ctypes.POINTER(i32), vp]
    lib.dsrg_fno_naf.argtypes = [i32, i32, i32, vp, d, i32, vp, vp, ctypes.POINTER(i32), vp]
    lib.dsrg_fno_ladder.argtypes = [i32, i32, vp, i32, vp, i32, vp, vp]
    lib.dsrg_fno_discarded_correction.argtypes = [P, i32, vp, ctypes.POINTER(d), ctypes.POINTER(d),
                                                  ctypes.POINTER(d), vp, vp]
    dp_ = ctypes.POINTER(d)
    lib.dsrg_fno_sa_densities.argtypes = [i32, i32, dp_, dp_, dp_, dp_, dp_]
    lib.dsrg_fno_batch_run.argtypes = [ctypes.POINTER(CBatchItem), i32, i32, vp]
    lib.dsrg_fno_batch_last_workers.argtypes = []
    lib.dsrg_fno_batch_last_workers.restype = i32
    lib.dsrg_fno_status_string.argtypes = [ctypes.c_int]
    lib.dsrg_fno_status_string.restype = ctypes.c_char_p
    lib.dsrg_fno_release.argtypes = []
    dp = ctypes.POINTER(d)
    lib.dsrg_fno_debug_sliced_gemm.argtypes = [i32, i32, i32, i32, dp, dp, dp]
    lib.dsrg_fno_debug_literal_gemm.argtypes = [i32, i32, i32, i32, i32, dp, dp, dp]
    lib.dsrg_fno_debug_literal_gemm.restype = ctypes.c_int
    lib.dsrg_fno_debug_slice_rows.argtypes = [i32, i32, i32, dp, ctypes.POINTER(ctypes.c_float),
                                              ctypes.POINTER(i32)]
    lib.dsrg_fno_debug_slice_rows_dd.argtypes = [i32, i32, i32, ctypes.POINTER(ctypes.c_float),
                                                 ctypes.POINTER(ctypes.c_float), ctypes.POINTER(i32)]
    lib.dsrg_fno_debug_regularizer.argtypes = [i32, dp, d, dp, dp]
    lib.dsrg_fno_debug_mma_schedule.argtypes = [i32, ctypes.POINTER(i32), i32]
    lib.dsrg_fno_debug_mma_schedule.restype = ctypes.c_int
    lib.dsrg_fno_debug_pair_tiles.argtypes = [i32, i32, i32, i32, ctypes.POINTER(i32), i32, i32,
                                              ctypes.POINTER(i32), i32]
    lib.dsrg_fno_debug_pair_tiles.restype = ctypes.c_int
    lib.dsrg_fno_debug_set_eig_colpair.argtypes = [i32]
    lib.dsrg_fno_debug_set_eig_colpair.restype = ctypes.c_int
    lib.dsrg_fno_debug_set_syrk_planes.argtypes = [i32]
    lib.dsrg_fno_debug_set_syrk_planes.restype = ctypes.c_int
    lib.dsrg_fno_debug_set_fused_epilogue.argtypes = [i32]
    lib.dsrg_fno_debug_set_fused_epilogue.restype = ctypes.c_int
    lib.dsrg_fno_debug_set_barrier_limit.argtypes = [ctypes.c_int64]
    lib.dsrg_fno_debug_set_barrier_limit.restype = ctypes.c_int
    lib.dsrg_fno_debug_eig_batch.argtypes = [i32, ctypes.POINTER(i32), ctypes.POINTER(ctypes.POINTER(d)),
                                             ctypes.POINTER(ctypes.POINTER(d))]
    lib.dsrg_fno_debug_eig_batch.restype = ctypes.c_int
    lib.dsrg_fno_debug_workspace_bytes.argtypes = []
    lib.dsrg_fno_debug_workspace_bytes.restype = ctypes.c_int64
    lib.dsrg_fno_set_log_callback.argtypes = [LOG_FN, vp]
    lib.dsrg_fno_set_log_callback.restype = None
    lib.dsrg_fno_profile_enable.argtypes = [i32]
    lib.dsrg_fno_profile_enable.restype = None
    lib.dsrg_fno_profile_query.argtypes = [ctypes.c_char_p, ctypes.POINTER(d), ctypes.POINTER(ctypes.c_int64),
                                           ctypes.POINTER(d)]
    lib.dsrg_fno_launch_count.argtypes = [i32]
    lib.dsrg_fno_launch_count.restype = ctypes.c_int64
    for f in ("dsrg_fno_pt2_energy", "dsrg_fno_vv_opdm", "dsrg_fno_vv_opdm_lambda3", "dsrg_fno_sa_lambda3",
              "dsrg_fno_truncate", "dsrg_fno_truncate_noalloc",
              "dsrg_fno_cut", "dsrg_fno_naf", "dsrg_fno_ladder", "dsrg_fno_discarded_correction", "dsrg_fno_sa_densities", "dsrg_fno_batch_run"):
        getattr(lib, f).restype = ctypes.c_int
    _lib = lib
    return lib


def _check(func: str, status: int):
    if status != 0:
        raise DsrgFnoError(func, status, load().dsrg_fno_status_string(status).decode())


def _ptr(t):
    if t is None:
        return None
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return ctypes.c_void_p(getattr(stream, "cuda_stream", stream))


class Problem:
    """Holds the C struct and keeps its tensors alive."""

    def __init__(self, ncore, nact, nvir, naux, B, eps, gamma1=None, lambda2=None, f_hp=None,
                 weights=(1.0,), s=0.5, precision=FP64, nslices=0):
        self.tensors = (B, eps, gamma1, lambda2, f_hp)
        w = np.ascontiguousarray(np.asarray(weights, dtype=np.float64))
        self._w = w
        self.c = CProblem(ncore, nact, nvir, naux, _ptr(B), _ptr(eps), _ptr(gamma1), _ptr(lambda2), _ptr(f_hp),
                          len(w), w.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), float(s), int(precision),
                          int(nslices))
        self.ncore, self.nact, self.nvir, self.naux = ncore, nact, nvir, naux


def problem_from_synth(p, device="cuda", precision=FP64, nslices=0):
    """Uploads a synth.Problem (numpy) to the device and wraps it."""
    import torch
    t = lambda a: None if a is None else torch.from_numpy(np.ascontiguousarray(a)).to(device)  # noqa: E731
    return Problem(p.ncore, p.nact, p.nvir, p.naux, t(p.B), t(p.eps), t(p.gamma1), t(p.lambda2), t(p.f_hp),
                   p.weights, p.s, precision, nslices)


def dsrg_fno_pt2_energy(prob: Problem, stream=None) -> float:
    e = ctypes.c_double()
    _check("dsrg_fno_pt2_energy", load().dsrg_fno_pt2_energy(ctypes.byref(prob.c), ctypes.byref(e), _stream(stream)))
    return e.value


def dsrg_fno_pt2_energy_mr(prob: Problem, lambda3=None, stream=None):
    """Full E^(2) over every amplitude class; lambda3 (device [nact]^6) or None.
    Returns (E^(2), its vv-class part E_vv)."""
    e = ctypes.c_double()
    ev = ctypes.c_double()
    _check("dsrg_fno_pt2_energy_mr",
           load().dsrg_fno_pt2_energy_mr(ctypes.byref(prob.c), _ptr(lambda3) if lambda3 is not None else None,
                                         ctypes.byref(e), ctypes.byref(ev), _stream(stream)))
    return e.value, ev.value


def dsrg_fno_vv_opdm(prob: Problem, dvv_out, stream=None) -> float:
    e = ctypes.c_double()
    _check("dsrg_fno_vv_opdm", load().dsrg_fno_vv_opdm(ctypes.byref(prob.c), _ptr(dvv_out), ctypes.byref(e),
                                                      _stream(stream)))
    return e.value


def dsrg_fno_vv_opdm_lambda3(prob: Problem, lambda3, dvv_out, stream=None) -> float:
    """D_vv with Eq. A12 term 13 (lambda3: device [nact]^6 3-cumulant)."""
    e = ctypes.c_double()
    _check("dsrg_fno_vv_opdm_lambda3",
           load().dsrg_fno_vv_opdm_lambda3(ctypes.byref(prob.c), _ptr(lambda3), _ptr(dvv_out), ctypes.byref(e),
                                           _stream(stream)))
    return e.value


def dsrg_fno_sa_lambda3(weights, gamma1, lambda2, gamma3_states, lambda3_out, stream=None):
    """Ensemble spin-free 3-cumulant on the device from the ensemble Gamma1,
    Lambda2 and the per-state 3-RDMs gamma3_states [S][n]^6 (device tensors)."""
    w = np.ascontiguousarray(np.asarray(weights, dtype=np.float64))
    n = int(gamma1.shape[0])
    if tuple(gamma3_states.shape) != (len(w),) + (n,) * 6 or tuple(lambda3_out.shape) != (n,) * 6:
        raise ValueError("shapes: gamma3_states [S][n]^6, lambda3_out [n]^6")
    _check("dsrg_fno_sa_lambda3",
           load().dsrg_fno_sa_lambda3(n, len(w), w.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), _ptr(gamma1),
                                      _ptr(lambda2), _ptr(gamma3_states), _ptr(lambda3_out), _stream(stream)))


def dsrg_fno_truncate(nvir, dvv, mode, threshold, degen_ratio, on_out, no_out, stream=None) -> int:
    k = ctypes.c_int32()
    _check("dsrg_fno_truncate", load().dsrg_fno_truncate(nvir, _ptr(dvv), mode, float(threshold),
                                                        float(degen_ratio), _ptr(on_out), _ptr(no_out),
                                                        ctypes.byref(k), _stream(stream)))
    return k.value


def dsrg_fno_cut(nvir, ons, mode, threshold, degen_ratio, stream=None) -> int:
    """N' for ONs already on the device (further cuts of the same NOs)."""
    k = ctypes.c_int32()
    _check("dsrg_fno_cut", load().dsrg_fno_cut(nvir, _ptr(ons), mode, float(threshold), float(degen_ratio),
                                              ctypes.byref(k), _stream(stream)))
    return k.value


def dsrg_fno_naf(nh, np_, naux, B, threshold, precision, B_out, w_out=None, stream=None) -> int:
    """Natural auxiliary functions: B_out[:naux'] = U_kept^T B; returns naux'."""
    k = ctypes.c_int32()
    _check("dsrg_fno_naf", load().dsrg_fno_naf(int(nh), int(np_), int(naux), _ptr(B), float(threshold),
                                              int(precision), _ptr(B_out), _ptr(w_out), ctypes.byref(k),
                                              _stream(stream)))
    return k.value


def dsrg_fno_ladder(B_vv, T, C_out, precision=SLICED_BF16, stream=None):
    """Particle-particle ladder C[p] = sum_cd <ab|cd> T[p][c][d] (device tensors)."""
    naux, nv = int(B_vv.shape[0]), int(B_vv.shape[1])
    _check("dsrg_fno_ladder", load().dsrg_fno_ladder(nv, naux, _ptr(B_vv), int(T.shape[0]), _ptr(T), int(precision),
                                                    _ptr(C_out), _stream(stream)))


def dsrg_fno_truncate_noalloc(nvir, dvv, mode, threshold, degen_ratio, on_out, no_out, stream=None) -> int:
    """dsrg_fno_truncate that allocates nothing on the device (nvir <= 512)."""
    k = ctypes.c_int32()
    _check("dsrg_fno_truncate_noalloc",
           load().dsrg_fno_truncate_noalloc(nvir, _ptr(dvv), mode, float(threshold), float(degen_ratio),
                                            _ptr(on_out), _ptr(no_out), ctypes.byref(k), _stream(stream)))
    return k.value


def dsrg_fno_discarded_correction(prob: Problem, nkept, no, e2_mo=None, eps_fno_out=None, stream=None):
    de, ef = ctypes.c_double(), ctypes.c_double()
    emo = None if e2_mo is None else ctypes.byref(ctypes.c_double(e2_mo))
    _check("dsrg_fno_discarded_correction",
           load().dsrg_fno_discarded_correction(ctypes.byref(prob.c), int(nkept), _ptr(no), emo, ctypes.byref(de),
                                                ctypes.byref(ef), _ptr(eps_fno_out), _stream(stream)))
    return de.value, ef.value


def dsrg_fno_discarded_correction_mr(prob: Problem, nkept, no, lambda3=None, e2_mo=None, eps_fno_out=None,
                                     stream=None):
    """Eq. 11 with the full E^(2): returns (E^(2)(MO) - E^(2)(FNO), E^(2)(FNO))."""
    de, ef = ctypes.c_double(), ctypes.c_double()
    emo = None if e2_mo is None else ctypes.byref(ctypes.c_double(e2_mo))
    _check("dsrg_fno_discarded_correction_mr",
           load().dsrg_fno_discarded_correction_mr(ctypes.byref(prob.c), _ptr(lambda3) if lambda3 is not None else None,
                                                   int(nkept), _ptr(no), emo, ctypes.byref(de), ctypes.byref(ef),
                                                   _ptr(eps_fno_out), _stream(stream)))
    return de.value, ef.value


def dsrg_fno_sa_densities(weights, g1_states, g2_states):
    """SA Gamma1 and the ensemble 2-cumulant (Eq. A1) from per-state host arrays."""
    w = np.ascontiguousarray(np.asarray(weights, dtype=np.float64))
    g1 = np.ascontiguousarray(np.asarray(g1_states, dtype=np.float64))
    g2 = np.ascontiguousarray(np.asarray(g2_states, dtype=np.float64))
    nst, n = g1.shape[0], g1.shape[1]
    if g1.shape != (nst, n, n) or g2.shape != (nst, n, n, n, n) or w.shape != (nst,):
        raise ValueError("shapes: weights [S], g1_states [S][n][n], g2_states [S][n]^4")
    out1 = np.zeros((n, n))
    out2 = np.zeros((n, n, n, n))
    dp = ctypes.POINTER(ctypes.c_double)
    _check("dsrg_fno_sa_densities",
           load().dsrg_fno_sa_densities(n, nst, w.ctypes.data_as(dp), g1.ctypes.data_as(dp), g2.ctypes.data_as(dp),
                                        out1.ctypes.data_as(dp), out2.ctypes.data_as(dp)))
    return out1, out2


def dsrg_fno_batch_run(problems, dvv_outs=None, cut=None, on_outs=None, no_outs=None, correction=False,
                       nworkers=0, stream=None):
    """Runs independent instances concurrently (dsrg_fno_batch_run).

    problems: list of Problem; dvv_outs: list of device tensors or None
    (energy only); cut: (mode, threshold, degen_ratio) or None, with on_outs
    and no_outs; correction: discarded-virtual correction after the cut.
    Returns a list of dicts (e2, nkept, de) in input order; raises on the
    first failing instance (each status is in the 'status' key).
    """
    n = len(problems)
    arr = (CBatchItem * max(n, 1))()
    for i, p in enumerate(problems):
        it = arr[i]
        it.problem = p.c
        it.dvv_out = _ptr(dvv_outs[i]) if dvv_outs is not None else None
        if cut is not None:
            it.cut_mode, it.cut_threshold, it.cut_degen_ratio = int(cut[0]), float(cut[1]), float(cut[2])
            it.on_out = _ptr(on_outs[i])
            it.no_out = _ptr(no_outs[i])
        else:
            it.cut_mode = -1
        it.correction = 1 if correction else 0
    st = load().dsrg_fno_batch_run(arr, n, int(nworkers), _stream(stream))
    out = [dict(e2=arr[i].e2, nkept=arr[i].nkept, de=arr[i].de, status=arr[i].status) for i in range(n)]
    _check("dsrg_fno_batch_run", st)
    return out


def dsrg_fno_batch_last_workers() -> int:
    return load().dsrg_fno_batch_last_workers()


def dsrg_fno_release():
    load().dsrg_fno_release()


def dsrg_fno_profile_enable(enable: bool):
    load().dsrg_fno_profile_enable(1 if enable else 0)


def dsrg_fno_profile_query(name: str):
    """(total ms, launches, executed flops) of the recorded launches of `name`."""
    t, f = ctypes.c_double(), ctypes.c_double()
    n = ctypes.c_int64()
    load().dsrg_fno_profile_query(name.encode(), ctypes.byref(t), ctypes.byref(n), ctypes.byref(f))
    return t.value, n.value, f.value


def dsrg_fno_launch_count(reset: bool = False) -> int:
    return load().dsrg_fno_launch_count(1 if reset else 0)


def dsrg_fno_debug_mma_schedule(nslices: int):
    """Stacked-B MMA issue schedule of one k step (host only): a list of
    (A plane, first B plane, B planes, first level, N columns)."""
    buf = (ctypes.c_int32 * (5 * 64))()
    n = load().dsrg_fno_debug_mma_schedule(int(nslices), buf, 64)
    _check("dsrg_fno_debug_mma_schedule", min(n, 0))
    return [tuple(buf[5 * i:5 * i + 5]) for i in range(n)]


def dsrg_fno_debug_eig_batch(mats):
    """Eigensolves of up to 4 symmetric float64 matrices in one call (the
    density step's batched solve).  Returns [(A with eigenvalues on its
    diagonal, V)] per matrix."""
    n = len(mats)
    outA = [np.ascontiguousarray(np.array(m, dtype=np.float64)) for m in mats]
    outV = [np.zeros_like(a) for a in outA]
    dims = (ctypes.c_int32 * n)(*[a.shape[0] for a in outA])
    pa = (ctypes.POINTER(ctypes.c_double) * n)(*[a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) for a in outA])
    pv = (ctypes.POINTER(ctypes.c_double) * n)(*[v.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) for v in outV])
    _check("dsrg_fno_debug_eig_batch", load().dsrg_fno_debug_eig_batch(n, dims, pa, pv))
    return list(zip(outA, outV))


def dsrg_fno_debug_workspace_bytes() -> int:
    """Device workspace bytes the library holds on the current device."""
    return load().dsrg_fno_debug_workspace_bytes()


def dsrg_fno_set_log_callback(fn=None):
    """Routes the library's messages to fn(level, text); None drops them."""
    global _log_keep
    lib = load()
    if fn is None:
        lib.dsrg_fno_set_log_callback(LOG_FN(), None)
        _log_keep = None
        return
    cb = LOG_FN(lambda level, msg, user: fn(int(level), msg.decode(errors="replace")))
    lib.dsrg_fno_set_log_callback(cb, None)
    _log_keep = cb


def dsrg_fno_debug_pair_tiles(nslices, ncore, nact, nvir, pairs, energy_only=False):
    """Output tiles (row tile, column tile) of the pair contraction for one
    batch of hole pairs (host only)."""
    pr = np.ascontiguousarray(np.asarray(pairs, dtype=np.int32).reshape(-1))
    cap = max(16, 4 * len(pr) * ((nact + nvir) // 32 + 2) ** 2)
    buf = np.zeros(2 * cap, dtype=np.int32)
    ip = ctypes.POINTER(ctypes.c_int32)
    n = load().dsrg_fno_debug_pair_tiles(int(nslices), int(ncore), int(nact), int(nvir), pr.ctypes.data_as(ip),
                                         len(pr) // 2, 1 if energy_only else 0, buf.ctypes.data_as(ip), cap)
    _check("dsrg_fno_debug_pair_tiles", min(n, 0))
    return [tuple(buf[2 * t:2 * t + 2]) for t in range(n)]


def dsrg_fno_debug_set_barrier_limit(spins: int):
    """Spin limit of the eigensolver's grid barrier (<= 0: default)."""
    _check("dsrg_fno_debug_set_barrier_limit", load().dsrg_fno_debug_set_barrier_limit(int(spins)))


def dsrg_fno_debug_set_fused_epilogue(on: bool):
    """Eq. A7 epilogue inside the contraction kernel (True) or separate."""
    _check("dsrg_fno_debug_set_fused_epilogue", load().dsrg_fno_debug_set_fused_epilogue(1 if on else 0))


def dsrg_fno_debug_set_syrk_planes(nslices: int):
    """Digit planes of the rank-K update of D_vv (0: library rule)."""
    _check("dsrg_fno_debug_set_syrk_planes", load().dsrg_fno_debug_set_syrk_planes(int(nslices)))


def dsrg_fno_debug_set_eig_colpair(on: bool):
    """Column-pair Jacobi kernel (True, default) or the round-parallel one."""
    _check("dsrg_fno_debug_set_eig_colpair", load().dsrg_fno_debug_set_eig_colpair(1 if on else 0))
