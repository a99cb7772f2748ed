"""dsrg_fno_truncate_noalloc: the allocation-free truncation.

For callers that cannot allocate device memory (a framework owning all
device memory through its own pool, or a latency-critical loop where a
cudaMalloc, which may synchronise the device, is not acceptable).  The call
must give what dsrg_fno_truncate gives, on two calls in a row that reuse its
fixed scratch array, up to the largest size the array serves, and must leave
the library's workspace untouched.  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import oracle as O  # noqa: E402
import paper_2312_07008_gb300 as pkg  # noqa: E402
from synth import make_problem  # noqa: E402

NOALLOC_NVIR_MAX = 512


def _noalloc_c(d, mode, thr, on, no):
    """dsrg_fno_truncate_noalloc through the C ABI directly."""
    lib = pkg.load()
    k = ctypes.c_int32()
    st = lib.dsrg_fno_truncate_noalloc(d.shape[0], ctypes.c_void_p(d.data_ptr()), mode, thr, 0.01,
                                       ctypes.c_void_p(on.data_ptr()), ctypes.c_void_p(no.data_ptr()),
                                       ctypes.byref(k), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 0, st
    torch.cuda.synchronize()
    return k.value


def _reference_and_noalloc(dvv, mode, thr):
    nv = dvv.shape[0]
    d = torch.from_numpy(np.ascontiguousarray(dvv)).cuda()
    on1 = torch.empty(nv, dtype=torch.float64, device="cuda")
    no1 = torch.empty((nv, nv), dtype=torch.float64, device="cuda")
    on2 = torch.empty_like(on1)
    no2 = torch.empty_like(no1)
    k1 = pkg.dsrg_fno_truncate(nv, d, mode, thr, 0.01, on1, no1)
    k2 = _noalloc_c(d, mode, thr, on2, no2)
    return (k1, on1.cpu().numpy(), no1.cpu().numpy()), (k2, on2.cpu().numpy(), no2.cpu().numpy())


def _same(ref, got):
    assert got[0] == ref[0]
    assert np.max(np.abs(got[1] - ref[1])) <= 1e-9
    k = got[0]
    P1 = got[2][:, :k] @ got[2][:, :k].T
    P2 = ref[2][:, :k] @ ref[2][:, :k].T
    assert np.max(np.abs(P1 - P2)) <= 1e-9


def test_noalloc_matches_truncate_on_two_calls_in_a_row():
    # two different D_vv matrices, so the second call cannot lean on the first's contents
    pa = make_problem(ncore=4, nact=2, nvir=130, naux=90, seed=51, nstates=2)
    pb = make_problem(ncore=3, nact=0, nvir=77, naux=60, seed=52)
    for p, mode, thr in ((pa, 0, 98.5), (pb, 1, 40.0)):
        ref, got = _reference_and_noalloc(O.dvv(p), mode, thr)
        _same(ref, got)


def test_noalloc_at_the_largest_size_allocates_nothing():
    """nvir = 512 fills the fixed array exactly.  After dsrg_fno_release()
    the library holds no workspace; two noalloc calls leave it at zero bytes
    and the device's free memory unchanged (any cudaMalloc would take at
    least 2 MiB), and match dsrg_fno_truncate."""
    nv = NOALLOC_NVIR_MAX
    p = make_problem(ncore=3, nact=0, nvir=nv, naux=40, seed=53)
    dvv = O.dvv(p)
    d = torch.from_numpy(np.ascontiguousarray(dvv)).cuda()
    on_r = torch.empty(nv, dtype=torch.float64, device="cuda")
    no_r = torch.empty((nv, nv), dtype=torch.float64, device="cuda")
    k_r = pkg.dsrg_fno_truncate(nv, d, 0, 98.5, 0.01, on_r, no_r)
    ref = (k_r, on_r.cpu().numpy(), no_r.cpu().numpy())
    on = torch.empty(nv, dtype=torch.float64, device="cuda")
    no = torch.empty((nv, nv), dtype=torch.float64, device="cuda")
    _noalloc_c(d, 0, 98.5, on, no)   # first call on the device: set-up (loads the array's module)
    pkg.dsrg_fno_release()
    assert pkg.dsrg_fno_debug_workspace_bytes() == 0
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(2):
        on.fill_(0.0)
        no.fill_(0.0)
        k = _noalloc_c(d, 0, 98.5, on, no)
        _same(ref, (k, on.cpu().numpy(), no.cpu().numpy()))
    free1 = torch.cuda.mem_get_info()[0]
    assert pkg.dsrg_fno_debug_workspace_bytes() == 0
    assert abs(free1 - free0) < (2 << 20), (free0, free1)


def test_noalloc_rejects_sizes_beyond_its_array():
    nv = NOALLOC_NVIR_MAX + 1
    d = torch.zeros((nv, nv), dtype=torch.float64, device="cuda")
    on = torch.empty(nv, dtype=torch.float64, device="cuda")
    no = torch.empty((nv, nv), dtype=torch.float64, device="cuda")
    with pytest.raises(pkg.DsrgFnoError) as ei:
        pkg.dsrg_fno_truncate_noalloc(nv, d, 0, 98.5, 0.01, on, no)
    assert ei.value.status == -1


def test_noalloc_rejects_a_host_output_before_any_work():
    nv = 16
    d = torch.eye(nv, dtype=torch.float64, device="cuda")
    on_host = np.zeros(nv)
    no = torch.empty((nv, nv), dtype=torch.float64, device="cuda")
    lib = pkg.load()
    k = ctypes.c_int32(-3)
    st = lib.dsrg_fno_truncate_noalloc(nv, ctypes.c_void_p(d.data_ptr()), 0, 98.5, 0.01,
                                       ctypes.c_void_p(on_host.ctypes.data), ctypes.c_void_p(no.data_ptr()),
                                       ctypes.byref(k), None)
    assert st == -1
    assert k.value == -3 and not on_host.any()
