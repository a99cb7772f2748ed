"""dsrg_fno_truncate_noalloc: the allocation-free truncation.

For callers that cannot allocate device memory (a framework owning all
device memory through its own pool, or a latency-critical loop where a
cudaMalloc, which may synchronise the device, is not acceptable).  The call
must give what dsrg_fno_truncate gives, on two calls in a row that reuse its
fixed scratch array.  This file is collected last on purpose.
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


def _reference_and_noalloc(dvv, mode, thr):
    nv = dvv.shape[0]
    d = torch.from_numpy(np.ascontiguousarray(dvv)).cuda()
    on1 = torch.empty(nv, dtype=torch.float64, device="cuda")
    no1 = torch.empty((nv, nv), dtype=torch.float64, device="cuda")
    on2 = torch.empty_like(on1)
    no2 = torch.empty_like(no1)
    k1 = pkg.dsrg_fno_truncate(nv, d, mode, thr, 0.01, on1, no1)
    # through the C ABI directly
    lib = pkg.load()
    k2 = ctypes.c_int32()
    st = lib.dsrg_fno_truncate_noalloc(nv, ctypes.c_void_p(d.data_ptr()), mode, thr, 0.01,
                                       ctypes.c_void_p(on2.data_ptr()), ctypes.c_void_p(no2.data_ptr()),
                                       ctypes.byref(k2), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 0
    torch.cuda.synchronize()
    return (k1, on1.cpu().numpy(), no1.cpu().numpy()), (k2.value, on2.cpu().numpy(), no2.cpu().numpy())


def test_noalloc_matches_truncate_on_two_calls_in_a_row():
    # two different D_vv matrices, so the second call cannot lean on the first's contents
    pa = make_problem(ncore=4, nact=2, nvir=130, naux=90, seed=51, nstates=2)
    pb = make_problem(ncore=3, nact=0, nvir=77, naux=60, seed=52)
    for p, mode, thr in ((pa, 0, 98.5), (pb, 1, 40.0)):
        ref, got = _reference_and_noalloc(O.dvv(p), mode, thr)
        assert got[0] == ref[0]
        assert np.max(np.abs(got[1] - ref[1])) <= 1e-9
        k = got[0]
        P1 = got[2][:, :k] @ got[2][:, :k].T
        P2 = ref[2][:, :k] @ ref[2][:, :k].T
        assert np.max(np.abs(P1 - P2)) <= 1e-9


def test_noalloc_rejects_sizes_beyond_its_array():
    nv = 513
    d = torch.zeros((nv, nv), dtype=torch.float64, device="cuda")
    on = torch.empty(nv, dtype=torch.float64, device="cuda")
    no = torch.empty((nv, nv), dtype=torch.float64, device="cuda")
    with pytest.raises(pkg.DsrgFnoError) as ei:
        pkg.dsrg_fno_truncate_noalloc(nv, d, 0, 98.5, 0.01, on, no)
    assert ei.value.status == -1
