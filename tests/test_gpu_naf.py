"""Natural auxiliary functions on the GPU (dsrg_fno_naf) against the oracle.

The eigenvalues of W = B B^T, the kept count at a threshold, the integrals
of the compressed factors (nu' = B'^T B', independent of the eigenvectors'
signs) and the PT2 step run on the compressed problem (E_vv, D_vv, ONs, N'),
in both arithmetic forms.
"""
import numpy as np
import pytest

import oracle as O
from synth import make_problem

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2312_07008_gb300 as pkg  # noqa: E402


def gpu_naf(p, thr, prec):
    B = torch.from_numpy(np.ascontiguousarray(p.B)).cuda()
    Bo = torch.zeros_like(B)
    w = torch.empty(p.naux, dtype=torch.float64, device="cuda")
    nh, np_ = p.ncore + p.nact, p.nact + p.nvir
    k = pkg.dsrg_fno_naf(nh, np_, p.naux, B, thr, prec, Bo, w)
    torch.cuda.synchronize()
    return k, Bo, w.cpu().numpy()


@pytest.mark.parametrize("prec", [pkg.FP64, pkg.SLICED_BF16], ids=["fp64", "fast"])
def test_naf_matches_oracle(prec):
    p = make_problem(ncore=5, nact=3, nvir=90, naux=260, seed=91, nstates=2)
    _, w_ref, _ = O.naf(p, -1.0)
    keep = 180
    thr = 0.5 * (w_ref[keep - 1] + w_ref[keep])
    k, Bo, w = gpu_naf(p, thr, prec)
    tol = 1e-12 if prec == pkg.FP64 else 1e-10
    assert np.max(np.abs(w - w_ref)) <= tol * w_ref[0]
    assert k == keep
    Bp_ref, _, _ = O.naf(p, thr)
    A = Bo[:k].cpu().numpy().reshape(k, -1)
    R = Bp_ref.reshape(k, -1)
    nu, nu_ref = A.T @ A, R.T @ R
    assert np.max(np.abs(nu - nu_ref)) <= 1e-10 * np.max(np.abs(nu_ref))
    # the PT2 step on the compressed problem
    q = O.naf_problem(p, thr)
    ref = O.solve(q, cuts=(98.5,))
    gp = pkg.problem_from_synth(p, "cuda", prec, 5 if prec == pkg.SLICED_BF16 else 0)
    gq = pkg.Problem(p.ncore, p.nact, p.nvir, k, Bo[:k].contiguous(), gp.tensors[1], gp.tensors[2], gp.tensors[3],
                     None, p.weights, p.s, prec, 5 if prec == pkg.SLICED_BF16 else 0)
    d = torch.empty((p.nvir, p.nvir), dtype=torch.float64, device="cuda")
    e2 = pkg.dsrg_fno_vv_opdm(gq, d)
    on = torch.empty(p.nvir, dtype=torch.float64, device="cuda")
    no = torch.empty((p.nvir, p.nvir), dtype=torch.float64, device="cuda")
    kk = pkg.dsrg_fno_truncate(p.nvir, d, pkg.MODE_PO, 98.5, 0.01, on, no)
    e_tol, on_tol = (1e-8, 1e-9) if prec == pkg.FP64 else (1e-7, 1e-8)
    print(f"NAF {keep}/{p.naux}: E_vv {e2:.10f} (full basis {O.e_vv(p):.10f}), oracle diff {e2 - ref['e2']:.2e}")
    assert abs(e2 - ref["e2"]) <= e_tol
    assert np.max(np.abs(d.cpu().numpy() - ref["dvv"])) <= 1e-9 * np.max(np.abs(ref["dvv"]))
    assert np.max(np.abs(on.cpu().numpy() - ref["ons"])) <= on_tol
    assert kk == ref["cuts"][98.5]["nkept"]


def test_naf_keeping_everything_leaves_the_energy():
    p = make_problem(ncore=4, nact=2, nvir=70, naux=150, seed=92, nstates=2)
    k, Bo, _ = gpu_naf(p, -1.0, pkg.SLICED_BF16)
    assert k == p.naux
    gp = pkg.problem_from_synth(p, "cuda", pkg.SLICED_BF16, 5)
    gq = pkg.Problem(p.ncore, p.nact, p.nvir, k, Bo, gp.tensors[1], gp.tensors[2], gp.tensors[3], None,
                     p.weights, p.s, pkg.SLICED_BF16, 5)
    assert abs(pkg.dsrg_fno_pt2_energy(gq) - O.e_vv(p)) <= 1e-7


def test_naf_rejects_host_arrays():
    import ctypes
    p = make_problem(ncore=2, nact=0, nvir=20, naux=30, seed=93)
    Bo = torch.zeros((p.naux, 2, 20), dtype=torch.float64, device="cuda")
    k = ctypes.c_int32(-9)
    st = pkg.load().dsrg_fno_naf(2, 20, p.naux, ctypes.c_void_p(p.B.ctypes.data), 0.0, pkg.SLICED_BF16,
                                 ctypes.c_void_p(Bo.data_ptr()), None, ctypes.byref(k), None)
    assert st == -1 and k.value == -9


def test_naf_rejects_non_finite_factors():
    p = make_problem(ncore=2, nact=1, nvir=20, naux=30, seed=94, nstates=2)
    B = torch.from_numpy(np.ascontiguousarray(p.B)).cuda()
    B[3, 1, 7] = float("nan")
    Bo = torch.zeros_like(B)
    with pytest.raises(pkg.DsrgFnoError) as ei:
        pkg.dsrg_fno_naf(3, 21, p.naux, B, 0.0, pkg.SLICED_BF16, Bo)
    assert ei.value.status == -6
