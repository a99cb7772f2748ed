"""GPU (CUDA path through the C ABI) against the FP64 CPU oracle.

Tolerances of the plain float64 form: |dE| <= 1e-8 E_h, max |dON| <= 1e-9,
identical N'; D_vv elements within 1e-10 of max |D|; the correction within
1e-8 E_h.
"""
import numpy as np
import pytest

import oracle as O
from synth import make_problem, workload, CUTS

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2312_07008_gb300 as pkg  # noqa: E402

E_TOL, ON_TOL = 1e-8, 1e-9


def gpu_solve(p, cuts, precision=pkg.FP64):
    gp = pkg.problem_from_synth(p, "cuda", precision)
    nv = p.nvir
    d = torch.empty((nv, nv), dtype=torch.float64, device="cuda")
    e2 = pkg.dsrg_fno_vv_opdm(gp, d)
    on = torch.empty(nv, dtype=torch.float64, device="cuda")
    no = torch.empty((nv, nv), dtype=torch.float64, device="cuda")
    out = dict(e2=e2, dvv=d.cpu().numpy(), cuts={})
    for c in cuts:
        k = pkg.dsrg_fno_truncate(nv, d, pkg.MODE_PO, c, 0.01, on, no)
        epsf = torch.empty(max(k, 1), dtype=torch.float64, device="cuda")
        de, ef = pkg.dsrg_fno_discarded_correction(gp, k, no, e2_mo=e2, eps_fno_out=epsf if k else None)
        out["cuts"][c] = dict(nkept=k, de=de, e_fno=ef, eps=epsf.cpu().numpy()[:k])
    out["ons"] = on.cpu().numpy()
    out["no"] = no.cpu().numpy()
    out["e2_only"] = pkg.dsrg_fno_pt2_energy(gp)
    return out


def compare(p, cuts, ref=None):
    if ref is None:
        ref = O.solve(p, cuts=cuts)
    got = gpu_solve(p, cuts)
    assert abs(got["e2"] - ref["e2"]) <= E_TOL, (got["e2"], ref["e2"])
    assert abs(got["e2_only"] - ref["e2"]) <= E_TOL
    dmax = np.max(np.abs(ref["dvv"]))
    assert np.max(np.abs(got["dvv"] - ref["dvv"])) <= 1e-10 * max(dmax, 1e-300)
    assert np.max(np.abs(got["ons"] - ref["ons"])) <= ON_TOL
    for c in cuts:
        g, r = got["cuts"][c], ref["cuts"][c]
        assert g["nkept"] == r["nkept"], (c, g["nkept"], r["nkept"])
        assert abs(g["de"] - r["de"]) <= E_TOL, (c, g["de"], r["de"])
        k = g["nkept"]
        if k:
            assert np.max(np.abs(g["eps"] - r["eps_fno"])) <= 1e-10
            # kept NO subspace (projector) agrees
            P1 = got["no"][:, :k] @ got["no"][:, :k].T
            P2 = ref["no"][:, :k] @ ref["no"][:, :k].T
            assert np.max(np.abs(P1 - P2)) <= 1e-7
    return got, ref


def test_single_reference_workload():
    name = "sr_nocc10_nvir90_naux300"
    compare(workload(name), CUTS[name])


def test_state_averaged_cas6_workload():
    name = "sa_cas6_ncore20_nvir300_naux1000"
    compare(workload(name), CUTS[name])


@pytest.mark.parametrize("shape", [
    dict(ncore=3, nact=2, nvir=67, naux=130, nstates=2),     # ragged tiles
    dict(ncore=1, nact=0, nvir=5, naux=3, nstates=1),         # tiny
    dict(ncore=5, nact=5, nvir=129, naux=65, nstates=3),      # 2 tiles + 1, naux < tile multiples
    dict(ncore=0, nact=4, nvir=40, naux=33, nstates=2),       # no core
    dict(ncore=70, nact=1, nvir=64, naux=17, nstates=2),      # many pairs, one active
])
def test_ragged_shapes(shape):
    p = make_problem(seed=31, s=0.5, **shape)
    compare(p, (98.5, 90.0))


def test_off_diagonal_fock_and_small_s():
    p = make_problem(ncore=4, nact=3, nvir=50, naux=40, seed=33, nstates=2, s=1e-4)
    rng = np.random.default_rng(9)
    p.f_hp = 1e-3 * rng.standard_normal((7, 53))
    compare(p, (99.0,))


def test_s_zero_gives_zero():
    p = make_problem(ncore=3, nact=2, nvir=20, naux=10, seed=34, nstates=2, s=0.0)
    gp = pkg.problem_from_synth(p)
    d = torch.full((20, 20), 7.0, dtype=torch.float64, device="cuda")
    assert pkg.dsrg_fno_vv_opdm(gp, d) == 0.0
    assert torch.count_nonzero(d).item() == 0


def test_truncation_modes_match_oracle():
    p = make_problem(ncore=4, nact=2, nvir=60, naux=50, seed=35, nstates=2)
    ref_d = O.dvv(p)
    n_ref, _ = O.natural_orbitals(ref_d)
    d = torch.from_numpy(ref_d).cuda()
    on = torch.empty(60, dtype=torch.float64, device="cuda")
    no = torch.empty((60, 60), dtype=torch.float64, device="cuda")
    for mode, thr in ((0, 95.0), (0, 100.0), (1, 25.0), (1, 100.0), (2, 1e-3), (2, 1e3), (3, 17.0), (3, 60.0)):
        for ratio in (0.01, 0.0, 0.5):
            k = pkg.dsrg_fno_truncate(60, d, mode, thr, ratio, on, no)
            assert k == O.truncate(n_ref, mode, thr, ratio), (mode, thr, ratio)


def test_cut_matches_truncate_in_every_mode():
    """dsrg_fno_cut on the ONs dsrg_fno_truncate wrote gives the same N' as a
    fresh truncation, for every mode, threshold and widening ratio."""
    p = make_problem(ncore=4, nact=2, nvir=60, naux=50, seed=35, nstates=2)
    ref_d = O.dvv(p)
    n_ref, _ = O.natural_orbitals(ref_d)
    d = torch.from_numpy(ref_d).cuda()
    on = torch.empty(60, dtype=torch.float64, device="cuda")
    no = torch.empty((60, 60), dtype=torch.float64, device="cuda")
    pkg.dsrg_fno_truncate(60, d, 0, 98.0, 0.01, on, no)
    for mode, thr in ((0, 95.0), (0, 100.0), (1, 25.0), (1, 100.0), (2, 1e-3), (2, 1e3), (3, 17.0), (3, 60.0)):
        for ratio in (0.01, 0.0, 0.5):
            k = pkg.dsrg_fno_cut(60, on, mode, thr, ratio)
            assert k == O.truncate(n_ref, mode, thr, ratio), (mode, thr, ratio)


def test_invalid_arguments_are_rejected():
    p = make_problem(ncore=2, nact=2, nvir=10, naux=8, seed=36, nstates=2)
    gp = pkg.problem_from_synth(p)
    d = torch.empty((10, 10), dtype=torch.float64, device="cuda")
    bad = pkg.Problem(2, 2, 10, 8, *gp.tensors, weights=(0.5, 0.6), s=0.5)
    with pytest.raises(pkg.DsrgFnoError) as ei:
        pkg.dsrg_fno_vv_opdm(bad, d)
    assert ei.value.status == -1
    B = gp.tensors[0].clone()
    B[0, 0, 0] = float("nan")
    nanp = pkg.Problem(2, 2, 10, 8, B, *gp.tensors[1:], weights=(0.5, 0.5), s=0.5)
    with pytest.raises(pkg.DsrgFnoError) as ei:
        pkg.dsrg_fno_pt2_energy(nanp)
    assert ei.value.status == -6
    with pytest.raises(pkg.DsrgFnoError):
        pkg.dsrg_fno_truncate(10, d, 7, 1.0, 0.01, d[0], d)
    with pytest.raises(pkg.DsrgFnoError):
        pkg.dsrg_fno_discarded_correction(gp, 11, d)
