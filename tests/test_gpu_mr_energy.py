"""Full multi-reference PT2 energy E^(2) = <[H, A]> + 1/2 <[[H0, A], A]> over
every amplitude class, and Eq. 11's correction with it, on the GPU (C ABI)
against the FP64 oracle.

Tolerances (the spec bar for energies): |dE| <= 1e-8 E_h in the
float64 form, 1e-7 E_h in the digit-plane form (whose E_vv part and, for
naux >= 256, the integrals of the rest run on the tensor cores; the rest's
element stages are float64 in both); the same N'.  Sizes span
several GEMM tiles with ragged tails, no core, no active orbitals (singles
of f_hp only), with and without the 3-cumulant.
"""
import numpy as np
import pytest

import oracle as O
from synth import make_problem, random_cumulant3, workload

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2312_07008_gb300 as pkg  # noqa: E402

FORMS = ((pkg.FP64, 1e-8), (pkg.SLICED_BF16, 1e-7))


def cuda(a):
    return None if a is None else torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


def with_fock(p, seed, scale=0.02):
    rng = np.random.default_rng(seed)
    p.f_hp = scale * rng.standard_normal((p.nh, p.np_))
    return p


# ncore, nact, nvir, naux, nstates, seed, off-diagonal Fock, 3-cumulant
CASES = [
    (6, 4, 40, 90, 2, 41, True, False),
    (6, 4, 40, 90, 2, 41, True, True),
    (0, 5, 30, 60, 3, 42, False, True),
    (8, 0, 50, 90, 1, 43, True, False),
    (14, 6, 200, 400, 3, 44, True, True),
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: "nc%d_na%d_nv%d_f%d_l3%d" % (c[0], c[1], c[2], c[6], c[7]))
def test_full_energy_matches_oracle(case):
    nc, na, nv, nq, ns, seed, wf, wl3 = case
    p = make_problem(nc, na, nv, nq, seed=seed, nstates=ns)
    if wf:
        with_fock(p, seed)
    l3 = random_cumulant3(na, seed) if (wl3 and na) else None
    ref = O.pt2_energy(p, l3)
    ref_vv = O.e_vv(p)
    assert abs(ref - ref_vv) > 1e-6 * abs(ref)      # the classes beyond vv are not empty
    for prec, tol in FORMS:
        gp = pkg.problem_from_synth(p, "cuda", prec)
        e, evv = pkg.dsrg_fno_pt2_energy_mr(gp, cuda(l3))
        print(f"prec {prec}: E2 {e:.12f} dE {e - ref:+.2e}  E_vv {evv:.12f} dE_vv {evv - ref_vv:+.2e}")
        assert abs(e - ref) <= tol, (e, ref)
        assert abs(evv - ref_vv) <= tol, (evv, ref_vv)
        assert abs(evv - pkg.dsrg_fno_pt2_energy(gp)) <= 1e-12 * abs(evv)


@pytest.mark.parametrize("with_l3", [False, True])
def test_full_energy_cas6_nvir300(with_l3):
    """The CAS(6,6) workload (ncore 20, nvir 300, naux 1000, three states)."""
    p = workload("sa_cas6_ncore20_nvir300_naux1000")
    l3 = random_cumulant3(p.nact, 1) if with_l3 else None
    ref = O.pt2_energy(p, l3)
    for prec, tol in FORMS:
        gp = pkg.problem_from_synth(p, "cuda", prec)
        e, _ = pkg.dsrg_fno_pt2_energy_mr(gp, cuda(l3))
        print(f"prec {prec}: E2 {e:.10f} oracle {ref:.10f} dE {e - ref:+.2e}")
        assert abs(e - ref) <= tol, (e, ref)


def test_full_correction_matches_oracle():
    """Eq. 11 with the full energy at the p_o = 98.5 % cut, and its limits:
    keeping every NO gives 0, keeping none leaves the active particles."""
    p = with_fock(make_problem(10, 4, 120, 240, seed=45, nstates=2), 45)
    l3 = random_cumulant3(p.nact, 45)
    ons_ref, no_ref = O.natural_orbitals(O.dvv(p))
    k_ref = O.truncate(ons_ref, O.MODE_PO, 98.5)
    de_ref, ef_ref, _ = O.discarded_correction_mr(p, no_ref, k_ref, l3)
    _, ef0_ref, _ = O.discarded_correction_mr(p, no_ref, 0, l3)
    for prec, tol in FORMS:
        gp = pkg.problem_from_synth(p, "cuda", prec)
        d = torch.empty((p.nvir, p.nvir), dtype=torch.float64, device="cuda")
        pkg.dsrg_fno_vv_opdm(gp, d)
        on = torch.empty(p.nvir, dtype=torch.float64, device="cuda")
        no = torch.empty((p.nvir, p.nvir), dtype=torch.float64, device="cuda")
        k = pkg.dsrg_fno_truncate(p.nvir, d, pkg.MODE_PO, 98.5, 0.01, on, no)
        assert k == k_ref
        e_mo, _ = pkg.dsrg_fno_pt2_energy_mr(gp, cuda(l3))
        de, ef = pkg.dsrg_fno_discarded_correction_mr(gp, k, no, cuda(l3), e2_mo=e_mo)
        print(f"prec {prec}: N' {k} dE {de:.10f} oracle {de_ref:.10f} diff {de - de_ref:+.2e}")
        assert abs(de - de_ref) <= tol, (de, de_ref)
        assert abs(ef - ef_ref) <= tol, (ef, ef_ref)
        de2, _ = pkg.dsrg_fno_discarded_correction_mr(gp, k, no, cuda(l3))   # E^(2)(MO) evaluated inside
        assert abs(de2 - de) <= tol
        de_all, _ = pkg.dsrg_fno_discarded_correction_mr(gp, p.nvir, no, cuda(l3), e2_mo=e_mo)
        assert abs(de_all) <= tol, de_all
        _, ef0 = pkg.dsrg_fno_discarded_correction_mr(gp, 0, no, cuda(l3), e2_mo=e_mo)
        assert abs(ef0 - ef0_ref) <= 1e-9 * max(1.0, abs(ef0_ref)), (ef0, ef0_ref)


def test_full_energy_rejects_bad_arguments():
    p = make_problem(3, 4, 12, 20, seed=46, nstates=2)
    gp = pkg.problem_from_synth(p, "cuda")
    host_l3 = torch.zeros((4,) * 6, dtype=torch.float64)
    with pytest.raises(pkg.DsrgFnoError):
        pkg.dsrg_fno_pt2_energy_mr(gp, host_l3)
    bad = torch.full((4,) * 6, float("nan"), dtype=torch.float64, device="cuda")
    with pytest.raises(pkg.DsrgFnoError):
        pkg.dsrg_fno_pt2_energy_mr(gp, bad)
    # the workspace stays usable after the rejected calls
    e, _ = pkg.dsrg_fno_pt2_energy_mr(gp)
    assert abs(e - O.pt2_energy(p)) <= 1e-8


def test_full_energy_nvir1200_properties():
    """The benchmark's nvir 1200 / naux 3600 CAS(10,10) workload, fast form,
    where the dense oracle does not fit in memory: its E_vv part against the
    stored oracle value, and the full energy unchanged (to the fast form's
    tolerance) by an orthogonal transformation of the auxiliary index (pairs
    of functions rotated by seeded angles, then permuted), which leaves every
    integral sum_Q B^Q B^Q unchanged in exact arithmetic."""
    import json
    import os
    name = "sa_cas10_ncore60_nvir1200_naux3600"
    ref = json.load(open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", name + ".json")))
    p = workload(name)
    l3 = cuda(random_cumulant3(p.nact, 2))
    e, evv = pkg.dsrg_fno_pt2_energy_mr(pkg.problem_from_synth(p, "cuda", pkg.SLICED_BF16), l3)
    print(f"E2 {e:.9f} E_vv {evv:.9f} stored E_vv {ref['e2']:.9f}")
    assert abs(evv - ref["e2"]) <= 1e-7
    assert abs(e - evv) > 1e-3 * abs(e)
    rng = np.random.default_rng(7)
    th = rng.uniform(0.0, 2.0 * np.pi, p.naux // 2)[:, None, None]
    B = p.B
    B2 = np.empty_like(B)
    B2[0::2] = np.cos(th) * B[0::2] - np.sin(th) * B[1::2]
    B2[1::2] = np.sin(th) * B[0::2] + np.cos(th) * B[1::2]
    p.B = np.ascontiguousarray(B2[rng.permutation(p.naux)])
    del B, B2
    e_rot, evv_rot = pkg.dsrg_fno_pt2_energy_mr(pkg.problem_from_synth(p, "cuda", pkg.SLICED_BF16), l3)
    print(f"rotated: E2 {e_rot:.9f} (diff {e_rot - e:+.2e}), E_vv diff {evv_rot - evv:+.2e}")
    assert abs(e_rot - e) <= 1e-7 and abs(evv_rot - evv) <= 1e-7
