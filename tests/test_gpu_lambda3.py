"""Eq. A12 term 13 (the 3-cumulant contraction) and the ensemble 3-cumulant on
the GPU (C ABI) against the FP64 oracle.

Tolerances: the cumulant elementwise within 1e-13 of its largest entry;
D_vv with term 13 as the other D_vv parity tests (float64 form: elements
within 1e-10 of max |D|, ONs 1e-9; digit-plane form: ONs 1e-8), identical N'.
"""
import functools
import time

import numpy as np
import pytest

import oracle as O
from synth import ci, make_problem, random_cumulant3, random_density3, workload

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2312_07008_gb300 as pkg  # noqa: E402


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


def ci_gamma3_states(p):
    """Per-state spin-free 3-RDMs of the problem's own CI vectors."""
    n = p.nact
    sa = ci.strings(n, n // 2)
    ta = ci.excitation_table(sa, n)
    return ci.state_gamma3(p.extra["ci"], n, ta, ta)


def gpu_lambda3(w, g1, l2, g3s):
    n = g1.shape[0]
    out = torch.empty((n,) * 6, dtype=torch.float64, device="cuda")
    pkg.dsrg_fno_sa_lambda3(w, cuda(g1), cuda(l2), cuda(g3s), out)
    return out.cpu().numpy()


@pytest.mark.parametrize("nact,nstates", [(6, 3), (7, 2), (4, 1)])
def test_cumulant_from_ci_densities(nact, nstates):
    p = make_problem(2, nact, 5, 7, seed=30 + nact, nstates=nstates, keep_states=True)
    g3s = ci_gamma3_states(p)
    ref = O.sa_lambda3(p.gamma1, p.lambda2, np.einsum("a,a...->...", p.weights, g3s))
    got = gpu_lambda3(p.weights, p.gamma1, p.lambda2, g3s)
    assert np.max(np.abs(got - ref)) <= 1e-13 * np.max(np.abs(ref))


@pytest.mark.parametrize("nact,nstates", [(12, 5), (1, 1), (16, 2)])
def test_cumulant_pointwise_at_size(nact, nstates):
    """Any inputs: the formula is pointwise (sizes up to the nact limit)."""
    rng = np.random.default_rng(nact)
    g1 = rng.standard_normal((nact, nact))
    g1 = g1 + g1.T
    l2 = 0.05 * rng.standard_normal((nact,) * 4)
    g3s = random_density3(nact, nstates, seed=nact) if nact <= 12 else \
        0.05 * rng.standard_normal((nstates,) + (nact,) * 6)
    w = rng.uniform(0.5, 1.0, nstates)
    w /= w.sum()
    ref = O.sa_lambda3(g1, l2, np.einsum("a,a...->...", w, g3s))
    got = gpu_lambda3(w, g1, l2, g3s)
    assert np.max(np.abs(got - ref)) <= 1e-13 * np.max(np.abs(ref))


def test_cumulant_argument_errors():
    g1 = torch.zeros((3, 3), dtype=torch.float64, device="cuda")
    l2 = torch.zeros((3,) * 4, dtype=torch.float64, device="cuda")
    g3 = torch.zeros((2,) + (3,) * 6, dtype=torch.float64, device="cuda")
    out = torch.empty((3,) * 6, dtype=torch.float64, device="cuda")
    with pytest.raises(pkg.DsrgFnoError):
        pkg.dsrg_fno_sa_lambda3([0.7, 0.7], g1, l2, g3, out)        # weights do not sum to 1
    with pytest.raises(pkg.DsrgFnoError):
        pkg.dsrg_fno_sa_lambda3([0.5, 0.5], g1, l2, g3.cpu(), out)  # host 3-RDMs
    bad = g3.clone()
    bad[0, 0, 0, 0, 0, 0, 0] = float("nan")
    with pytest.raises(pkg.DsrgFnoError):
        pkg.dsrg_fno_sa_lambda3([0.5, 0.5], g1, l2, bad, out)


def solve_with_lambda3(p, lam3, precision, cut):
    gp = pkg.problem_from_synth(p, "cuda", precision)
    nv = p.nvir
    d = torch.empty((nv, nv), dtype=torch.float64, device="cuda")
    e2 = pkg.dsrg_fno_vv_opdm_lambda3(gp, cuda(lam3), d)
    on = torch.empty(nv, dtype=torch.float64, device="cuda")
    no = torch.empty((nv, nv), dtype=torch.float64, device="cuda")
    k = pkg.dsrg_fno_truncate(nv, d, pkg.MODE_PO, cut, 0.01, on, no)
    return e2, d.cpu().numpy(), on.cpu().numpy(), k


SHAPES = {
    "cas6": dict(name="sa_cas6_ncore20_nvir300_naux1000"),             # CAS(6,6), 3 states
    "cas7": dict(ncore=4, nact=7, nvir=97, naux=150, nstates=2, seed=8),  # nact^3 = 343: tensor-core contraction
    "cas4": dict(ncore=0, nact=4, nvir=45, naux=40, nstates=2, seed=9),   # no core, nact^3 < 256
}


@functools.lru_cache(maxsize=None)
def reference(key):
    shape = dict(SHAPES[key])
    if "name" in shape:
        p = workload(shape.pop("name"), keep_states=True)
    else:
        p = make_problem(keep_states=True, **shape)
    g3s = ci_gamma3_states(p)
    lam3 = O.sa_lambda3(p.gamma1, p.lambda2, np.einsum("a,a...->...", p.weights, g3s))
    terms = O.dvv_terms(p, lambda3=lam3)
    d = sum(terms.values())
    ref = 0.5 * (d + d.T)
    ons_ref, _ = O.natural_orbitals(ref)
    k_ref = O.truncate(ons_ref, O.MODE_PO, 98.5)
    return p, lam3, ref, ons_ref, k_ref, O.e_vv(p), 0.5 * (terms[13] + terms[13].T)


@pytest.mark.parametrize("key", list(SHAPES))
@pytest.mark.parametrize("precision", ["fp64", "fast"])
def test_dvv_with_term13_matches_oracle(key, precision):
    p, lam3, ref, ons_ref, k_ref, e_ref, sym13 = reference(key)
    prec = pkg.FP64 if precision == "fp64" else pkg.SLICED_BF16
    e2, d, ons, k = solve_with_lambda3(p, lam3, prec, 98.5)
    assert abs(e2 - e_ref) <= (1e-8 if precision == "fp64" else 1e-7)
    dmax = np.max(np.abs(ref))
    assert np.max(np.abs(d - ref)) <= (1e-10 if precision == "fp64" else 1e-9) * dmax
    assert np.max(np.abs(ons - ons_ref)) <= (1e-9 if precision == "fp64" else 1e-8)
    assert k == k_ref
    # term 13 is visible at this tolerance
    assert np.max(np.abs(sym13)) > 1e3 * (1e-10 * dmax)


def test_dvv_without_active_space_ignores_lambda3():
    p = make_problem(3, 0, 20, 30, seed=2)
    gp = pkg.problem_from_synth(p, "cuda", pkg.FP64)
    d0 = torch.empty((20, 20), dtype=torch.float64, device="cuda")
    d1 = torch.empty_like(d0)
    e0 = pkg.dsrg_fno_vv_opdm(gp, d0)
    e1 = pkg.dsrg_fno_vv_opdm_lambda3(gp, None, d1)
    assert abs(e0 - e1) <= 1e-14 * abs(e0)
    assert float(torch.max(torch.abs(d0 - d1))) <= 1e-15 * float(torch.max(torch.abs(d0)))


def test_dvv_lambda3_argument_errors():
    p = make_problem(2, 3, 10, 12, seed=3, nstates=2)
    gp = pkg.problem_from_synth(p, "cuda", pkg.FP64)
    d = torch.empty((10, 10), dtype=torch.float64, device="cuda")
    with pytest.raises(pkg.DsrgFnoError):
        pkg.dsrg_fno_vv_opdm_lambda3(gp, None, d)                      # nact > 0 needs lambda3
    lam = torch.zeros((3,) * 6, dtype=torch.float64)
    with pytest.raises(pkg.DsrgFnoError):
        pkg.dsrg_fno_vv_opdm_lambda3(gp, lam, d)                       # host pointer
    lam = lam.cuda()
    lam[1, 1, 1, 1, 1, 1] = float("inf")
    with pytest.raises(pkg.DsrgFnoError):
        pkg.dsrg_fno_vv_opdm_lambda3(gp, lam, d)


def test_term13_at_cas10_size():
    """CAS(10,10) / ncore 60 / nvir 1200 / naux 3600 with a seeded synthetic
    3-cumulant: D_vv(with term 13) - D_vv(terms 1-12) from the digit-plane
    form against the oracle's symmetrised term 13; prints the added time."""
    p = workload("sa_cas10_ncore60_nvir1200_naux3600")
    lam3 = random_cumulant3(p.nact, seed=77)
    gp = pkg.problem_from_synth(p, "cuda", pkg.SLICED_BF16)
    nv = p.nvir
    d0 = torch.empty((nv, nv), dtype=torch.float64, device="cuda")
    d1 = torch.empty_like(d0)
    lt = cuda(lam3)
    pkg.dsrg_fno_vv_opdm(gp, d0)
    pkg.dsrg_fno_vv_opdm_lambda3(gp, lt, d1)
    times = {}
    for name, f in (("terms 1-12", lambda: pkg.dsrg_fno_vv_opdm(gp, d0)),
                    ("terms 1-13", lambda: pkg.dsrg_fno_vv_opdm_lambda3(gp, lt, d1))):
        torch.cuda.synchronize()
        t = time.perf_counter()
        for _ in range(3):
            f()
        torch.cuda.synchronize()
        times[name] = (time.perf_counter() - t) / 3
    print(f"vv_opdm CAS(10,10) nvir 1200: {times['terms 1-12'] * 1e3:.1f} ms, "
          f"with term 13 {times['terms 1-13'] * 1e3:.1f} ms")
    A = np.arange(p.ncore, p.ncore + p.nact)
    taa = O.t2_semi_internal(p, holes=A)
    t13 = O.dvv_term13(taa, lam3)
    ref = 0.5 * (t13 + t13.T)
    got = (d1 - d0).cpu().numpy()
    dmax = float(torch.max(torch.abs(d0)))
    assert np.max(np.abs(ref)) > 1e-8 * dmax
    assert np.max(np.abs(got - ref)) <= 1e-10 * dmax
