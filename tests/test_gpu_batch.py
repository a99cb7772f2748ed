"""Batched runs over ragged instances (dsrg_fno_batch_run) and the SA
densities helper (dsrg_fno_sa_densities), through the C ABI.

Every instance of a batch must give what the oracle gives for it alone:
E_vv, D_vv, ONs, N' and the discarded-virtual correction, in both
arithmetic forms, with the tolerances of the single-instance parity tests.
"""
import numpy as np
import pytest

import oracle as O
from synth import make_problem
from synth import ci
from synth.problems import batch_sizes, batch_problem

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2312_07008_gb300 as pkg  # noqa: E402

CUT = 98.5


def ragged_small(count=7, seed=41):
    rng = np.random.default_rng(seed)
    out = []
    for k in range(count):
        nc = int(rng.integers(2, 9))
        na = int(rng.choice([0, 2, 4]))
        nv = int(rng.integers(15, 70))
        out.append(make_problem(nc, na, nv, 3 * (nc + na + nv), seed=5000 + k, nstates=int(rng.integers(1, 4))))
    return out


def run_batch(problems, precision, nworkers):
    gps = [pkg.problem_from_synth(p, "cuda", precision) for p in problems]
    dvv = [torch.empty((p.nvir, p.nvir), dtype=torch.float64, device="cuda") for p in problems]
    on = [torch.empty(p.nvir, dtype=torch.float64, device="cuda") for p in problems]
    no = [torch.empty((p.nvir, p.nvir), dtype=torch.float64, device="cuda") for p in problems]
    res = pkg.dsrg_fno_batch_run(gps, dvv, (pkg.MODE_PO, CUT, 0.01), on, no, correction=True, nworkers=nworkers)
    torch.cuda.synchronize()
    return res, dvv, on


@pytest.mark.parametrize("precision,nworkers", [(pkg.FP64, 3), (pkg.SLICED_BF16, 0), (pkg.SLICED_BF16, 1)])
def test_ragged_batch_matches_oracle_per_instance(precision, nworkers):
    problems = ragged_small()
    res, dvv, on = run_batch(problems, precision, nworkers)
    e_tol = 1e-8 if precision == pkg.FP64 else 1e-7
    for p, r, d, o in zip(problems, res, dvv, on):
        ref = O.solve(p, cuts=(CUT,))
        assert r["status"] == 0
        assert abs(r["e2"] - ref["e2"]) <= e_tol
        dmax = np.abs(ref["dvv"]).max()
        assert np.abs(d.cpu().numpy() - ref["dvv"]).max() <= 1e-9 * dmax
        assert np.abs(o.cpu().numpy() - ref["ons"]).max() <= 1e-8
        assert r["nkept"] == ref["cuts"][CUT]["nkept"]
        assert abs(r["de"] - ref["cuts"][CUT]["de"]) <= e_tol


def test_autotuner_tries_each_candidate_then_settles():
    problems = ragged_small(count=5, seed=43)
    seen = []
    for _ in range(4):
        run_batch(problems, pkg.SLICED_BF16, 0)
        seen.append(pkg.dsrg_fno_batch_last_workers())
    # 5 instances: candidates 2, 4, 8 (capped at 5), then the fastest of them
    assert seen[:3] == [2, 4, 5]
    assert seen[3] in (2, 4, 5)


def test_energy_only_items_and_bad_requests():
    problems = ragged_small(count=3, seed=44)
    gps = [pkg.problem_from_synth(p, "cuda", pkg.FP64) for p in problems]
    res = pkg.dsrg_fno_batch_run(gps, nworkers=2)
    for p, r in zip(problems, res):
        assert r["status"] == 0 and r["nkept"] == 0 and r["de"] == 0.0
        assert abs(r["e2"] - O.e_vv(p)) <= 1e-8
    # a cut without D_vv output is rejected per item
    on = [torch.empty(p.nvir, dtype=torch.float64, device="cuda") for p in problems]
    with pytest.raises(pkg.DsrgFnoError):
        pkg.dsrg_fno_batch_run(gps, None, (pkg.MODE_PO, CUT, 0.01), on, on, nworkers=2)


def test_sampled_instances_of_the_64_instance_batch():
    """The 64-instance ragged batch at full size, as the benchmark runs it:
    the three smallest instances are checked against the oracle."""
    sizes = batch_sizes()
    problems = [batch_problem(k) for k in range(len(sizes))]
    res, dvv, on = run_batch(problems, pkg.SLICED_BF16, 0)
    assert all(r["status"] == 0 for r in res)
    cost = [s["naux"] * s["nvir"] ** 2 * (s["ncore"] + s["nact"]) ** 2 for s in sizes]
    for k in np.argsort(cost)[:3]:
        ref = O.solve(problems[k], cuts=(CUT,))
        assert abs(res[k]["e2"] - ref["e2"]) <= 1e-7
        assert np.abs(on[k].cpu().numpy() - ref["ons"]).max() <= 1e-8
        assert res[k]["nkept"] == ref["cuts"][CUT]["nkept"]
        assert abs(res[k]["de"] - ref["cuts"][CUT]["de"]) <= 1e-7


def test_sa_densities_match_ensemble_definition():
    rng = np.random.default_rng(9)
    nact, nst = 4, 3
    vecs, _, ta, tb = ci.random_ci_vectors(rng, nact, nst, None)
    w = np.array([0.5, 0.3, 0.2])
    g1s, g2s = zip(*[ci.spin_free_rdms(c, nact, ta, tb) for c in vecs])
    g1, lam2 = pkg.dsrg_fno_sa_densities(w, np.array(g1s), np.array(g2s))
    g1_ref = sum(wi * a for wi, a in zip(w, g1s))
    g2_ref = sum(wi * b for wi, b in zip(w, g2s))
    np.testing.assert_allclose(g1, g1_ref, atol=1e-14)
    # the cumulant reproduces the averaged Gamma2 through the oracle's relation
    np.testing.assert_allclose(O.gamma2_from_cumulant(g1, lam2), g2_ref, atol=1e-13)
    with pytest.raises(pkg.DsrgFnoError):
        pkg.dsrg_fno_sa_densities([0.5, 0.3, 0.3], np.array(g1s), np.array(g2s))
    with pytest.raises(pkg.DsrgFnoError):
        pkg.dsrg_fno_sa_densities([1.2, -0.1, -0.1], np.array(g1s), np.array(g2s))
