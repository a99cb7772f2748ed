"""Full-size workloads against stored oracle values (tests/golden/*.json).

The oracle cannot rerun the full-size workloads inside a test (nvir 1200 takes
about an hour on eight cores), so tests/golden/make_golden.py stored its
results once; here the CUDA path, in both arithmetic forms and in the launch
configuration the benchmark uses, is compared with them: E_vv, every ON,
diag and row 0 of D_vv (and its products with seeded probe vectors where
stored), N' and the correction of every cut.
"""
import functools
import glob
import json
import os

import numpy as np
import pytest

from synth import workload

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import bench  # noqa: E402
import paper_2312_07008_gb300 as pkg  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))
# single workloads (the ragged batch has its own test)
FILES = sorted(f for f in glob.glob(os.path.join(HERE, "golden", "*.json")) if "batch" not in os.path.basename(f))


@functools.lru_cache(maxsize=None)
def problem(name):
    return workload(name)  # generated once for both arithmetic forms


def run(p, cuts, precision):
    gp = pkg.problem_from_synth(p, "cuda", precision, 5 if precision == pkg.SLICED_BF16 else 0)
    nv = p.nvir
    d = torch.empty((nv, nv), dtype=torch.float64, device="cuda")
    e2 = pkg.dsrg_fno_vv_opdm(gp, d)
    on = torch.empty(nv, dtype=torch.float64, device="cuda")
    no = torch.empty((nv, nv), dtype=torch.float64, device="cuda")
    out = {"e2": e2, "dvv": d.cpu().numpy(), "cuts": {}}
    for i, c in enumerate(cuts):
        if i == 0:
            k = pkg.dsrg_fno_truncate(nv, d, pkg.MODE_PO, c, 0.01, on, no)
        else:
            k = pkg.dsrg_fno_cut(nv, on, pkg.MODE_PO, c, 0.01)
        de, ef = pkg.dsrg_fno_discarded_correction(gp, k, no, e2_mo=e2)
        out["cuts"][c] = (k, de, ef)
    out["ons"] = on.cpu().numpy()
    return out


@pytest.mark.parametrize("precision", [pkg.SLICED_BF16, pkg.FP64], ids=["fast", "fp64"])
@pytest.mark.parametrize("path", FILES, ids=[os.path.basename(f)[:-5] for f in FILES])
def test_workload_matches_stored_oracle(path, precision):
    ref = json.load(open(path))
    p = problem(ref["workload"])
    cuts = [float(c) for c in ref["cuts"]]
    got = run(p, cuts, precision)
    e_tol = 1e-7 if precision == pkg.SLICED_BF16 else 1e-8
    on_tol = 1e-8 if precision == pkg.SLICED_BF16 else 1e-9
    assert abs(got["e2"] - ref["e2"]) <= e_tol, (got["e2"], ref["e2"])
    assert np.abs(got["ons"] - np.array(ref["ons"])).max() <= on_tol
    dmax = np.abs(np.array(ref["dvv_diag"])).max()
    assert np.abs(np.diag(got["dvv"]) - np.array(ref["dvv_diag"])).max() <= 1e-9 * dmax
    assert np.abs(got["dvv"][0] - np.array(ref["dvv_row0"])).max() <= 1e-9 * dmax
    if "dvv_probe" in ref:   # D_vv applied to seeded normal vectors: every element enters
        R = np.random.default_rng(ref["probe_seed"]).standard_normal((p.nvir, ref["probes"]))
        pr = (got["dvv"] @ R).T
        assert np.abs(pr - np.array(ref["dvv_probe"])).max() <= 1e-9 * dmax * np.sqrt(p.nvir)
    for c in cuts:
        k, de, ef = got["cuts"][c]
        r = ref["cuts"][str(c)] if str(c) in ref["cuts"] else ref["cuts"][repr(c)]
        # how far the cut was from moving (cumulative-fraction margins, widening stop gap)
        print(ref["workload"], precision, bench.cut_margins(got["ons"], c, k))
        assert k == r["nkept"], (c, k, r["nkept"])
        assert abs(de - r["de"]) <= e_tol, (c, de, r["de"])
