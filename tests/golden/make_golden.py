"""Writes oracle results of a named synthetic workload to tests/golden/.

The stored values come from oracle/ alone (float64 CPU restatement of the
paper: E_vv of Eq. A4 under the vv-class reading, D_vv of Eq. A12, the NOs
of Eq. 8, the cut of Eq. 10 with the near-degeneracy rule and the scalar
correction of Eq. 11) on the seeded inputs of synth/.  They let the GPU
tests check full-size workloads that the oracle cannot rerun within a test.
Besides every ON, the diagonal and row 0 of D_vv, files written now hold
D_vv applied to PROBES seeded normal vectors (every element of D_vv enters).

    OPENBLAS_NUM_THREADS=8 python tests/golden/make_golden.py sa_cas10_ncore60_nvir1200_naux3600
    OPENBLAS_NUM_THREADS=8 python tests/golden/make_golden.py ragged_batch64_seed3
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle as O  # noqa: E402
from synth import workload, CUTS, batch_sizes, batch_problem  # noqa: E402

PROBES, PROBE_SEED = 4, 12345
BATCH = "ragged_batch64_seed3"
BATCH_CUT = 98.5
CITES = ("E_vv: Eq. A4 (vv-class reading); D_vv: Eq. A12 terms 1-12; ONs: Eq. 8; "
         "N': Eq. 10 + near-degeneracy rule of Sec. 2; de: Eq. 11 (scalar)")


def probes(nvir):
    return np.random.default_rng(PROBE_SEED).standard_normal((nvir, PROBES))


def record(p, cuts):
    t0 = time.time()
    res = O.solve(p, cuts=cuts)
    d = res["dvv"]
    return {
        "e2": res["e2"],
        "ons": res["ons"].tolist(),
        "dvv_diag": np.diag(d).tolist(),
        "dvv_row0": d[0].tolist(),
        "dvv_probe": (d @ probes(p.nvir)).T.tolist(),
        "dvv_trace": float(np.trace(d)),
        "dvv_fro": float(np.linalg.norm(d)),
        "asym": float(res["asym"]),
        "cuts": {str(c): {"nkept": int(v["nkept"]), "de": float(v["de"]), "e_fno": float(v["e_fno"])}
                 for c, v in res["cuts"].items()},
        "oracle_seconds": time.time() - t0,
    }


def main(name):
    t0 = time.time()
    if name == BATCH:
        sizes = batch_sizes()
        out = {"workload": name, "source": "oracle/dsrg_pt2.py solve() per instance; inputs "
                                           "synth.batch_problem(k), k = 0..63",
               "cites": CITES, "probe_seed": PROBE_SEED, "probes": PROBES, "cut": BATCH_CUT, "instances": []}
        for k in range(len(sizes)):
            r = record(batch_problem(k), (BATCH_CUT,))
            r.update(k=k, **sizes[k])
            out["instances"].append(r)
            print(f"instance {k}: E2 = {r['e2']:.10f}, {r['oracle_seconds']:.0f} s", flush=True)
    else:
        p = workload(name)
        out = {"workload": name, "source": "oracle/dsrg_pt2.py solve(); inputs synth.workload(name)",
               "cites": CITES, "probe_seed": PROBE_SEED, "probes": PROBES}
        out.update(record(p, CUTS.get(name, (98.5,))))
    out["total_seconds"] = time.time() - t0
    with open(os.path.join(HERE, f"{name}.json"), "w") as f:
        json.dump(out, f, indent=1)
    print(f"{name}: {time.time() - t0:.0f} s")


if __name__ == "__main__":
    main(sys.argv[1])
