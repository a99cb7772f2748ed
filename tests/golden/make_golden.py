"""Writes oracle results of a named synthetic workload to tests/golden/.

The stored values come from oracle/ alone (float64 CPU restatement of the
paper: E_vv of Eq. A4 under the vv-class reading, D_vv of Eq. A12, the NOs
of Eq. 8, the cut of Eq. 10 with the near-degeneracy rule and the scalar
correction of Eq. 11) on the seeded inputs of synth/.  They let the GPU
tests check full-size workloads that the oracle cannot rerun within a test.

    OPENBLAS_NUM_THREADS=8 python tests/golden/make_golden.py sa_cas10_ncore60_nvir1200_naux3600
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
from synth import workload, CUTS  # noqa: E402


def main(name):
    t0 = time.time()
    p = workload(name)
    cuts = CUTS.get(name, (98.5,))
    res = O.solve(p, cuts=cuts)
    d = res["dvv"]
    out = {
        "workload": name,
        "source": "oracle/dsrg_pt2.py solve(); inputs synth.workload(name)",
        "cites": "E_vv: Eq. A4 (vv-class reading); D_vv: Eq. A12 terms 1-12; ONs: Eq. 8; "
                 "N': Eq. 10 + near-degeneracy rule of Sec. 2; de: Eq. 11 (scalar)",
        "e2": res["e2"],
        "ons": res["ons"].tolist(),
        "dvv_diag": np.diag(d).tolist(),
        "dvv_row0": d[0].tolist(),
        "dvv_trace": float(np.trace(d)),
        "dvv_fro": float(np.linalg.norm(d)),
        "asym": float(res["asym"]),
        "cuts": {str(c): {"nkept": int(v["nkept"]), "de": float(v["de"]), "e_fno": float(v["e_fno"])}
                 for c, v in res["cuts"].items()},
        "oracle_seconds": time.time() - t0,
    }
    with open(os.path.join(HERE, f"{name}.json"), "w") as f:
        json.dump(out, f, indent=1)
    print(f"{name}: E2 = {res['e2']:.12f}, {time.time() - t0:.0f} s")


if __name__ == "__main__":
    main(sys.argv[1])
