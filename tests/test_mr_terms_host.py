"""The element bodies of the full PT2 energy kernels (csrc/mr_terms.cuh),
compiled for the host and replayed in stage order by plain loops
(tests/host_replay/mr_terms_replay.cpp), against the oracle's
E^(2) - E_vv on small problems: every index map of the GPU stages checked
without a GPU, over shapes with and without core or active orbitals,
off-diagonal Fock and the 3-cumulant.  Built with AddressSanitizer where the
compiler offers it, so an index outside a buffer fails the test."""
import os
import shutil
import struct
import subprocess

import numpy as np
import pytest

import oracle as O
from synth import make_problem, random_cumulant3

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "host_replay", "mr_terms_replay.cpp")
CUDA_INC = "/usr/local/cuda/include"


@pytest.fixture(scope="module")
def replay(tmp_path_factory):
    cxx = shutil.which("g++")
    if cxx is None or not os.path.exists(os.path.join(CUDA_INC, "cuda_runtime.h")):
        pytest.skip("needs g++ and the CUDA headers")
    exe = str(tmp_path_factory.mktemp("replay") / "mr_replay")
    base = [cxx, "-x", "c++", "-std=c++17", "-O1", "-g", f"-I{CUDA_INC}", SRC, "-o", exe]
    r = subprocess.run(base[:4] + ["-fsanitize=address", "-fno-omit-frame-pointer"] + base[4:],
                       capture_output=True, text=True)
    if r.returncode != 0:
        r = subprocess.run(base, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-2000:]
    return exe


def run_replay(exe, p, l3, path):
    with open(path, "wb") as f:
        f.write(struct.pack("6i", p.ncore, p.nact, p.nvir, p.naux, int(p.f_hp is not None), int(l3 is not None)))
        f.write(struct.pack("d", p.s))
        for a in (p.B, p.eps, p.f_hp, p.gamma1 if p.nact else None, p.lambda2 if p.nact else None, l3):
            if a is not None:
                f.write(np.ascontiguousarray(a, dtype=np.float64).tobytes())
    out = subprocess.run([exe, path], capture_output=True, text=True, check=True)
    return float(out.stdout.split()[0])


# ncore, nact, nvir, naux, nstates, seed
SHAPES = [(3, 4, 9, 20, 2, 1), (2, 3, 7, 15, 3, 2), (4, 0, 8, 20, 1, 3), (0, 4, 6, 12, 2, 4), (5, 6, 10, 25, 3, 5),
          (1, 1, 3, 5, 1, 6)]


@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: "nc%d_na%d_nv%d" % s[:3])
@pytest.mark.parametrize("fock,cum3", [(False, False), (True, False), (True, True)])
def test_element_bodies_replay_the_oracle(replay, tmp_path, shape, fock, cum3):
    nc, na, nv, nq, ns, seed = shape
    p = make_problem(nc, na, nv, nq, seed=seed, nstates=ns)
    if fock:
        p.f_hp = 0.05 * np.random.default_rng(seed).standard_normal((p.nh, p.np_))
    l3 = random_cumulant3(na, seed) if (cum3 and na) else None
    got = run_replay(replay, p, l3, str(tmp_path / "in.bin"))
    ref = O.pt2_energy(p, l3) - O.e_vv(p)
    assert abs(got - ref) <= 1e-12 * max(abs(ref), 1e-3), (got, ref)
