"""Seeded synthetic SA-DSRG-PT2 problems shaped like the paper's workloads.

The paper's molecules (QUESTDB, Ni(CO)4, FeCl(Cor)) need integrals and
SA-CASSCF references that are not available here, so every problem is drawn
from a seeded generator with the shapes of those workloads.  This module only
draws numbers; it contains none of the SA-DSRG arithmetic.

Recipe for one problem with seed `seed` (all draws from one
numpy.random.default_rng(seed), in this order):
  1. Z = standard_normal((naux, nh, np)), nh = ncore + nact holes,
     np = nact + nvir particles.  The active(hole) x active(particle) block is
     symmetrised, Z[:, u, x] <- (Z[:, u, x] + Z[:, x, u]) / sqrt(2), because
     B^Q_{uv} = B^Q_{vu} for a real orbital pair.
  2. eps_core ~ U[-2.0, -0.3], eps_act ~ U[-0.5, 0.3], eps_vir ~ U[0.1, 5.0],
     each sorted ascending (semicanonical orbital energies, E_h).
  3. nstates random normalised CI vectors in the Sz = 0 CAS(nact, nact)
     determinant space (dense, or with `ndet_sparse` nonzeros each).
  B[Q, p, q] = 0.05 * exp(-0.01 * (loc(p) + loc(q))) * Z[Q, p, q], where
  loc() is the index inside the orbital's own block (core, active, virtual).
The state weights are equal.  The SA Gamma1 / Lambda2 follow from `synth.ci`.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import ci


@dataclass
class Problem:
    ncore: int
    nact: int
    nvir: int
    naux: int
    B: np.ndarray                 # [naux][ncore+nact][nact+nvir], float64
    eps: np.ndarray               # [ncore+nact+nvir], core | active | virtual
    gamma1: np.ndarray | None     # [nact][nact] SA spin-free 1-RDM
    lambda2: np.ndarray | None    # [nact]^4 SA spin-free 2-cumulant
    weights: np.ndarray           # state weights
    s: float = 0.5                # flow parameter s1 (E_h^-2)
    f_hp: np.ndarray | None = None  # optional off-diagonal Fock f_a^i, [nh][np]
    name: str = ""
    extra: dict = field(default_factory=dict)

    @property
    def nh(self) -> int:
        return self.ncore + self.nact

    @property
    def np_(self) -> int:
        return self.nact + self.nvir


def make_problem(ncore: int, nact: int, nvir: int, naux: int, seed: int,
                 nstates: int = 1, s: float = 0.5, ndet_sparse: int | None = None,
                 name: str = "", keep_states: bool = False) -> Problem:
    rng = np.random.default_rng(seed)
    nh, npart = ncore + nact, nact + nvir
    Z = rng.standard_normal((naux, nh, npart))
    if nact:
        za = Z[:, ncore:, :nact]
        Z[:, ncore:, :nact] = (za + za.transpose(0, 2, 1)) / np.sqrt(2.0)
    eps_c = np.sort(rng.uniform(-2.0, -0.3, ncore))
    eps_a = np.sort(rng.uniform(-0.5, 0.3, nact))
    eps_v = np.sort(rng.uniform(0.1, 5.0, nvir))
    loc_h = np.concatenate([np.arange(ncore), np.arange(nact)]).astype(np.float64)
    loc_p = np.concatenate([np.arange(nact), np.arange(nvir)]).astype(np.float64)
    scale = 0.05 * np.exp(-0.01 * (loc_h[:, None] + loc_p[None, :]))
    B = Z * scale[None, :, :]
    del Z
    gamma1 = lambda2 = None
    extra = {}
    if nact:
        vecs, _, ta, tb = ci.random_ci_vectors(rng, nact, nstates, ndet_sparse)
        w = np.full(nstates, 1.0 / nstates)
        gamma1, g2, lambda2 = ci.state_averaged_densities(vecs, w, nact, ta, tb)
        if keep_states:
            extra["gamma2"] = g2
            extra["ci"] = vecs
    else:
        w = np.full(max(nstates, 1), 1.0 / max(nstates, 1))
    return Problem(ncore, nact, nvir, naux, np.ascontiguousarray(B),
                   np.concatenate([eps_c, eps_a, eps_v]), gamma1, lambda2, w, s,
                   None, name, extra)


# The five workloads, by what they are.  "sr" = single-reference limit.
WORKLOADS = {
    "sr_nocc10_nvir90_naux300": dict(ncore=10, nact=0, nvir=90, naux=300, seed=0, nstates=1),
    "sa_cas6_ncore20_nvir300_naux1000": dict(ncore=20, nact=6, nvir=300, naux=1000, seed=1, nstates=3),
    "sa_cas10_ncore60_nvir1200_naux3600": dict(ncore=60, nact=10, nvir=1200, naux=3600, seed=2, nstates=4),
    "sa_cas12_ncore95_nvir1000_naux4200": dict(ncore=95, nact=12, nvir=1000, naux=4200, seed=4,
                                               nstates=5, ndet_sparse=20000),
}

# FNO cuts (percent of cumulative occupation) quoted with each workload.
CUTS = {
    "sr_nocc10_nvir90_naux300": (98.5,),
    "sa_cas6_ncore20_nvir300_naux1000": (98.5,),
    "sa_cas10_ncore60_nvir1200_naux3600": (98.0, 99.0),
    "sa_cas12_ncore95_nvir1000_naux4200": (98.5,),
}


def workload(name: str, **kw) -> Problem:
    args = dict(WORKLOADS[name])
    args.update(kw)
    return make_problem(name=name, **args)


def batch_sizes(seed: int = 3, count: int = 64):
    """Shapes of the 64-instance ragged batch: ncore U{10..60},
    nact in {0,4,6,8}, 2-5 states, nvir U{100..800}, naux = 3 (ncore+nact+nvir)."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        ncore = int(rng.integers(10, 61))
        nact = int(rng.choice([0, 4, 6, 8]))
        nstates = int(rng.integers(2, 6))
        nvir = int(rng.integers(100, 801))
        out.append(dict(ncore=ncore, nact=nact, nvir=nvir,
                        naux=3 * (ncore + nact + nvir), nstates=nstates))
    return out


def batch_problem(k: int, seed: int = 3) -> Problem:
    """Instance k of the ragged batch; its data come from seed 1000*seed + k."""
    sz = batch_sizes(seed)[k]
    return make_problem(seed=1000 * seed + k, name=f"batch{seed}_{k}", **sz)


def _pair_symmetrised(R: np.ndarray) -> np.ndarray:
    """Average of a [n]^6 tensor over the six simultaneous permutations of its
    index pairs (0,3), (1,4), (2,5) and over the exchange of the upper and
    lower triples: the symmetries of a real 3-RDM and of its cumulant."""
    import itertools
    out = np.zeros_like(R)
    for perm in itertools.permutations(range(3)):
        out += np.transpose(R, list(perm) + [3 + i for i in perm])
    out = out + np.transpose(out, (3, 4, 5, 0, 1, 2))
    return out / 12.0


def random_density3(nact: int, nstates: int, seed: int, scale: float = 0.05) -> np.ndarray:
    """[nstates][nact]^6 seeded random tensors with the symmetries of spin-free
    3-RDMs: stand-ins for the per-state 3-RDMs of active spaces whose CI
    3-RDM is too costly to form here (normal draws, pair-symmetrised, times
    `scale`)."""
    rng = np.random.default_rng(seed)
    return np.array([scale * _pair_symmetrised(rng.standard_normal((nact,) * 6)) for _ in range(nstates)])


def random_cumulant3(nact: int, seed: int, scale: float = 0.03) -> np.ndarray:
    """[nact]^6 seeded random tensor with the symmetries of the spin-free
    3-cumulant: mean |entry| about scale/4, largest about 1.4 scale, which for
    the default matches the 3-cumulants of the random CAS(6,6) ensembles here
    (mean 0.008, largest 0.05)."""
    rng = np.random.default_rng(seed)
    return scale * _pair_symmetrised(rng.standard_normal((nact,) * 6))
