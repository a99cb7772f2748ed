"""Determinant-space helpers for the synthetic reference ensembles.

The reference states of a state-averaged computation are CI vectors in a
complete active space (CAS).  This module builds spin-free reduced density
matrices of such vectors.  It is input preparation (what an SA-CASSCF code
hands to SA-DSRG), not part of the SA-DSRG method, and serves both the CUDA
path's tests and the oracle's.

Conventions (paper Appendix A, Eq. A1 and the definitions after Eq. A12):
  E_pq = sum_sigma a^+_{p sigma} a_{q sigma}
  Gamma1[p][q]       = <E_pq>
  Gamma2[p][q][r][s] = sum_{sigma tau} <a^+_{p s} a^+_{q t} a_{s t} a_{r s}>
                     = <E_pr E_qs> - delta_qr <E_ps>
A determinant is an (alpha string, beta string) pair, with all alpha creators
ordered before the beta creators; a string is a bitmask over active orbitals.
"""
from __future__ import annotations

import itertools
from dataclasses import dataclass

import numpy as np


def strings(norb: int, nel: int) -> np.ndarray:
    """All bitmasks of `norb` orbitals holding `nel` electrons, ascending."""
    out = []
    for occ in itertools.combinations(range(norb), nel):
        m = 0
        for o in occ:
            m |= 1 << o
        out.append(m)
    return np.array(sorted(out), dtype=np.int64)


def _popcount_below(mask: int, k: int) -> int:
    return bin(mask & ((1 << k) - 1)).count("1")


@dataclass
class ExcitationTable:
    """For every (p, q): the strings reached by a^+_p a_q, with signs."""
    norb: int
    src: dict
    dst: dict
    sign: dict


def excitation_table(strs: np.ndarray, norb: int) -> ExcitationTable:
    index = {int(s): i for i, s in enumerate(strs)}
    src, dst, sgn = {}, {}, {}
    for p in range(norb):
        for q in range(norb):
            a, b, c = [], [], []
            for i, s in enumerate(strs):
                s = int(s)
                if not (s >> q) & 1:
                    continue
                s1 = s & ~(1 << q)
                ph = (-1) ** _popcount_below(s, q)
                if (s1 >> p) & 1:
                    continue
                s2 = s1 | (1 << p)
                ph *= (-1) ** _popcount_below(s1, p)
                a.append(i)
                b.append(index[s2])
                c.append(ph)
            src[(p, q)] = np.array(a, dtype=np.int64)
            dst[(p, q)] = np.array(b, dtype=np.int64)
            sgn[(p, q)] = np.array(c, dtype=np.float64)
    return ExcitationTable(norb, src, dst, sgn)


def apply_E(C: np.ndarray, p: int, q: int, ta: ExcitationTable, tb: ExcitationTable) -> np.ndarray:
    """E_pq acting on a CI matrix C[alpha string][beta string]."""
    out = np.zeros_like(C)
    # a^+_p a_q is one-to-one on the strings where it is defined, so the
    # destination indices are unique and plain fancy indexing accumulates.
    s, d, g = ta.src[(p, q)], ta.dst[(p, q)], ta.sign[(p, q)]
    out[d, :] += g[:, None] * C[s, :]
    s, d, g = tb.src[(p, q)], tb.dst[(p, q)], tb.sign[(p, q)]
    out[:, d] += g[None, :] * C[:, s]
    return out


def spin_free_rdms(C: np.ndarray, norb: int, ta: ExcitationTable, tb: ExcitationTable):
    """Spin-free Gamma1 and Gamma2 of one CI vector (see module docstring)."""
    X = np.empty((norb, norb) + C.shape)
    for p in range(norb):
        for q in range(norb):
            X[p, q] = apply_E(C, p, q, ta, tb)
    flat = X.reshape(norb * norb, -1)
    g1 = (flat @ C.reshape(-1)).reshape(norb, norb)
    gram = flat @ flat.T                      # <E_ab Psi | E_cd Psi>
    gram = gram.reshape(norb, norb, norb, norb)
    # <E_pr E_qs> = <E_rp Psi | E_qs Psi> = gram[r][p][q][s]
    g2 = np.einsum("rpqs->pqrs", gram).copy()
    eye = np.eye(norb)
    g2 -= np.einsum("qr,ps->pqrs", eye, g1)
    return g1, g2


def spin_free_rdm3(C: np.ndarray, norb: int, ta: ExcitationTable, tb: ExcitationTable,
                   g2: np.ndarray) -> np.ndarray:
    """Spin-free 3-RDM of one CI vector,
    Gamma3[p][q][r][s][t][u] = sum_{sigma tau rho} <a+_{p sigma} a+_{q tau} a+_{r rho} a_{u rho} a_{t tau} a_{s sigma}>,
    from products of E operators:
      E_qt E_ru       = e^{qr}_{tu} + delta_tr E_qu
      E_ps e^{qr}_{tu} = e^{pqr}_{stu} + delta_sq e^{pr}_{tu} + delta_sr e^{pq}_{ut}
    so Gamma3 = <E_ps E_qt E_ru> - delta_tr <E_ps E_qu> - delta_sq Gamma2[p][r][t][u]
              - delta_sr Gamma2[p][q][u][t], with <E_ps X> = <E_sp Psi | X Psi>.
    g2 is the same vector's Gamma2 (spin_free_rdms)."""
    n = norb
    X = np.empty((n, n) + C.shape)
    for p in range(n):
        for q in range(n):
            X[p, q] = apply_E(C, p, q, ta, tb)
    flat = X.reshape(n * n, -1)               # row (s, p): E_sp Psi
    m3 = np.empty((n,) * 6)                   # m3[s][p][q][t][r][u] = <E_sp Psi | E_qt E_ru Psi>
    for r in range(n):
        for u in range(n):
            Y = np.empty((n, n) + C.shape)
            for q in range(n):
                for t in range(n):
                    Y[q, t] = apply_E(X[r, u], q, t, ta, tb)
            m3[:, :, :, :, r, u] = (flat @ Y.reshape(n * n, -1).T).reshape(n, n, n, n)
    g3 = np.einsum("spqtru->pqrstu", m3).copy()
    gram = (flat @ flat.T).reshape(n, n, n, n)   # gram[s][p][q][u] = <E_ps E_qu>
    eye = np.eye(n)
    g3 -= np.einsum("tr,spqu->pqrstu", eye, gram)
    g3 -= np.einsum("sq,prtu->pqrstu", eye, g2)
    g3 -= np.einsum("sr,pqut->pqrstu", eye, g2)
    return g3


def random_ci_vectors(rng: np.random.Generator, norb: int, nstates: int,
                      ndet_sparse: int | None = None):
    """Seeded random normalised CI vectors in the Sz = 0 CAS(norb, norb) space.

    With `ndet_sparse`, each vector has that many nonzero determinants, drawn
    without replacement; otherwise all determinants carry a N(0,1) coefficient.
    Returns (list of C matrices, alpha strings, alpha table, beta table).
    """
    nel = norb // 2
    sa = strings(norb, nel)
    na = len(sa)
    ta = excitation_table(sa, norb)
    vecs = []
    for _ in range(nstates):
        if ndet_sparse is None:
            c = rng.standard_normal((na, na))
        else:
            idx = rng.choice(na * na, size=ndet_sparse, replace=False)
            val = rng.standard_normal(ndet_sparse)
            c = np.zeros(na * na)
            c[idx] = val
            c = c.reshape(na, na)
        c /= np.linalg.norm(c)
        vecs.append(c)
    return vecs, sa, ta, ta


def state_averaged_densities(vecs, weights, norb, ta, tb):
    """SA Gamma1 (Eq. A1), SA Gamma2, and the SA 2-cumulant.

    Lambda2[p][q][r][s] = Gamma2 - Gamma1[p][r] Gamma1[q][s]
                          + 1/2 Gamma1[p][s] Gamma1[q][r]
    i.e. the relation stated after Eq. A12 solved for the cumulant, applied to
    the ensemble-averaged Gamma1 and Gamma2.
    """
    g1 = np.zeros((norb, norb))
    g2 = np.zeros((norb,) * 4)
    for w, c in zip(weights, vecs):
        a, b = spin_free_rdms(c, norb, ta, tb)
        g1 += w * a
        g2 += w * b
    lam2 = g2 - np.einsum("pr,qs->pqrs", g1, g1) + 0.5 * np.einsum("ps,qr->pqrs", g1, g1)
    return g1, g2, lam2


def state_gamma3(vecs, norb, ta, tb):
    """Per-state spin-free 3-RDMs [nstates][norb]^6 (spin_free_rdm3)."""
    out = []
    for c in vecs:
        _, g2 = spin_free_rdms(c, norb, ta, tb)
        out.append(spin_free_rdm3(c, norb, ta, tb, g2))
    return np.array(out)
