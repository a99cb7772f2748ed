"""Determinant Fock-space brute force of the SA-DSRG-PT2 scalars (test helper).

Evaluates, with explicit matrices over N-electron determinants, the
definitions that Eq. A12 and the vv energy are derived from:
  Gamma^(2)_ef = 1/2 sum_a w_a <Psi_a| [[E_ef, A], A] |Psi_a>      (Eq. A11)
  E_vv         = sum_a w_a <Psi_a| [V, A_vv] + 1/2 [[H0, A_vv], A_vv] |Psi_a>  (Eq. A4)
  E^(2)        = sum_a w_a <Psi_a| [H, A] + 1/2 [[H0, A], A] |Psi_a>  (every class,
                 the Hamiltonian's every block; `hamiltonian`, `energy`)
with A = T - T^+, the cluster operators normal ordered (Mukherjee-Kutzelnigg)
with respect to the ensemble.  The ensemble expectation of a product of
normal-ordered operators is its fully contracted part, so these expectations
are the "[...]_0" scalars of the paper.  Constants dropped from normal-ordered
operators commute with everything and do not change a commutator.

Spin orbital of spatial orbital p and spin s: 2 p + s (s = 0 alpha, 1 beta).
"""
from __future__ import annotations

import itertools

import numpy as np
import scipy.sparse as sps


class FockSpace:
    def __init__(self, norb: int, nelec: int):
        self.norb = norb
        self.nso = 2 * norb
        self.nelec = nelec
        dets = []
        for occ in itertools.combinations(range(self.nso), nelec):
            m = 0
            for o in occ:
                m |= 1 << o
            dets.append(m)
        self.dets = np.array(sorted(dets), dtype=np.int64)
        self.index = {int(d): i for i, d in enumerate(self.dets)}
        self.dim = len(self.dets)
        self._e1 = {}

    def e1(self, p: int, q: int):
        """a^+_p a_q (spin orbitals) as a sparse matrix on the N-electron space."""
        key = (p, q)
        if key in self._e1:
            return self._e1[key]
        rows, cols, vals = [], [], []
        for i, d in enumerate(self.dets):
            d = int(d)
            if not (d >> q) & 1:
                continue
            s = (-1) ** bin(d & ((1 << q) - 1)).count("1")
            d1 = d & ~(1 << q)
            if (d1 >> p) & 1:
                continue
            s *= (-1) ** bin(d1 & ((1 << p) - 1)).count("1")
            d2 = d1 | (1 << p)
            rows.append(self.index[d2])
            cols.append(i)
            vals.append(float(s))
        m = sps.csr_matrix((vals, (rows, cols)), shape=(self.dim, self.dim))
        self._e1[key] = m
        return m

    def e2(self, p, q, r, s):
        """a^{pq}_{rs} = a^+_p a^+_q a_s a_r = a^+_p a_r a^+_q a_s - delta_qr a^+_p a_s."""
        out = self.e1(p, r) @ self.e1(q, s)
        if q == r:
            out = out - self.e1(p, s)
        return out

    # --- states ---------------------------------------------------------
    def vector(self, amplitudes: dict):
        v = np.zeros(self.dim)
        for d, c in amplitudes.items():
            v[self.index[d]] = c
        return v


def so(p, s):
    return 2 * p + s


def _annihilate(vec: dict, q: int):
    out = {}
    for d, c in vec.items():
        if (d >> q) & 1:
            s = (-1) ** bin(d & ((1 << q) - 1)).count("1")
            nd = d & ~(1 << q)
            out[nd] = out.get(nd, 0.0) + s * c
    return out


def _create(vec: dict, p: int):
    out = {}
    for d, c in vec.items():
        if not (d >> p) & 1:
            s = (-1) ** bin(d & ((1 << p) - 1)).count("1")
            nd = d | (1 << p)
            out[nd] = out.get(nd, 0.0) + s * c
    return out


def _dot(a: dict, b: dict):
    return sum(c * b.get(d, 0.0) for d, c in a.items())


def _ket_matrix(fs: FockSpace, psi, idx, order: int):
    """Rows: a_{idx[c]} .. a_{idx[b]} a_{idx[a]} |psi> for every index tuple (a, b, ..)."""
    vec = {int(d): c for d, c in zip(fs.dets, psi) if c != 0.0}
    k = len(idx)
    kets = {}
    for tup in itertools.product(range(k), repeat=order):
        v = vec
        for t in tup:
            v = _annihilate(v, idx[t])
        kets[tup] = v
    keys = sorted({d for v in kets.values() for d in v})
    pos = {d: i for i, d in enumerate(keys)}
    M = np.zeros((k ** order, max(len(keys), 1)))
    for r, tup in enumerate(itertools.product(range(k), repeat=order)):
        for d, c in kets[tup].items():
            M[r, pos[d]] = c
    return M


def rdm_spin_orbital(fs: FockSpace, states, weights, idx, order: int):
    """order 2: gamma2[p][q][r][s] = <a+p a+q a_s a_r>
    order 3: gamma3[p][q][r][s][t][u] = <a+p a+q a+r a_u a_t a_s>, indices in idx.
    <psi| a+p a+q a+r a_u a_t a_s |psi> = <a_r a_q a_p psi | a_u a_t a_s psi>."""
    k = len(idx)
    g = np.zeros((k ** order, k ** order))
    for w, psi in zip(weights, states):
        M = _ket_matrix(fs, psi, idx, order)
        g += w * (M @ M.T)
    return g.reshape((k,) * (2 * order))


def gamma1_spin_orbital(fs: FockSpace, states, weights):
    n = fs.nso
    g1 = np.zeros((n, n))
    for w, psi in zip(weights, states):
        for p in range(n):
            for q in range(n):
                g1[p, q] += w * psi @ (fs.e1(p, q) @ psi)
    return g1


def cumulants(g1, g2, g3=None):
    """Spin-orbital cumulants: lambda2 = gamma2 - (g g - g g);
    lambda3 = gamma3 - sum (-1)^{i+j} g1 lambda2 - sum_perm sgn g1 g1 g1."""
    lam2 = g2 - np.einsum("pr,qs->pqrs", g1, g1) + np.einsum("ps,qr->pqrs", g1, g1)
    if g3 is None:
        return lam2, None
    k = g3.shape[0]
    lam3 = g3.copy()
    up = "pqr"
    lo = "stu"
    for i in range(3):
        for j in range(3):
            ru = "".join(c for n_, c in enumerate(up) if n_ != i)
            rl = "".join(c for n_, c in enumerate(lo) if n_ != j)
            term = np.einsum(f"{up[i]}{lo[j]},{ru}{rl}->pqrstu", g1, lam2)
            lam3 -= (-1) ** (i + j) * term
    for perm in itertools.permutations(range(3)):
        sgn = np.linalg.det(np.eye(3)[list(perm)])
        l = "".join(lo[x] for x in perm)
        term = np.einsum(f"p{l[0]},q{l[1]},r{l[2]}->pqrstu", g1, g1, g1)
        lam3 -= sgn * term
    return lam2, lam3


# ---------------------------------------------------------------------------
# Tiny SA-DSRG system: core doubly occupied, active CAS singlets, virtual empty
# ---------------------------------------------------------------------------
class TinySystem:
    """nc core, na active (with nel_act electrons), nv virtual spatial orbitals.
    Spatial order: core, active, virtual.  Hole h -> spatial h; particle p ->
    spatial nc + p (the same active orbitals appear as holes and particles)."""

    def __init__(self, nc, na, nv, nel_act, nstates, seed, weights=None):
        self.nc, self.na, self.nv = nc, na, nv
        self.norb = nc + na + nv
        self.fs = FockSpace(self.norb, 2 * nc + nel_act)
        rng = np.random.default_rng(seed)
        core = 0
        for m in range(nc):
            core |= (1 << so(m, 0)) | (1 << so(m, 1))
        cas = []
        for occ_a in itertools.combinations(range(na), nel_act // 2):
            for occ_b in itertools.combinations(range(na), nel_act - nel_act // 2):
                d = core
                for u in occ_a:
                    d |= 1 << so(nc + u, 0)
                for u in occ_b:
                    d |= 1 << so(nc + u, 1)
                cas.append(self.fs.index[d])
        cas = np.array(sorted(cas))
        # S^2 = S- S+ + Sz^2 + Sz restricted to the CAS determinants
        fs = self.fs
        splus = sum(fs.e1(so(p, 0), so(p, 1)) for p in range(self.norb))
        sminus = sum(fs.e1(so(p, 1), so(p, 0)) for p in range(self.norb))
        sz = 0.5 * sum(fs.e1(so(p, 0), so(p, 0)) - fs.e1(so(p, 1), so(p, 1))
                       for p in range(self.norb))
        s2 = (sminus @ splus + sz @ sz + sz).toarray()[np.ix_(cas, cas)]
        w, v = np.linalg.eigh(s2)
        singlets = v[:, np.abs(w) < 1e-8]
        coef = singlets @ np.linalg.qr(rng.standard_normal((singlets.shape[1], nstates)))[0]
        self.states = []
        for k in range(nstates):
            psi = np.zeros(fs.dim)
            psi[cas] = coef[:, k]
            self.states.append(psi)
        self.weights = (np.full(nstates, 1.0 / nstates) if weights is None
                        else np.asarray(weights, dtype=np.float64))
        self.g1so = gamma1_spin_orbital(fs, self.states, self.weights)
        act_so = [so(nc + u, s) for u in range(na) for s in (0, 1)]
        self.act_so = act_so
        g2a = rdm_spin_orbital(fs, self.states, self.weights, act_so, 2)
        g3a = rdm_spin_orbital(fs, self.states, self.weights, act_so, 3)
        g1a = self.g1so[np.ix_(act_so, act_so)]
        lam2, lam3 = cumulants(g1a, g2a, g3a)
        # spin-free sums over aligned spins (active index u, spin s -> 2u + s)
        g1r = g1a.reshape(na, 2, na, 2)
        self.gamma1 = np.einsum("usvs->uv", g1r)
        l2r = lam2.reshape(na, 2, na, 2, na, 2, na, 2)
        self.lambda2 = np.einsum("uavbxayb->uvxy", l2r)
        g2r = g2a.reshape(na, 2, na, 2, na, 2, na, 2)
        self.gamma2 = np.einsum("uavbxayb->uvxy", g2r)
        l3r = lam3.reshape(na, 2, na, 2, na, 2, na, 2, na, 2, na, 2)
        self.lambda3 = np.einsum("xaybzcuavbwc->xyzuvw", l3r)
        g3r = g3a.reshape(na, 2, na, 2, na, 2, na, 2, na, 2, na, 2)
        self.gamma3 = np.einsum("xaybzcuavbwc->xyzuvw", g3r)

    # -- index maps
    def hole_spatial(self, h):
        return h

    def part_spatial(self, p):
        return self.nc + p

    def gno2(self, p, q, r, s):
        """{a^{pq}_{rs}} up to a constant (see module docstring)."""
        fs, g = self.fs, self.g1so
        out = fs.e2(p, q, r, s)
        for coef, a, b in ((-g[p, r], q, s), (g[p, s], q, r), (g[q, r], p, s), (-g[q, s], p, r)):
            if coef != 0.0:
                out = out + coef * fs.e1(a, b)
        return out

    def cluster(self, t1=None, t2=None, tol=0.0):
        """T = sum_{ia} t1[i][a] sum_s a+_{a s} a_{i s}
             + 1/2 sum_{ijab} t2[i][j][a][b] sum_{st} {a^{a s, b t}_{i s, j t}}.
        t1: [nh][np], t2: [nh][nh][np][np] spin-free amplitudes."""
        fs = self.fs
        T = sps.csr_matrix((fs.dim, fs.dim))
        nh, npart = self.nc + self.na, self.na + self.nv
        if t1 is not None:
            for i in range(nh):
                for a in range(npart):
                    if abs(t1[i, a]) > tol:
                        for s in (0, 1):
                            T = T + t1[i, a] * fs.e1(so(self.part_spatial(a), s), so(i, s))
        if t2 is not None:
            for i in range(nh):
                for j in range(nh):
                    for a in range(npart):
                        for b in range(npart):
                            t = t2[i, j, a, b]
                            if abs(t) <= tol:
                                continue
                            pa, pb = self.part_spatial(a), self.part_spatial(b)
                            for s in (0, 1):
                                for u in (0, 1):
                                    T = T + 0.5 * t * self.gno2(so(pa, s), so(pb, u), so(i, s), so(j, u))
        return T

    def expect(self, op_apply):
        return sum(w * psi @ op_apply(psi) for w, psi in zip(self.weights, self.states))

    def dvv(self, A):
        """1/2 <[[E_ef, A], A]> for e, f virtual."""
        nv = self.nv
        out = np.zeros((nv, nv))
        base = self.nc + self.na
        for e in range(nv):
            for f in range(nv):
                E = sum(self.fs.e1(so(base + e, s), so(base + f, s)) for s in (0, 1))
                def app(psi):
                    a1 = A @ psi
                    return E @ (A @ a1) - 2.0 * (A @ (E @ a1)) + A @ (A @ (E @ psi))
                out[e, f] = 0.5 * self.expect(app)
        return out

    def h0(self, eps):
        """sum_p eps_p E_pp (constants dropped)."""
        return sum(eps[p] * (self.fs.e1(so(p, 0), so(p, 0)) + self.fs.e1(so(p, 1), so(p, 1)))
                   for p in range(self.norb))

    def v_vv(self, nu_vv):
        """1/2 sum_{klef} <ef|kl> (E^{ef}_{kl} + E^{kl}_{ef}) with <ef|kl> = nu_vv[k][l][e][f]."""
        fs = self.fs
        nh = self.nc + self.na
        base = self.nc + self.na
        V = sps.csr_matrix((fs.dim, fs.dim))
        for k in range(nh):
            for l in range(nh):
                for e in range(self.nv):
                    for f in range(self.nv):
                        c = nu_vv[k, l, e, f]
                        for s in (0, 1):
                            for u in (0, 1):
                                op = fs.e2(so(base + e, s), so(base + f, u), so(k, s), so(l, u))
                                V = V + 0.5 * c * (op + op.T)
        return V

    def hamiltonian(self, eri, f):
        """1/2 sum_{pqrs} <pq|rs> {E^{pq}_{rs}} + sum_{pq} f[p][q] E^p_q over all
        spatial orbitals (eri[p][q][r][s] = <pq|rs>; constants dropped)."""
        fs = self.fs
        H = sps.csr_matrix((fs.dim, fs.dim))
        n = self.norb
        for p in range(n):
            for q in range(n):
                for r in range(n):
                    for s in range(n):
                        c = eri[p, q, r, s]
                        if c == 0.0:
                            continue
                        for a in (0, 1):
                            for b in (0, 1):
                                H = H + 0.5 * c * self.gno2(so(p, a), so(q, b), so(r, a), so(s, b))
                if f[p, q] != 0.0:
                    for a in (0, 1):
                        H = H + f[p, q] * fs.e1(so(p, a), so(q, a))
        return H

    def energy(self, V, H0, A):
        def app(psi):
            a1 = A @ psi
            comm1 = V @ a1 - A @ (V @ psi)
            h = H0 @ a1 - A @ (H0 @ psi)           # [H0, A] psi ... build [[H0,A],A] psi
            ha = H0 @ (A @ a1) - A @ (H0 @ a1)      # [H0, A] (A psi)
            aha = A @ h                              # A [H0, A] psi
            return comm1 + 0.5 * (ha - aha)
        return self.expect(app)
