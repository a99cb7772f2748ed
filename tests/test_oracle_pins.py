"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: a closed
form, a limit, brute force over explicit indices or over determinants, a
library routine, or an invariance.
"""
import itertools

import numpy as np
import pytest

import oracle as O
from synth import make_problem, random_cumulant3
from fockspace import TinySystem, so


# ---------------------------------------------------------------- regularizer
def test_regularizer_against_high_precision():
    """Eq. A7 regularizer, both branches, against 50-digit arithmetic."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 50
    s = 0.5
    deltas = [-7.3, -2.0, -0.8, -0.2, -0.05, -0.044, -0.0447, -1e-3, -1e-6, -1e-12,
              1e-9, 0.02, 0.0447213, 0.3, 1.7]
    for c in (1.0, 2.0):
        got = O.regularizer(np.array(deltas), s, c)
        for d, g in zip(deltas, got):
            ref = (1 - mp.exp(-c * s * mp.mpf(d) ** 2)) / mp.mpf(d)
            assert abs(g - float(ref)) <= 4e-16 * abs(float(ref)), (d, c, g, ref)
    assert O.regularizer(np.array([0.0]), s)[0] == 0.0
    assert np.all(O.regularizer(np.array([-1.0, 0.5]), 0.0) == 0.0)


# ------------------------------------------------------- single-reference limit
@pytest.fixture(scope="module")
def sr_problem():
    return make_problem(ncore=4, nact=0, nvir=9, naux=17, seed=5, s=0.5)


def _so_integrals(prob):
    """Antisymmetrised spin-orbital <ij||ab> for a closed-shell SR problem,
    built by explicit loops from the DF factors."""
    nc, nv = prob.ncore, prob.nvir
    B = prob.B
    g = np.zeros((2 * nc, 2 * nc, 2 * nv, 2 * nv))
    for I, J, A, Bb in itertools.product(range(2 * nc), range(2 * nc), range(2 * nv), range(2 * nv)):
        i, si = divmod(I, 2)
        j, sj = divmod(J, 2)
        a, sa = divmod(A, 2)
        b, sb = divmod(Bb, 2)
        direct = sum(B[q, i, a] * B[q, j, b] for q in range(B.shape[0])) if (si == sa and sj == sb) else 0.0
        exch = sum(B[q, i, b] * B[q, j, a] for q in range(B.shape[0])) if (si == sb and sj == sa) else 0.0
        g[I, J, A, Bb] = direct - exch
    return g


def test_sr_large_s_is_mp2(sr_problem):
    """s -> infinity: E_vv -> closed-shell MP2, D_vv -> MP2 unrelaxed vv density
    (the single-reference statement after Eq. A12).  MP2 is evaluated in the
    spin-orbital textbook form: E = 1/4 sum <ij||ab>^2/D, P_ab = 1/2 sum t_ac t_bc."""
    prob = sr_problem
    prob_inf = make_problem(ncore=4, nact=0, nvir=9, naux=17, seed=5, s=1.0e4)
    g = _so_integrals(prob)
    nc, nv = prob.ncore, prob.nvir
    e = np.repeat(prob.eps[:nc], 2)
    ev = np.repeat(prob.eps[nc:], 2)
    D = e[:, None, None, None] + e[None, :, None, None] - ev[None, None, :, None] - ev[None, None, None, :]
    t = g / D
    emp2 = 0.25 * np.sum(g * t)
    pab = 0.5 * np.einsum("ijac,ijbc->ab", t, t)
    p_sf = pab[0::2, 0::2] + pab[1::2, 1::2]
    assert abs(O.e_vv(prob_inf) - emp2) <= 1e-12 * abs(emp2)
    d = O.dvv(prob_inf)
    assert np.max(np.abs(d - p_sf)) <= 1e-12 * np.max(np.abs(p_sf))
    # at finite s the energy is strictly smaller in magnitude
    assert abs(O.e_vv(prob)) < abs(emp2)


def test_sr_small_s_limit(sr_problem):
    """s -> 0: R2 = 2 s Delta + O(s^2), so E_vv / s -> 2 sum nu (2 nu - nu_swap) Delta;
    D_vv = O(s^2); at s = 0 everything vanishes."""
    base = dict(ncore=4, nact=0, nvir=9, naux=17, seed=5)
    p0 = make_problem(s=0.0, **base)
    assert O.e_vv(p0) == 0.0
    assert np.all(O.dvv(p0) == 0.0)
    nc, nv = 4, 9
    lin = 0.0
    for m in range(nc):
        for n in range(nc):
            nu = p0.B[:, m, :].T @ p0.B[:, n, :]
            nus = p0.B[:, n, :].T @ p0.B[:, m, :]      # nu^{nm}_{ef} = (en|fm)
            d = p0.eps[m] + p0.eps[n] - p0.eps[nc:][:, None] - p0.eps[nc:][None, :]
            lin += np.sum(nu * (2 * nu - nus) * 2.0 * d)
    for s in (1e-4, 1e-5):
        ps = make_problem(s=s, **base)
        assert abs(O.e_vv(ps) / s - lin) <= 2.0 * s * 60.0 * abs(lin)
        d2 = O.dvv(ps)
        ps2 = make_problem(s=2 * s, **base)
        ratio = np.linalg.norm(O.dvv(ps2)) / np.linalg.norm(d2)
        # D ~ s^2 (1 + O(s Delta^2)); Delta^2 <= 60 here
        assert abs(ratio - 4.0) < 4.0 * 2.0 * s * 60.0


# ----------------------------------------------------------- 4-index brute force
def test_four_index_brute_force_energy():
    """E_vv from explicitly formed (ai|bj) integrals and index loops."""
    prob = make_problem(ncore=2, nact=2, nvir=3, naux=5, seed=8, nstates=2, s=0.6)
    nc, na, nv = 2, 2, 3
    nh = nc + na
    B = prob.B
    I4 = np.zeros((nh, na + nv, nh, na + nv))
    for i, a, j, b in itertools.product(range(nh), range(na + nv), range(nh), range(na + nv)):
        I4[i, a, j, b] = sum(B[q, i, a] * B[q, j, b] for q in range(B.shape[0]))
    g1h = np.zeros((nh, nh))
    g1h[:nc, :nc] = 2 * np.eye(nc)
    g1h[nc:, nc:] = prob.gamma1
    lam = np.zeros((nh,) * 4)
    lam[nc:, nc:, nc:, nc:] = prob.lambda2
    eps = prob.eps
    ep = eps[nc:]
    e = 0.0
    for k, l, i, j in itertools.product(range(nh), repeat=4):
        g2 = lam[k, l, i, j] + g1h[k, i] * g1h[l, j] - 0.5 * g1h[l, i] * g1h[k, j]
        if g2 == 0.0:
            continue
        for a, b in itertools.product(range(na, na + nv), repeat=2):
            dij = eps[i] + eps[j] - ep[a] - ep[b]
            dkl = eps[k] + eps[l] - ep[a] - ep[b]
            rij = (1 - np.exp(-prob.s * dij * dij)) / dij
            rkl = (1 - np.exp(-prob.s * dkl * dkl)) / dkl
            tij = I4[i, a, j, b] * rij
            tkl = I4[k, a, l, b] * rkl
            e += 0.5 * g2 * tij * (2 * I4[k, a, l, b] - dij * tkl)
    assert abs(O.e_vv(prob) - e) <= 1e-13 * abs(e)


# ----------------------------------------------------- Fock-space brute force
def _full_t2(prob, ts):
    nc, na, nv = prob.ncore, prob.nact, prob.nvir
    nh, npart = nc + na, na + nv
    t2 = np.zeros((nh, nh, npart, npart))
    for i in range(nh):
        for j in range(nh):
            t2[i, j, na:, na:] = O.t2_vv(prob, i, j)[0]
            if na:
                t2[i, j, na:, :na] = ts[i, j]
                t2[i, j, :na, na:] = ts[j, i].T
    return t2


@pytest.mark.parametrize("nel_act,weights,seed", [(2, (0.6, 0.4), 7), (4, (0.3, 0.7), 3),
                                                   (4, (0.2, 0.3, 0.5), 17)])
def test_fock_space_dvv_energy_and_t1(nel_act, weights, seed):
    """Eq. A12 terms 1-12 (+ the Lambda3 term 13, formed here from the CI),
    E_vv, and the one-body part of [H0, T2] in Eq. A6, all against explicit
    determinant-space evaluation with spin-adapted (singlet) ensembles."""
    nc, na, nv = 2, 3, 2
    sysm = TinySystem(nc, na, nv, nel_act=nel_act, nstates=len(weights), seed=seed, weights=weights)
    prob = make_problem(nc, na, nv, 6, seed=11 + seed, nstates=1, s=0.7)
    prob.gamma1, prob.lambda2 = sysm.gamma1, sysm.lambda2
    nh, npart = nc + na, na + nv
    ts = O.t2_semi_internal(prob)
    t1 = O.t1_amplitudes(prob, ts)
    t2 = _full_t2(prob, ts)
    t1f = np.zeros((nh, npart))
    t1f[:, na:] = t1
    T = sysm.cluster(t1f, t2)
    brute = sysm.dvv(T - T.T)
    lam3 = O.sa_lambda3(sysm.gamma1, sysm.lambda2, sysm.gamma3)
    terms = O.dvv_terms(prob, ts=ts, t1=t1, lambda3=lam3)
    assert set(terms) == set(range(1, 14))
    d = sum(terms.values())
    scale = np.max(np.abs(brute))
    assert np.max(np.abs(d - brute)) <= 1e-12 * scale
    # each amplitude class separately (no cross-class contraction survives)
    t2vv = np.zeros_like(t2)
    t2vv[:, :, na:, na:] = t2[:, :, na:, na:]
    Tv = sysm.cluster(None, t2vv)
    assert np.allclose(sysm.dvv(Tv - Tv.T), terms[4] + terms[5] + terms[7], rtol=0, atol=1e-12 * scale)
    # term 13 is what the brute force adds beyond terms 1-12
    assert np.max(np.abs(terms[13])) > 1e-6 * scale
    assert np.max(np.abs(d - terms[13] - brute)) > 1e-6 * scale
    # E_vv
    nu_vv = np.zeros((nh, nh, nv, nv))
    for k in range(nh):
        for l in range(nh):
            nu_vv[k, l] = O.nu_pair(prob, k, l, slice(na, None), slice(na, None))
    H0 = sysm.h0(prob.eps)
    eb = sysm.energy(sysm.v_vv(nu_vv), H0, Tv - Tv.T)
    assert abs(O.e_vv(prob) - eb) <= 1e-12 * abs(eb)
    # Eq. A6: one-body part of [H0, T2] for core -> virtual
    T2 = sysm.cluster(None, t2)
    X = H0 @ T2 - T2 @ H0
    base = nc + na
    eh, ep = O.hole_eps(prob), O.particle_eps(prob)
    R = O.regularizer(eh[:nc, None] - ep[na:][None, :], prob.s)
    ref = t1[:nc] / R
    for m in range(nc):
        for e in range(nv):
            op = sysm.fs.e1(so(m, 0), so(base + e, 0))
            y = sysm.expect(lambda psi: op @ (X @ psi))
            assert abs(y - ref[m, e]) <= 1e-12 * np.max(np.abs(ref))


@pytest.mark.parametrize("nel_act,weights,seed", [(2, (0.6, 0.4), 7), (4, (0.3, 0.7), 3), (2, (0.5, 0.5), 13)])
def test_fock_space_t1_active_holes(nel_act, weights, seed):
    """Eq. A6 for active holes u: t^u_e / R(Delta^u_e) is the one-body part of
    [H0, T2].  Brute force: X = [H0, T2] as a determinant-space matrix; its
    two-body part is sum Delta^{ij}_{ab} t^{ij}_{ab} {a^{ab}_{ij}} (H0 is
    diagonal), built with the same normal ordering and subtracted; what is left
    is a normal-ordered one-body operator plus a constant, whose ensemble
    projection <a+_v a_e (.)> equals sum_w X1[w][e] gamma[v][w] (e is empty),
    so X1 follows from a linear solve with the active 1-RDM."""
    nc, na, nv = 2, 3, 2
    sysm = TinySystem(nc, na, nv, nel_act=nel_act, nstates=2, seed=seed, weights=weights)
    prob = make_problem(nc, na, nv, 6, seed=21 + seed, nstates=1, s=0.6)
    prob.gamma1, prob.lambda2 = sysm.gamma1, sysm.lambda2
    ts = O.t2_semi_internal(prob)
    t1 = O.t1_amplitudes(prob, ts)
    t2 = _full_t2(prob, ts)
    eh, ep = O.hole_eps(prob), O.particle_eps(prob)
    delta = (ep[None, None, :, None] + ep[None, None, None, :]
             - eh[:, None, None, None] - eh[None, :, None, None])
    T2 = sysm.cluster(None, t2)
    H0 = sysm.h0(prob.eps)
    R = (H0 @ T2 - T2 @ H0) - sysm.cluster(None, delta * t2)
    base = nc + na
    y = np.zeros((na, nv))
    for v in range(na):
        for e in range(nv):
            op = sysm.fs.e1(so(nc + v, 0), so(base + e, 0))
            y[v, e] = sysm.expect(lambda psi: op @ (R @ psi))
    act_a = [so(nc + u, 0) for u in range(na)]
    g_aa = sysm.g1so[np.ix_(act_a, act_a)]
    x1 = np.linalg.solve(g_aa, y)
    ref = t1[nc:] / O.regularizer(eh[nc:, None] - ep[na:][None, :], prob.s)
    assert np.max(np.abs(ref)) > 1e-4
    assert np.max(np.abs(x1 - ref)) <= 1e-11 * np.max(np.abs(ref))


def test_fock_space_sr_number_conservation():
    """Single reference: the trace of the core block of Gamma^(2) (brute force)
    cancels the trace of the oracle's D_vv; the vv block is PSD."""
    nc, na, nv = 2, 0, 3
    sysm = TinySystem(nc, 1, nv, nel_act=0, nstates=1, seed=1)
    prob = make_problem(nc, 1, nv, 7, seed=2, nstates=1, s=0.9)
    # no active electrons: the single active orbital is empty; drop its amplitudes
    prob.gamma1 = np.zeros((1, 1))
    prob.lambda2 = np.zeros((1, 1, 1, 1))
    nh, npart = nc + 1, 1 + nv
    t2 = np.zeros((nh, nh, npart, npart))
    for m in range(nc):
        for n in range(nc):
            t2[m, n, 1:, 1:] = O.t2_vv(prob, m, n)[0]
    T = sysm.cluster(None, t2)
    A = T - T.T
    occ = 0.0
    for m in range(nc):
        E = sum(sysm.fs.e1(so(m, s), so(m, s)) for s in (0, 1))
        occ += 0.5 * sysm.expect(lambda psi: E @ (A @ (A @ psi)) - 2 * (A @ (E @ (A @ psi)))
                                  + A @ (A @ (E @ psi)))
    d = O.dvv_terms(prob, terms=(4,))[4]
    assert abs(np.trace(d) + occ) <= 1e-12 * abs(occ)
    assert np.min(np.linalg.eigvalsh(0.5 * (d + d.T))) > -1e-15


# ---------------------------------------------------------- structural pins
def test_vv_terms_match_hole_rdm_form():
    """Terms 4 + 5 + 7 equal 1/2 sum Gamma2_H[k][l][i][j] (tau^{kl} tau^{ij T}
    + tau^{kl T} tau^{ij}), the form the vv block takes when the particle
    pair is virtual (derived like E_vv)."""
    prob = make_problem(ncore=3, nact=3, nvir=7, naux=11, seed=4, nstates=3, s=0.5)
    terms = O.dvv_terms(prob, terms=(4, 5, 7))
    g2h = O.gamma2_holes(prob)
    nh = 6
    tau = {(i, j): O.t2_vv(prob, i, j)[0] for i in range(nh) for j in range(nh)}
    d = np.zeros((7, 7))
    for k, l, i, j in itertools.product(range(nh), repeat=4):
        w = g2h[k, l, i, j]
        if w:
            d += 0.5 * w * (tau[(k, l)] @ tau[(i, j)].T + tau[(k, l)].T @ tau[(i, j)])
    ref = terms[4] + terms[5] + terms[7]
    assert np.max(np.abs(d - ref)) <= 1e-13 * np.max(np.abs(ref))


def test_sr_term4_symmetric_output_form():
    """Single reference: term 4 of Eq. A12 equals
    2 [sum_{m<n} (1/2 P + 3/2 M) + sum_m A_m A_m^T] with A = t^{mn} as an
    (e, e') matrix, P = (A + A^T)(A + A^T)^T and M = (A - A^T)(A - A^T)^T, the
    symmetric (A + A^T) / (A - A^T) split the core-pair dressing uses; hence
    D_vv is positive semidefinite."""
    prob = make_problem(ncore=4, nact=0, nvir=9, naux=13, seed=23, s=0.5)
    t4 = O.dvv_terms(prob, terms=(4,))[4]
    ref = np.zeros((9, 9))
    for m in range(4):
        for n in range(m, 4):
            A = O.t2_vv(prob, m, n)[0]
            if m == n:
                ref += 2.0 * A @ A.T
            else:
                P = (A + A.T) @ (A + A.T).T
                M = (A - A.T) @ (A - A.T).T
                ref += 2.0 * (0.5 * P + 1.5 * M)
    assert np.max(np.abs(t4 - ref)) <= 1e-13 * np.max(np.abs(ref))
    assert np.linalg.eigvalsh(0.5 * (t4 + t4.T)).min() >= -1e-14 * np.max(np.abs(t4))


def test_dvv_symmetric_and_invariant_under_aux_rotation():
    prob = make_problem(ncore=3, nact=2, nvir=6, naux=9, seed=12, nstates=2, s=0.5)
    d, asym = O.dvv(prob, return_asym=True)
    assert asym <= 1e-12 * np.linalg.norm(d)
    q, _ = np.linalg.qr(np.random.default_rng(0).standard_normal((9, 9)))
    p2 = make_problem(ncore=3, nact=2, nvir=6, naux=9, seed=12, nstates=2, s=0.5)
    p2.B = np.einsum("PQ,Qhp->Php", q, prob.B)
    assert abs(O.e_vv(p2) - O.e_vv(prob)) <= 1e-12 * abs(O.e_vv(prob))
    assert np.max(np.abs(O.dvv(p2) - d)) <= 1e-12 * np.max(np.abs(d))


def test_dvv_covariant_under_virtual_permutation_and_sign():
    prob = make_problem(ncore=2, nact=2, nvir=5, naux=8, seed=13, nstates=2, s=0.5)
    d = O.dvv(prob)
    perm = np.array([3, 0, 4, 1, 2])
    sign = np.array([1, -1, 1, 1, -1.0])
    p2 = make_problem(ncore=2, nact=2, nvir=5, naux=8, seed=13, nstates=2, s=0.5)
    na = 2
    p2.B = prob.B.copy()
    p2.B[:, :, na:] = prob.B[:, :, na:][:, :, perm] * sign[None, None, :]
    p2.eps = prob.eps.copy()
    p2.eps[4:] = prob.eps[4:][perm]
    d2 = O.dvv(p2)
    ref = d[np.ix_(perm, perm)] * np.outer(sign, sign)
    assert np.max(np.abs(d2 - ref)) <= 1e-13 * np.max(np.abs(d))
    assert abs(np.trace(d2) - np.trace(d)) <= 1e-13 * abs(np.trace(d))


def test_dvv_rotation_inside_degenerate_block():
    """Two virtuals with equal energies: rotating them rotates D_vv."""
    prob = make_problem(ncore=2, nact=0, nvir=4, naux=7, seed=14, s=0.5)
    prob.eps[3] = prob.eps[2]
    d = O.dvv(prob)
    th = 0.37
    U = np.eye(4)
    U[0:2, 0:2] = [[np.cos(th), -np.sin(th)], [np.sin(th), np.cos(th)]]
    p2 = make_problem(ncore=2, nact=0, nvir=4, naux=7, seed=14, s=0.5)
    p2.eps = prob.eps.copy()
    p2.B = np.einsum("Qhe,ef->Qhf", prob.B, U)
    assert np.max(np.abs(O.dvv(p2) - U.T @ d @ U)) <= 1e-13 * np.max(np.abs(d))


# ------------------------------------------------------------ eigen / truncate
def test_natural_orbitals_against_lapack():
    prob = make_problem(ncore=3, nact=2, nvir=12, naux=20, seed=15, nstates=2, s=0.5)
    d = O.dvv(prob)
    n, v = O.natural_orbitals(d)
    assert np.all(np.diff(n) <= 0)
    assert np.linalg.norm(d @ v - v * n) <= 1e-12 * np.linalg.norm(d)
    assert np.linalg.norm(v.T @ v - np.eye(12)) <= 1e-13
    ref = np.sort(np.linalg.eigvals(d).real)[::-1]
    assert np.max(np.abs(ref - n)) <= 1e-14 * np.max(np.abs(n)) * 10


@pytest.mark.parametrize("ons,mode,thr,expect", [
    ([4.0, 3.0, 2.0, 1.0], 0, 70.0, 2),         # cum 0.7 reached exactly at k = 2
    ([4.0, 3.0, 2.0, 1.0], 0, 70.0001, 3),
    ([4.0, 3.0, 2.0, 1.0], 0, 100.0, 4),
    ([4.0, 3.0, 2.0, 1.0], 0, 0.0, 1),
    ([4.0, 3.0, 2.0, 1.0], 1, 50.0, 2),
    ([4.0, 3.0, 2.0, 1.0], 1, 51.0, 3),
    ([4.0, 3.0, 2.0, 1.0], 2, 2.0, 3),
    ([4.0, 3.0, 2.0, 1.0], 2, 5.0, 0),
    ([1.0, 0.995, 0.9852, 0.5], 0, 30.0, 3),    # widening chain 1 -> 2 -> 3
    ([1.0, 0.99, 0.5, 0.49], 0, 30.0, 1),       # 0.01 difference is not < 0.01
    ([1.0, 0.5, 0.496, -1e-6], 0, 85.0, 3),     # negative ON in the denominator
    ([4.0, 3.0, 2.0, 1.0], 3, 2.0, 2),          # fixed N'
    ([4.0, 3.0, 2.0, 1.0], 3, 2.6, 3),          # rounded
    ([4.0, 3.0, 2.0, 1.0], 3, 9.0, 4),          # clamped to N_V
    ([4.0, 3.0, 2.0, 1.0], 3, -1.0, 0),
    ([1.0, 0.995, 0.9852, 0.5], 3, 1.0, 3),     # widening still applies
])
def test_truncation_rules(ons, mode, thr, expect):
    assert O.truncate(np.array(ons), mode, thr, 0.01) == expect


def test_correction_limits():
    prob = make_problem(ncore=3, nact=2, nvir=10, naux=14, seed=16, nstates=2, s=0.5)
    d = O.dvv(prob)
    n, v = O.natural_orbitals(d)
    e = O.e_vv(prob)
    de, efno, _ = O.discarded_correction(prob, v, 10, e)
    assert abs(de) <= 1e-12 * abs(e)
    de0, _, _ = O.discarded_correction(prob, v, 0, e)
    assert de0 == e
    de5, efno5, eps5 = O.discarded_correction(prob, v, 5, e)
    assert np.all(np.diff(eps5) >= 0)
    assert abs(efno5) < abs(e)


def test_correction_is_basis_free_inside_the_kept_space():
    """Recanonicalisation (Sec. 2) makes E_vv(FNO) a function of the kept
    space alone: any orthonormal basis of it gives the same energy and the
    same recanonicalised orbital energies."""
    prob = make_problem(ncore=3, nact=2, nvir=12, naux=15, seed=18, nstates=2, s=0.5)
    n, v = O.natural_orbitals(O.dvv(prob))
    k = 6
    de, efno, eps = O.discarded_correction(prob, v, k)
    q, _ = np.linalg.qr(np.random.default_rng(3).standard_normal((k, k)))
    v2 = v.copy()
    v2[:, :k] = v[:, :k] @ q
    de2, efno2, eps2 = O.discarded_correction(prob, v2, k)
    assert abs(efno2 - efno) <= 1e-12 * abs(efno)
    assert np.max(np.abs(eps2 - eps)) <= 1e-13


def test_correction_on_a_subset_of_canonical_virtuals():
    """Kept space = a subset S of the semicanonical virtuals: E_vv(FNO) is
    E_vv of the problem whose virtual space is S, built by slicing B and eps."""
    prob = make_problem(ncore=3, nact=2, nvir=12, naux=15, seed=19, nstates=2, s=0.5)
    S = [7, 2, 10, 4, 0]
    no = np.zeros((12, 12))
    for c, e in enumerate(S):
        no[e, c] = 1.0
    _, efno, eps = O.discarded_correction(prob, no, len(S))
    from copy import copy
    sub = copy(prob)
    keep = sorted(S)
    na = prob.nact
    sub.B = np.ascontiguousarray(np.concatenate([prob.B[:, :, :na], prob.B[:, :, [na + e for e in keep]]], axis=2))
    sub.nvir = len(keep)
    nh = prob.ncore + prob.nact
    sub.eps = np.concatenate([prob.eps[:nh], prob.eps[nh:][keep]])
    assert np.allclose(eps, prob.eps[nh:][keep], rtol=0, atol=1e-15)
    assert abs(efno - O.e_vv(sub)) <= 1e-12 * abs(efno)


# ------------------------------------------------------------- generator RDMs
def test_generator_rdms_against_fock_space():
    """synth.ci spin-free RDMs of a random CI vector agree with the
    determinant-space helper's spin-orbital RDMs summed over spin."""
    from synth import ci
    from fockspace import FockSpace, gamma1_spin_orbital, rdm_spin_orbital
    rng = np.random.default_rng(3)
    norb = 4
    vecs, sa, ta, tb = ci.random_ci_vectors(rng, norb, 1)
    g1, g2 = ci.spin_free_rdms(vecs[0], norb, ta, tb)
    fs = FockSpace(norb, norb)
    psi = np.zeros(fs.dim)
    for ia, a in enumerate(sa):
        for ib, b in enumerate(sa):
            d = 0
            for p in range(norb):
                if (int(a) >> p) & 1:
                    d |= 1 << so(p, 0)
                if (int(b) >> p) & 1:
                    d |= 1 << so(p, 1)
            # determinant order: alpha creators first, then beta; the Fock
            # space orders creators by spin orbital index (interleaved).
            occ_a = [so(p, 0) for p in range(norb) if (int(a) >> p) & 1]
            occ_b = [so(p, 1) for p in range(norb) if (int(b) >> p) & 1]
            seq = occ_a + occ_b
            inv = sum(1 for x in range(len(seq)) for y in range(x + 1, len(seq)) if seq[x] > seq[y])
            psi[fs.index[d]] = vecs[0][ia, ib] * (-1) ** inv
    w = [1.0]
    so_all = list(range(2 * norb))
    G1 = gamma1_spin_orbital(fs, [psi], w)
    G2 = rdm_spin_orbital(fs, [psi], w, so_all, 2)
    g1_ref = G1[0::2, 0::2] + G1[1::2, 1::2]
    g2_ref = np.einsum("uavbxayb->uvxy", G2.reshape((norb, 2) * 4))
    assert np.max(np.abs(g1 - g1_ref)) < 1e-13
    assert np.max(np.abs(g2 - g2_ref)) < 1e-13
    assert abs(np.trace(g1) - norb) < 1e-13
    assert abs(np.einsum("pqpq->", g2) - norb * (norb - 1)) < 1e-12


# ------------------------------------------------------------ 3-body cumulant
@pytest.mark.parametrize("nel_act,seed", [(2, 7), (4, 3), (4, 9)])
def test_sa_lambda3_is_the_spin_summed_cumulant(nel_act, seed):
    """The spin-free 3-cumulant formula equals the spin-orbital cumulant
    (determinant-space 3-RDM minus its antisymmetrised products) summed over
    the spins of the pairs, for spin-adapted (singlet) ensembles."""
    sysm = TinySystem(1, 3, 1, nel_act=nel_act, nstates=2, seed=seed, weights=(0.35, 0.65))
    lam3 = O.sa_lambda3(sysm.gamma1, sysm.lambda2, sysm.gamma3)
    assert np.max(np.abs(sysm.lambda3)) > 1e-3
    assert np.max(np.abs(lam3 - sysm.lambda3)) <= 1e-13


def _brute_spin_free_rdm3(C, norb, sa):
    """Spin-free 3-RDM of a CI matrix C[alpha string][beta string] by
    explicit creation/annihilation on determinants (alpha spin orbitals
    0..norb-1, beta norb..2norb-1, creators in ascending order)."""
    from fockspace import FockSpace, rdm_spin_orbital
    nel = 2 * bin(int(sa[0])).count("1")
    fs = FockSpace(norb, nel)
    psi = np.zeros(fs.dim)
    for ia, a in enumerate(sa):
        for ib, b in enumerate(sa):
            psi[fs.index[int(a) | (int(b) << norb)]] = C[ia, ib]
    g3 = rdm_spin_orbital(fs, [psi], [1.0], list(range(2 * norb)), 3)
    g3 = g3.reshape((2, norb) * 6)
    return np.einsum("axbycz aubvcw->xyzuvw".replace(" ", ""), g3)


def test_generator_gamma3_against_determinant_brute_force():
    """The input generator's spin-free 3-RDM (E-operator products) equals the
    determinant-space brute force for random (not spin-adapted) CI vectors."""
    from synth import ci
    rng = np.random.default_rng(12)
    vecs, sa, ta, tb = ci.random_ci_vectors(rng, 4, 2)
    for c in vecs:
        _, g2 = ci.spin_free_rdms(c, 4, ta, tb)
        got = ci.spin_free_rdm3(c, 4, ta, tb, g2)
        ref = _brute_spin_free_rdm3(c, 4, sa)
        assert np.max(np.abs(ref)) > 0.1
        assert np.max(np.abs(got - ref)) <= 1e-13


def test_sa_lambda3_vanishes_for_a_closed_shell_determinant():
    """A closed-shell determinant has no cumulants: Lambda2 = Lambda3 = 0."""
    from synth import ci
    norb = 4
    sa = ci.strings(norb, 2)
    ta = ci.excitation_table(sa, norb)
    k = 3
    C = np.zeros((len(sa), len(sa)))
    C[k, k] = 1.0
    g1, g2 = ci.spin_free_rdms(C, norb, ta, ta)
    lam2 = g2 - np.einsum("pr,qs->pqrs", g1, g1) + 0.5 * np.einsum("ps,qr->pqrs", g1, g1)
    g3 = ci.spin_free_rdm3(C, norb, ta, ta, g2)
    assert np.max(np.abs(g3)) > 1.0
    assert np.max(np.abs(lam2)) <= 1e-14
    assert np.max(np.abs(O.sa_lambda3(g1, lam2, g3))) <= 1e-13


def test_sa_lambda3_symmetries_and_partial_trace():
    """Lambda3 of a random ensemble keeps the pair-permutation and
    upper/lower symmetries of Gamma3; the generator's Gamma3 obeys the
    particle-number sum rule sum_w Gamma3[x][y][w][u][v][w] = (N - 2) Gamma2."""
    from synth import ci
    rng = np.random.default_rng(4)
    n = 4
    vecs, _, ta, tb = ci.random_ci_vectors(rng, n, 3)
    w = np.array([0.2, 0.3, 0.5])
    g1, g2, lam2 = ci.state_averaged_densities(vecs, w, n, ta, tb)
    g3 = np.einsum("a,a...->...", w, ci.state_gamma3(vecs, n, ta, tb))
    assert np.max(np.abs(np.einsum("xywuvw->xyuv", g3) - (n - 2) * g2)) <= 1e-12
    lam3 = O.sa_lambda3(g1, lam2, g3)
    for perm in itertools.permutations(range(3)):
        up = "xyz"
        lo = "uvw"
        spec = "".join(up[i] for i in perm) + "".join(lo[i] for i in perm)
        assert np.max(np.abs(np.einsum(f"{spec}->xyzuvw", lam3) - lam3)) <= 1e-13
    assert np.max(np.abs(np.einsum("xyzuvw->uvwxyz", lam3) - lam3)) <= 1e-13


def test_sampling_restrictions_partition_terms_4_5_7():
    """The restrictions of terms 4, 5 and 7 to listed core pairs, (m, u) and
    (u, v) are partial sums: over a partition of the index set they add up to
    the whole term, and the empty list gives zero."""
    p = make_problem(ncore=3, nact=3, nvir=11, naux=23, seed=71, nstates=2)
    nc, na = p.ncore, p.nact
    full = O.dvv_terms(p, terms=(4, 5, 7))
    cp = [(m, n) for m in range(nc) for n in range(m, nc)]
    ca = [(m, u) for m in range(nc) for u in range(na)]
    aa = [(u, v) for u in range(na) for v in range(na)]
    for term, key, idx in ((4, "core_pairs", cp), (5, "ca_pairs", ca), (7, "aa_pairs", aa)):
        halves = [idx[0::2], idx[1::2]]
        parts = [O.dvv_terms(p, terms=(term,), **{key: h})[term] for h in halves]
        ref = full[term]
        assert np.max(np.abs(parts[0] + parts[1] - ref)) <= 1e-13 * np.max(np.abs(ref))
        assert np.max(np.abs(O.dvv_terms(p, terms=(term,), **{key: []})[term])) == 0.0


# ------------------------------------------------- natural auxiliary functions
def test_naf_spectrum_is_the_squared_singular_values():
    """W = B B^T over the hole-particle pairs: its eigenvalues are the squared
    singular values of B as a naux x (nh np) matrix (LAPACK SVD)."""
    p = make_problem(ncore=3, nact=2, nvir=13, naux=31, seed=81, nstates=2)
    _, w, U = O.naf(p, -1.0)
    sv = np.linalg.svd(p.B.reshape(p.naux, -1), compute_uv=False)
    assert np.allclose(w, sv ** 2, rtol=1e-12, atol=1e-14 * sv[0] ** 2)
    assert np.allclose(U.T @ U, np.eye(p.naux), atol=1e-13)


def test_naf_keeping_every_function_changes_nothing():
    """With every function kept, B' is an orthogonal rotation of the
    auxiliary index, under which nu = B^T B, hence E_vv and D_vv, are exact
    invariants."""
    p = make_problem(ncore=3, nact=2, nvir=13, naux=31, seed=82, nstates=2)
    q = O.naf_problem(p, -1.0)
    assert q.naux == p.naux
    assert abs(O.e_vv(q) - O.e_vv(p)) <= 1e-12 * abs(O.e_vv(p))
    d0, d1 = O.dvv(p), O.dvv(q)
    assert np.max(np.abs(d1 - d0)) <= 1e-12 * np.max(np.abs(d0))


def test_naf_discarded_weight_and_integral_error():
    """Truncation to the functions with w > threshold: the projected-out part
    of the factors has squared norm sum_{discarded} w (the eigen-decomposition
    written as a sum of squares), and every integral nu^{ij}_{ab} changes by at
    most |B_ia - P B_ia| |B_jb - P B_jb| (Cauchy-Schwarz)."""
    p = make_problem(ncore=3, nact=2, nvir=13, naux=31, seed=83, nstates=2)
    _, w, U = O.naf(p, -1.0)
    thr = w[20]
    Bp, _, _ = O.naf(p, thr)
    k = Bp.shape[0]
    assert k == 20
    B2 = p.B.reshape(p.naux, -1)
    P = U[:, :k] @ U[:, :k].T
    R = B2 - P @ B2
    assert abs(np.sum(R * R) - np.sum(w[k:])) <= 1e-10 * np.sum(w)
    nu = B2.T @ B2
    nup = Bp.reshape(k, -1).T @ Bp.reshape(k, -1)
    rn = np.sqrt(np.sum(R * R, axis=0))
    assert np.all(np.abs(nu - nup) <= np.outer(rn, rn) * (1 + 1e-9) + 1e-14)


# ------------------------------------------------ particle-particle ladder
def test_ladder_against_explicit_loops():
    rng = np.random.default_rng(95)
    nq, nv, npairs = 4, 5, 3
    Bv = rng.standard_normal((nq, nv, nv))
    T = rng.standard_normal((npairs, nv, nv))
    C = O.ladder(Bv, T)
    ref = np.zeros_like(C)
    for p_ in range(npairs):
        for a in range(nv):
            for b in range(nv):
                s = 0.0
                for c in range(nv):
                    for d in range(nv):
                        v = sum(Bv[q, a, c] * Bv[q, b, d] for q in range(nq))
                        s += v * T[p_, c, d]
                ref[p_, a, b] = s
    assert np.max(np.abs(C - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_ladder_is_covariant_under_virtual_rotation():
    """Rotating the virtual basis (B'^Q = U^T B^Q U, T' = U^T T U for every
    pair) rotates the result the same way, C' = U^T C U."""
    rng = np.random.default_rng(96)
    nq, nv, npairs = 7, 9, 4
    Bv = rng.standard_normal((nq, nv, nv))
    Bv = Bv + Bv.transpose(0, 2, 1)
    T = rng.standard_normal((npairs, nv, nv))
    U, _ = np.linalg.qr(rng.standard_normal((nv, nv)))
    C = O.ladder(Bv, T)
    C2 = O.ladder(np.einsum("ea,Qef,fb->Qab", U, Bv, U), np.einsum("ca,pcd,db->pab", U, T, U))
    assert np.max(np.abs(C2 - np.einsum("ea,pef,fb->pab", U, C, U))) <= 1e-12 * np.max(np.abs(C))


def test_ladder_pair_transpose_symmetry():
    """With symmetric factors (B^Q_{ac} = B^Q_{ca}) the integrals satisfy
    <ab|cd> = <ba|dc>, so T^{ji} = (T^{ij})^T gives C^{ji} = (C^{ij})^T."""
    rng = np.random.default_rng(97)
    nq, nv = 6, 8
    Bv = rng.standard_normal((nq, nv, nv))
    Bv = Bv + Bv.transpose(0, 2, 1)
    t = rng.standard_normal((nv, nv))
    C = O.ladder(Bv, np.stack([t, t.T]))
    assert np.max(np.abs(C[1] - C[0].T)) <= 1e-12 * np.max(np.abs(C))


# ---------------------------------------------------------------------------
# Full multi-reference PT2 energy (Eq. A4's H-bar to second order)
# ---------------------------------------------------------------------------
def _tiny_full_problem(nc, na, nv, sysm, use_f, seed):
    """A problem whose integrals come from a DF factor over ALL orbitals, with
    an off-diagonal Fock matrix (zero in the core, active and virtual diagonal
    blocks, which make H0 = diag(eps)); returns (prob, eri, f) for the brute
    force, which uses every block of the Hamiltonian."""
    norb, nh = nc + na + nv, nc + na
    rng = np.random.default_rng(seed)
    naux = 6
    Bf = rng.standard_normal((naux, norb, norb)) * 0.3
    Bf = Bf + Bf.transpose(0, 2, 1)
    eps = np.concatenate([np.sort(rng.uniform(-2, -0.3, nc)), np.sort(rng.uniform(-0.5, 0.3, na)),
                          np.sort(rng.uniform(0.1, 2.0, nv))])
    f = np.zeros((norb, norb))
    if use_f:
        f = rng.standard_normal((norb, norb)) * 0.1
        f = f + f.T
        for b in (slice(0, nc), slice(nc, nh), slice(nh, norb)):
            f[b, b] = 0.0
    prob = make_problem(nc, na, nv, naux, seed=5, nstates=1, s=0.7)
    prob.B = np.ascontiguousarray(Bf[:, :nh, nc:])
    prob.eps = eps
    prob.gamma1, prob.lambda2 = sysm.gamma1, sysm.lambda2
    prob.f_hp = f[:nh, nc:].copy() if use_f else None
    eri = np.einsum("Qpr,Qqs->pqrs", Bf, Bf)     # <pq|rs> = (pr|qs)
    return prob, eri, f


@pytest.mark.parametrize("nc,na,nv,nel_act,use_f,seed", [(1, 3, 1, 2, False, 3), (1, 3, 1, 4, True, 4),
                                                         (2, 2, 2, 2, True, 5)])
def test_fock_space_full_pt2_energy(nc, na, nv, nel_act, use_f, seed):
    """E^(2) = <[H, A]> + 1/2 <[[H0, A], A]> with the Hamiltonian's every block
    (all 4-index integrals over all orbitals, the off-diagonal Fock matrix),
    A = T - T^+ from Eqs. A6, A7 over every amplitude class, evaluated with
    determinant-space matrices over singlet ensembles; the oracle's closed form
    (Lambda3 from the CI vectors) must agree to rounding, and without Lambda3
    it must differ (the 3-cumulant terms are not empty)."""
    sysm = TinySystem(nc, na, nv, nel_act=nel_act, nstates=2, seed=seed, weights=(0.3, 0.7))
    prob, eri, f = _tiny_full_problem(nc, na, nv, sysm, use_f, seed)
    T2, _, _ = O.t2_general(prob)
    T1, _, _, _ = O.t1_general(prob, T2)
    T = sysm.cluster(T1, T2)
    brute = sysm.energy(sysm.hamiltonian(eri, f), sysm.h0(prob.eps), T - T.T)
    e = O.pt2_energy(prob, sysm.lambda3)
    assert abs(e - brute) <= 1e-13 * abs(brute), (e, brute)
    assert abs(O.pt2_energy(prob) - brute) > 1e-4 * abs(brute)


def test_fock_space_commutator_scalar_random_operators():
    """<[X, T]> of random normal-ordered de-excitation X and excitation T
    (one- and two-body, pair-symmetric) against determinant space: the
    generalised-Wick closed form holds for any operators, not only the PT2
    amplitudes."""
    nc, na, nv = 1, 3, 1
    sysm = TinySystem(nc, na, nv, nel_act=2, nstates=2, seed=8, weights=(0.45, 0.55))
    prob = make_problem(nc, na, nv, 4, seed=2, nstates=1)
    prob.gamma1, prob.lambda2 = sysm.gamma1, sysm.lambda2
    nh, npart = nc + na, na + nv
    rng = np.random.default_rng(12)
    X2 = rng.standard_normal((nh, nh, npart, npart))
    X2 = X2 + X2.transpose(1, 0, 3, 2)
    T2 = rng.standard_normal((nh, nh, npart, npart))
    T2 = T2 + T2.transpose(1, 0, 3, 2)
    T2[nc:, nc:, :na, :na] = 0.0
    X1 = rng.standard_normal((nh, npart))
    T1 = rng.standard_normal((nh, npart))
    T1[nc:, :na] = 0.0
    Xo = sysm.cluster(X1, X2).T          # E^{ij}_{ab} = (E^{ab}_{ij})^+
    To = sysm.cluster(T1, T2)
    brute = sysm.expect(lambda psi: Xo @ (To @ psi) - To @ (Xo @ psi))
    e = O.commutator_scalar(prob, X1, X2, T1, T2, sysm.lambda3)
    assert abs(e - brute) <= 1e-12 * max(1.0, abs(brute)), (e, brute)


def test_full_pt2_energy_vv_part_is_e_vv():
    """Restricted to the doubles whose particles are both virtual, the
    closed form of <[X, T]> reproduces E_vv (a separate derivation through
    the hole 2-RDM) on a CAS(6,6) problem."""
    p = make_problem(3, 6, 12, 30, seed=6, nstates=3)
    na = p.nact
    T2, nu, d = O.t2_general(p)
    keep = np.zeros_like(T2, dtype=bool)
    keep[:, :, na:, na:] = True
    T2v = np.where(keep, T2, 0.0)
    X2v = np.where(keep, nu - 0.5 * d * T2, 0.0)
    z = np.zeros((p.nh, p.np_))
    e = 2.0 * O.commutator_scalar(p, z, X2v, z, T2v)
    ref = O.e_vv(p)
    assert abs(e - ref) <= 1e-12 * abs(ref)


def test_full_pt2_energy_single_reference_is_mp2():
    """No active orbitals, large s: E^(2) is the closed-shell MP2 energy
    including the singles of an off-diagonal Fock matrix,
    sum (ia|jb)[2(ia|jb) - (ib|ja)]/Delta + 2 sum |f_ia|^2/Delta_i^a."""
    p = make_problem(5, 0, 20, 40, seed=9, nstates=1, s=1.0e3)
    rng = np.random.default_rng(4)
    p.f_hp = 0.05 * rng.standard_normal((p.nh, p.np_))
    nu = np.einsum("Qia,Qjb->ijab", p.B, p.B)
    eh, ep = O.hole_eps(p), O.particle_eps(p)
    d = eh[:, None, None, None] + eh[None, :, None, None] - ep[None, None, :, None] - ep[None, None, None, :]
    mp2 = np.sum(nu * (2.0 * nu - nu.transpose(0, 1, 3, 2)) / d)
    mp2 += 2.0 * np.sum(p.f_hp ** 2 / (eh[:, None] - ep[None, :]))
    e = O.pt2_energy(p)
    assert abs(e - mp2) <= 1e-12 * abs(mp2), (e, mp2)


def test_full_correction_limits():
    """Eq. 11 with the full energy: keeping every NO gives 0; keeping none
    leaves the problem with active particles only, whose energy is that of
    the same problem sliced to no virtuals (a separate construction)."""
    p = make_problem(3, 4, 14, 30, seed=12, nstates=2)
    rng = np.random.default_rng(2)
    p.f_hp = 0.05 * rng.standard_normal((p.nh, p.np_))
    ons, no = O.natural_orbitals(O.dvv(p))
    de, _, _ = O.discarded_correction_mr(p, no, p.nvir)
    assert abs(de) <= 1e-12 * abs(O.pt2_energy(p))
    from copy import copy
    q = copy(p)
    q.nvir = 0
    q.B = np.ascontiguousarray(p.B[:, :, : p.nact])
    q.eps = p.eps[: p.ncore + p.nact]
    q.f_hp = p.f_hp[:, : p.nact]
    de0, efno, _ = O.discarded_correction_mr(p, no, 0)
    assert abs(efno - O.pt2_energy(q)) <= 1e-13 * max(1.0, abs(efno))
    assert abs(de0 - (O.pt2_energy(p) - O.pt2_energy(q))) <= 1e-12 * abs(de0)
    # a kept subset of the semicanonical virtuals (NOs = identity columns)
    # equals the problem sliced to those virtuals
    eye = np.eye(p.nvir)
    k = 9
    _, efk, _ = O.discarded_correction_mr(p, eye, k)
    r = copy(p)
    r.nvir = k
    r.B = np.ascontiguousarray(p.B[:, :, : p.nact + k])
    r.eps = p.eps[: p.ncore + p.nact + k]
    r.f_hp = p.f_hp[:, : p.nact + k]
    assert abs(efk - O.pt2_energy(r)) <= 1e-12 * abs(efk)


def test_full_pt2_energy_invariances_and_s_limit():
    """E^(2) over every class is unchanged by an orthogonal rotation of the
    auxiliary index, by a permutation of the virtuals (with their energies and
    Fock columns) and by sign flips of virtual orbitals (their B and f
    columns), and vanishes at s = 0 (every amplitude does)."""
    p = make_problem(3, 4, 10, 24, seed=31, nstates=2)
    rng = np.random.default_rng(31)
    p.f_hp = 0.05 * rng.standard_normal((p.nh, p.np_))
    l3 = random_cumulant3(p.nact, 31)
    e = O.pt2_energy(p, l3)
    from copy import copy
    q = copy(p)
    Q, _ = np.linalg.qr(rng.standard_normal((p.naux, p.naux)))
    q.B = np.einsum("PQ,Qhp->Php", Q, p.B)
    assert abs(O.pt2_energy(q, l3) - e) <= 1e-12 * abs(e)
    r = copy(p)
    perm = rng.permutation(p.nvir)
    sign = rng.choice([-1.0, 1.0], p.nvir)
    cols = np.concatenate([np.arange(p.nact), p.nact + perm])
    scale = np.concatenate([np.ones(p.nact), sign])
    r.B = p.B[:, :, cols] * scale
    r.f_hp = p.f_hp[:, cols] * scale
    r.eps = np.concatenate([p.eps[: p.nh], p.eps[p.nh:][perm]])
    assert abs(O.pt2_energy(r, l3) - e) <= 1e-12 * abs(e)
    z = copy(p)
    z.s = 0.0
    assert O.pt2_energy(z, l3) == 0.0
