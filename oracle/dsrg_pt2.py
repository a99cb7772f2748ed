"""FP64 CPU oracle for the FNO SA-DSRG-PT2 hot path.

TEST INFRASTRUCTURE ONLY.  Only tests, the smoke check and the bench's CPU
baseline may import this module; the CUDA path never calls it.

Plain, slow restatement of arXiv:2312.07008 (Sec. 2 and Appendix A) in
float64.  Numpy matmul / einsum / eigh serve as library steps; no blocking,
fusion or reordering beyond what each definition states.

Index conventions (Appendix A, definitions below Eq. A7 and Eq. A12):
  holes      i, j, k, l in core + active   (array index h, core first)
  particles  a, b       in active + virtual (array index p, active first)
  m, n core; u, v, w, x, y, z active; e, f, e' virtual.
  t^{ij}_{ab}: upper indices holes, lower particles.
  Delta^{ij..}_{ab..} = eps_i + eps_j + .. - eps_a - eps_b - ..
  Gamma1[u][v] = Gamma^u_v, Lambda2[u][v][x][y] = Lambda^{uv}_{xy},
  Theta = 2 delta - Gamma1 (the hole density of the active orbitals),
  Gamma2[u][v][x][y] = Lambda2 + Gamma1[u][x] Gamma1[v][y] - 1/2 Gamma1[v][x] Gamma1[u][y].
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
from scipy.sparse import coo_matrix
from scipy.sparse.csgraph import connected_components

# Below this x = s Delta^2 the regularizer uses its Taylor series.
SERIES_X0 = 1.0e-3


# --------------------------------------------------------------------------
# Regularizer (Eq. A7): R(Delta) = (1 - exp(-c s Delta^2)) / Delta
# --------------------------------------------------------------------------
def regularizer(delta, s: float, c: float = 1.0):
    """(1 - exp(-c s Delta^2)) / Delta, elementwise, float64.

    For x = c s Delta^2 < SERIES_X0 the Taylor series of 1 - exp(-x) is used:
    R = c s Delta (1 - x/2 + x^2/6 - x^3/24 + x^4/120), truncation error below
    x^5/720 relative.  Delta = 0 gives 0 (the limit of the expression).
    """
    d = np.asarray(delta, dtype=np.float64)
    x = c * s * d * d
    series = c * s * d * (1.0 - x / 2.0 + x * x / 6.0 - x ** 3 / 24.0 + x ** 4 / 120.0)
    with np.errstate(divide="ignore", invalid="ignore"):
        closed = -np.expm1(-x) / d
    out = np.where(x < SERIES_X0, series, closed)
    return np.where(d == 0.0, 0.0, out)


# --------------------------------------------------------------------------
# Problem bookkeeping
# --------------------------------------------------------------------------
@dataclass
class Spaces:
    nc: int
    na: int
    nv: int

    @property
    def nh(self):
        return self.nc + self.na

    @property
    def np_(self):
        return self.na + self.nv


def spaces(prob) -> Spaces:
    return Spaces(prob.ncore, prob.nact, prob.nvir)


def hole_eps(prob):
    return prob.eps[: prob.ncore + prob.nact]


def particle_eps(prob):
    return prob.eps[prob.ncore:]


def gamma1_holes(prob):
    """SA 1-RDM over the holes: 2 on the core diagonal, Gamma1 on active."""
    sp = spaces(prob)
    g = np.zeros((sp.nh, sp.nh))
    g[: sp.nc, : sp.nc] = 2.0 * np.eye(sp.nc)
    if sp.na:
        g[sp.nc:, sp.nc:] = prob.gamma1
    return g


def gamma2_from_cumulant(g1, lam2):
    """Gamma^{uv}_{xy} = Lambda^{uv}_{xy} + Gamma^u_x Gamma^v_y - 1/2 Gamma^v_x Gamma^u_y
    (definition following Eq. A12)."""
    return (lam2 + np.einsum("ux,vy->uvxy", g1, g1)
            - 0.5 * np.einsum("vx,uy->uvxy", g1, g1))


def gamma2_holes(prob):
    """SA spin-free 2-RDM over all holes.  The cumulant vanishes whenever an
    index is core, so only the active block of Lambda2 enters."""
    sp = spaces(prob)
    g1 = gamma1_holes(prob)
    lam = np.zeros((sp.nh,) * 4)
    if sp.na:
        a = slice(sp.nc, sp.nh)
        lam[a, a, a, a] = prob.lambda2
    return gamma2_from_cumulant(g1, lam)


def theta(prob):
    return 2.0 * np.eye(prob.nact) - prob.gamma1


def sa_lambda3(g1, lam2, g3):
    """Spin-free 3-cumulant Lambda^{xyz}_{uvw} = lambda3[x][y][z][u][v][w] of
    the ensemble from its spin-free Gamma1, 2-cumulant and 3-RDM
    Gamma3[x][y][z][u][v][w] = sum_{s,t,r} <a+_{xs} a+_{yt} a+_{zr} a_{wr} a_{vt} a_{us}>
    (the 3-body density cumulant named after Eq. A12; R-Gamma extended).

    Definition used: the spin-orbital cumulant (Gamma3 minus its antisymmetrised
    Gamma1 x lambda2 and Gamma1 x Gamma1 x Gamma1 parts) summed over the spins
    of the pairs (x,u), (y,v), (z,w), with the spin-orbital 1-RDM taken as
    Gamma1 / 2 for either spin.  A Gamma1 factor that links an upper index to
    its own lower partner keeps weight 1; one that links it to another lower
    index ties two spins together and weighs 1/2, and the other two indices
    then pair as the spins dictate.  The Gamma1^3 part weighs 2^(cycles - 3)
    per permutation of the lower indices, with its sign.  Like Lambda2, it is
    formed from the ensemble-averaged densities."""
    G, L = g1, lam2
    e = np.einsum
    return (g3
            - e("xu,yzvw->xyzuvw", G, L) - e("yv,xzuw->xyzuvw", G, L) - e("zw,xyuv->xyzuvw", G, L)
            + 0.5 * (e("xv,yzuw->xyzuvw", G, L) + e("xw,yzvu->xyzuvw", G, L)
                     + e("yu,xzvw->xyzuvw", G, L) + e("yw,xzuv->xyzuvw", G, L)
                     + e("zu,xywv->xyzuvw", G, L) + e("zv,xyuw->xyzuvw", G, L))
            - e("xu,yv,zw->xyzuvw", G, G, G)
            + 0.5 * (e("xv,yu,zw->xyzuvw", G, G, G) + e("xw,yv,zu->xyzuvw", G, G, G)
                     + e("xu,yw,zv->xyzuvw", G, G, G))
            - 0.25 * (e("xv,yw,zu->xyzuvw", G, G, G) + e("xw,yu,zv->xyzuvw", G, G, G)))


# --------------------------------------------------------------------------
# Integrals and amplitudes (Eqs. A6, A7)
# --------------------------------------------------------------------------
def nu_pair(prob, i: int, j: int, a_sel=slice(None), b_sel=slice(None)):
    """nu^{ij}_{ab} = <ab|ij> = (ai|bj) = sum_Q B^Q_{ia} B^Q_{jb}  (DF, Sec. 3)."""
    return prob.B[:, i, a_sel].T @ prob.B[:, j, b_sel]


def delta2(prob, i, j, a_idx, b_idx):
    eh, ep = hole_eps(prob), particle_eps(prob)
    return eh[i] + eh[j] - ep[a_idx][:, None] - ep[b_idx][None, :]


def t2_vv(prob, i, j):
    """t^{ij}_{ef} for e, f virtual: Eq. A7, as an [e][f] matrix."""
    sp = spaces(prob)
    v = np.arange(sp.na, sp.np_)
    nu = nu_pair(prob, i, j, v, v)
    return regularizer(delta2(prob, i, j, v, v), prob.s) * nu, nu


def t2_semi_internal(prob, holes=None):
    """ts[i][j][e][x] = t^{ij}_{ex} (e virtual, x active particle), Eq. A7,
    for every ordered hole pair (i, j); `holes` (an index array) restricts
    i and j to those holes, in that order."""
    sp = spaces(prob)
    h = np.arange(sp.nh) if holes is None else np.asarray(holes)
    Bv = prob.B[:, h, sp.na:]
    Ba = prob.B[:, h, : sp.na]
    nu = np.einsum("Qie,Qjx->ijex", Bv, Ba, optimize=True)
    eh, ep = hole_eps(prob)[h], particle_eps(prob)
    d = (eh[:, None, None, None] + eh[None, :, None, None]
         - ep[sp.na:][None, None, :, None] - ep[: sp.na][None, None, None, :])
    return nu * regularizer(d, prob.s)


def t1_amplitudes(prob, ts=None):
    """t1[i][e] = t^i_e for i hole, e virtual (Eq. A6):
    t^i_a = [f^i_a + 1/2 sum_{ux} Delta^x_u Gamma^x_u tcheck^{iu}_{ax}] R(Delta^i_a),
    with tcheck^{ij}_{ab} = 2 t^{ij}_{ab} - t^{ji}_{ab} and Delta^x_u = eps_x - eps_u."""
    sp = spaces(prob)
    eh, ep = hole_eps(prob), particle_eps(prob)
    ev = ep[sp.na:]
    f = np.zeros((sp.nh, sp.nv))
    if prob.f_hp is not None:
        f = np.array(prob.f_hp[:, sp.na:], dtype=np.float64)
    if sp.na:
        if ts is None:
            ts = t2_semi_internal(prob)
        act = slice(sp.nc, sp.nh)
        eu = eh[act]
        ex = ep[: sp.na]
        dxu = ex[None, :] - eu[:, None]            # [u][x] = eps_x - eps_u
        g_xu = prob.gamma1                          # [x][u] = Gamma^x_u
        tcheck = 2.0 * ts[:, act, :, :] - np.transpose(ts[act, :, :, :], (1, 0, 2, 3))  # [i][u][e][x]
        f = f + 0.5 * np.einsum("ux,xu,iuex->ie", dxu, g_xu, tcheck)
    dia = eh[:, None] - ev[None, :]
    return f * regularizer(dia, prob.s)


# --------------------------------------------------------------------------
# E_vv: second-order energy of the doubles with both particles virtual
# --------------------------------------------------------------------------
def hole_pair_components(prob, g2h=None):
    """Connected components of ordered hole pairs coupled by Gamma2_H != 0."""
    sp = spaces(prob)
    if g2h is None:
        g2h = gamma2_holes(prob)
    nh = sp.nh
    flat = g2h.reshape(nh * nh, nh * nh)
    r, c = np.nonzero(flat)
    adj = coo_matrix((np.ones(len(r)), (r, c)), shape=(nh * nh, nh * nh))
    ncomp, lab = connected_components(adj, directed=False)
    comps = [[] for _ in range(ncomp)]
    for idx, l in enumerate(lab):
        comps[l].append((idx // nh, idx % nh))
    return [cmp for cmp in comps if any(flat[i * nh + j].any() for i, j in cmp)]


def _pair_blocks(prob, pairs):
    """nu, tau, Delta for the ordered pairs; (j, i) is the transpose of (i, j)."""
    cache = {}
    for (i, j) in pairs:
        if (i, j) in cache:
            continue
        tau, nu = t2_vv(prob, i, j)
        sp = spaces(prob)
        v = np.arange(sp.na, sp.np_)
        d = delta2(prob, i, j, v, v)
        cache[(i, j)] = (nu, tau, d)
        cache[(j, i)] = (nu.T, tau.T, d.T)
    return cache


def e_vv(prob, components=None):
    """E_vv = 1/2 sum_{ijkl in H, ef in V} Gamma2_H[k][l][i][j] tau^{ij}_{ef}
                 [2 nu^{kl}_{ef} - Delta^{ij}_{ef} tau^{kl}_{ef}]

    The scalar of <[V, A]> + 1/2 <[[H0, A], A]> (Eq. A4) restricted to the
    doubles whose particles are both virtual.  Those operators carry no
    normal-ordering contractions, so the reference enters through the SA
    2-RDM over holes only.  `components` restricts the sum to some coupled
    pair groups (used for sampling)."""
    g2h = gamma2_holes(prob)
    nh = spaces(prob).nh
    comps = hole_pair_components(prob, g2h) if components is None else components
    total = 0.0
    for comp in comps:
        blocks = _pair_blocks(prob, comp)
        keys = list(comp)
        nu = np.stack([blocks[k][0].ravel() for k in keys])
        tau = np.stack([blocks[k][1].ravel() for k in keys])
        dt = np.stack([(blocks[k][2] * blocks[k][1]).ravel() for k in keys])
        g1 = tau @ nu.T          # [ij][kl] = <tau^{ij}, nu^{kl}>
        g2 = dt @ tau.T          # [ij][kl] = <Delta^{ij} tau^{ij}, tau^{kl}>
        for a, (i, j) in enumerate(keys):
            for b, (k, l) in enumerate(keys):
                w = g2h[k, l, i, j]
                if w != 0.0:
                    total += 0.5 * w * (2.0 * g1[a, b] - g2[a, b])
    return total


# --------------------------------------------------------------------------
# Full multi-reference SA-DSRG-PT2 energy (the scalar of Eq. A4's H-bar)
# --------------------------------------------------------------------------
def t2_general(prob):
    """Dense first-order doubles t^{ij}_{ab} = <ab|ij> R(Delta^{ij}_{ab}) of
    Eq. A7 for every hole pair (i, j in core + active) and particle pair
    (a, b in active + virtual), zero on the all-active block, which the
    cluster operator excludes.  Returns (t [nh][nh][np][np], nu, Delta)."""
    sp = spaces(prob)
    eh, ep = hole_eps(prob), particle_eps(prob)
    nu = np.einsum("Qia,Qjb->ijab", prob.B, prob.B, optimize=True)
    d = (eh[:, None, None, None] + eh[None, :, None, None]
         - ep[None, None, :, None] - ep[None, None, None, :])
    t = nu * regularizer(d, prob.s)
    t[sp.nc:, sp.nc:, : sp.na, : sp.na] = 0.0
    return t, nu, d


def t1_general(prob, t2):
    """First-order singles t^i_a of Eq. A6 for every hole i and particle a
    (zero when both are active):
        t^i_a = [f^i_a + r^i_a] R(Delta^i_a),
        r^i_a = 1/2 sum_{ux} Delta^x_u Gamma^x_u tcheck^{iu}_{ax},
    with tcheck^{iu}_{ax} = 2 t^{iu}_{ax} - t^{ui}_{ax} and Delta^x_u =
    eps_x - eps_u.  r^i_a is the one-body part of [H0, T2] (the term Eq. A6
    adds to f).  Returns (t1 [nh][np], f, r, Delta^i_a)."""
    sp = spaces(prob)
    eh, ep = hole_eps(prob), particle_eps(prob)
    f = (np.zeros((sp.nh, sp.np_)) if prob.f_hp is None
         else np.array(prob.f_hp, dtype=np.float64))
    r = np.zeros_like(f)
    if sp.na:
        act = slice(sp.nc, sp.nh)
        dxu = ep[: sp.na][None, :] - eh[act][:, None]            # [u][x] = eps_x - eps_u
        tch = (2.0 * t2[:, act, :, : sp.na]
               - np.transpose(t2[act, :, :, : sp.na], (1, 0, 2, 3)))   # [i][u][a][x]
        r = 0.5 * np.einsum("ux,xu,iuax->ia", dxu, prob.gamma1, tch, optimize=True)
    d1 = eh[:, None] - ep[None, :]
    t1 = (f + r) * regularizer(d1, prob.s)
    t1[sp.nc:, : sp.na] = 0.0
    return t1, f, r, d1


def commutator_scalar(prob, X1, X2, T1, T2, lambda3=None):
    """<[X, T]>_0: the fully contracted part of the commutator of
        X = sum_{ia} X1[i][a] E^i_a + 1/2 sum_{ijab} X2[i][j][a][b] E^{ij}_{ab}
        T = sum_{kc} T1[k][c] E^c_k + 1/2 sum_{klcd} T2[k][l][c][d] E^{cd}_{kl}
    (i, j, k, l holes; a, b, c, d particles; X2 and T2 symmetric under the
    pair transpose), both normal ordered with respect to the ensemble in the
    Mukherjee-Kutzelnigg sense named after Eq. A2.

    The terms follow from the generalised Wick theorem: contractions between
    the two strings are gamma = Gamma/2 (creator of X with annihilator of T),
    eta = Theta/2 (annihilator of X with creator of T) and one density
    cumulant; a term made of cumulants alone is the same in both orders and
    cancels, so every term has at most one cumulant.  Spins are summed with
    the spin-free cumulants defined after Eq. A12 (the alpha and beta
    1-RDMs equal), which gives (Gamma over holes: 2 on the core diagonal;
    Theta over particles: 2 on the virtual diagonal; cumulants on the active
    indices only)
      1/2 X1 T1 Gamma Theta
      + 1/8 sum Gamma2_H[i][j][k][l] X2^{ij}_{ab} (Theta Theta T2)^{kl}_{ab}
      + the one-cumulant terms written out below."""
    sp = spaces(prob)
    nc, na, nh = sp.nc, sp.na, sp.nh
    G = gamma1_holes(prob)
    G2 = gamma2_holes(prob)
    Th = np.zeros((sp.np_, sp.np_))
    Th[na:, na:] = 2.0 * np.eye(sp.nv)
    if na:
        Th[:na, :na] = theta(prob)
    e = 0.5 * np.einsum("ia,kc,ik,ca->", X1, T1, G, Th, optimize=True)
    tt = np.einsum("ac,bd,klcd->klab", Th, Th, T2, optimize=True)
    e += 0.125 * np.einsum("ijkl,ijab,klab->", G2, X2, tt, optimize=True)
    if na == 0:
        return e
    L = prob.lambda2
    h, p = slice(nc, nh), slice(0, na)       # active holes, active particles
    # one-body X with two-body T
    e += 0.5 * np.einsum("ia,klcd,da,iclk->", X1[h], T2[h, h, p], Th, L, optimize=True)
    e -= 0.5 * np.einsum("ia,klcd,ik,cdal->", X1[:, p], T2[:, h, p, p], G, L, optimize=True)
    # two-body X with one-body T
    e += 0.5 * np.einsum("ijab,kc,ca,ijkb->", X2[h, h, :, p], T1[h], Th, L, optimize=True)
    e -= 0.5 * np.einsum("ijab,kc,jk,icab->", X2[h, :, p, p], T1[:, p], G, L, optimize=True)
    # two-body X with two-body T, one 2-cumulant
    e -= 0.25 * np.einsum("ijab,klcd,jk,da,iclb->", X2[h, :, :, p], T2[:, h, p], G, Th, L, optimize=True)
    e -= 0.25 * np.einsum("ijab,klcd,jl,da,icbk->", X2[h, :, :, p], T2[h, :, p], G, Th, L, optimize=True)
    e -= 0.25 * np.einsum("ijab,klcd,jk,db,ical->", X2[h, :, p], T2[:, h, p], G, Th, L, optimize=True)
    e += 0.5 * np.einsum("ijab,klcd,jl,db,icak->", X2[h, :, p], T2[h, :, p], G, Th, L, optimize=True)
    e += 0.125 * np.einsum("ijab,klcd,il,jk,cdba->", X2[:, :, p, p], T2[:, :, p, p], G, G, L, optimize=True)
    if lambda3 is not None:
        # one 3-cumulant Lambda^{xyz}_{uvw} = lambda3[x][y][z][u][v][w]
        e += 0.5 * np.einsum("ijab,klcd,da,ijclbk->", X2[h, h, :, p], T2[h, h, p], Th, lambda3, optimize=True)
        e -= 0.5 * np.einsum("ijab,klcd,jk,icdabl->", X2[h, :, p, p], T2[:, h, p, p], G, lambda3, optimize=True)
    return e


def pt2_energy(prob, lambda3=None):
    """Second-order SA-DSRG energy E^(2) = <[H, A]>_0 + 1/2 <[[H0, A], A]>_0,
    the correlation part of <H-bar^[2]> (Eq. A4), with A = T - T^+ and the
    first-order T1, T2 of Eqs. A6, A7 over every class (core and active holes,
    active and virtual particles).  `lambda3` adds the 3-cumulant terms; without
    it they are dropped, which Sec. 2 allows when the 1-RDM drops them too.

    With H Hermitian and [H0, T] an excitation operator, every scalar reduces to
    2 <[X, T]>_0 with the de-excitation vertex X = H + 1/2 [H0, T]^+ restricted
    to upper holes and lower particles:
      X2^{ij}_{ab} = <ab|ij> - 1/2 Delta^{ij}_{ab} t^{ij}_{ab},
      X1^i_a       = f^i_a - 1/2 Delta^i_a t^i_a + 1/2 r^i_a
    (the all-active parts of X and of [H0, T] contract with nothing)."""
    T2, nu, d2 = t2_general(prob)
    T1, f, r, d1 = t1_general(prob, T2)
    X2 = nu - 0.5 * d2 * T2
    X1 = f - 0.5 * d1 * T1 + 0.5 * r
    return 2.0 * commutator_scalar(prob, X1, X2, T1, T2, lambda3)


# --------------------------------------------------------------------------
# D_vv (Eq. A12, terms 1-12; the Lambda3 term 13 only with a 3-cumulant)
# --------------------------------------------------------------------------
def dvv_terms(prob, terms=range(1, 14), ts=None, t1=None, core_pairs=None, lambda3=None, ca_pairs=None,
              aa_pairs=None):
    """Returns {term number: [nvir][nvir] contribution} for Eq. A12.
    `core_pairs` restricts term 4 to the listed unordered core pairs (m <= n),
    `ca_pairs` term 5 to the listed (m, u) (the sum over v kept whole), and
    `aa_pairs` term 7 to the listed (u, v) (the sum over x, y kept whole):
    partial sums, used to time a sample of the oracle.
    Term 13 is formed only when `lambda3` ([na]^6, Lambda^{xyz}_{uvw}) is given."""
    sp = spaces(prob)
    nc, na, nv = sp.nc, sp.na, sp.nv
    out = {}
    if na:
        if ts is None:
            ts = t2_semi_internal(prob)
        G = prob.gamma1
        L = prob.lambda2
        Th = theta(prob)
        G2 = gamma2_from_cumulant(G, L)
        A = slice(nc, nc + na)
        C = slice(0, nc)
    if t1 is None:
        t1 = t1_amplitudes(prob, ts)
    want = set(terms)

    if 1 in want:   # 2 t^m_e t^m_f
        tc = t1[:nc]
        out[1] = 2.0 * tc.T @ tc
    if na and 2 in want:   # t^u_e t^v_f Gamma^u_v
        ta = t1[nc:]
        out[2] = np.einsum("ue,vf,uv->ef", ta, ta, G)
    if na and 3 in want:   # (t^u_e t^{xy}_{fv} + t^{uv}_{ey} t^x_f) Lambda^{uv}_{xy}
        ta = t1[nc:]
        taa = ts[A, A]     # [x][y][f][v] = t^{xy}_{fv}
        out[3] = (np.einsum("ue,xyfv,uvxy->ef", ta, taa, L, optimize=True)
                  + np.einsum("uvey,xf,uvxy->ef", taa, ta, L, optimize=True))
    if 4 in want:   # 2 t^{mn}_{ee'} tcheck^{mn}_{fe'}
        d = np.zeros((nv, nv))
        plist = core_pairs if core_pairs is not None else [(m, n) for m in range(nc) for n in range(m, nc)]
        for m, n in plist:
            T, _ = t2_vv(prob, m, n)          # t^{mn}; t^{nm} = T^T
            d += 2.0 * T @ (2.0 * T - T.T).T
            if n != m:
                d += 2.0 * T.T @ (2.0 * T.T - T).T
        out[4] = d
    if na and 5 in want:   # S(t^{mu}_{ee'} tcheck^{mv}_{fe'}) Gamma^u_v
        d = np.zeros((nv, nv))
        msel = range(nc) if ca_pairs is None else sorted({m for m, _ in ca_pairs})
        for m in msel:
            Tm = [t2_vv(prob, m, nc + u)[0] for u in range(na)]   # t^{mu}; t^{um} = (t^{mu})^T
            for u in range(na):
                if ca_pairs is not None and (m, u) not in ca_pairs:
                    continue
                for v in range(na):
                    g = G[u, v]
                    if g == 0.0:
                        continue
                    tu, tv = Tm[u], Tm[v]
                    d += g * (tu @ (2.0 * tv - tv.T).T            # t^{mu} tcheck^{mv}
                              + tu.T @ (2.0 * tv.T - tv).T)       # t^{um} tcheck^{vm}
        out[5] = d
    if na and 6 in want:   # t^{mn}_{ev} tcheck^{mn}_{fu} Theta^u_v
        tcc = ts[C, C]
        tch = 2.0 * tcc - np.transpose(tcc, (1, 0, 2, 3))
        out[6] = np.einsum("mnev,mnfu,uv->ef", tcc, tch, Th, optimize=True)
    if na and 7 in want:   # t^{uv}_{ee'} t^{xy}_{fe'} Gamma^{uv}_{xy}
        Tuv = {}
        for u in range(na):
            for v in range(u, na):
                T, _ = t2_vv(prob, nc + u, nc + v)
                Tuv[(u, v)] = T
                Tuv[(v, u)] = T.T
        d = np.zeros((nv, nv))
        for u in range(na):
            for v in range(na):
                if aa_pairs is not None and (u, v) not in aa_pairs:
                    continue
                W = np.zeros((nv, nv))
                for x in range(na):
                    for y in range(na):
                        W += G2[u, v, x, y] * Tuv[(x, y)]
                d += Tuv[(u, v)] @ W.T
        out[7] = d
    if na and 8 in want:   # 1/2 S(t^{mu}_{ey} tcheck^{mv}_{fx}) Gamma^u_v Theta^x_y
        tca = ts[C, A]     # [m][u][e][y] = t^{mu}_{ey}
        tac = ts[A, C]     # [u][m][e][y] = t^{um}_{ey}
        tch_ca = 2.0 * tca - np.transpose(tac, (1, 0, 2, 3))   # tcheck^{mv}_{fx}
        tch_ac = 2.0 * tac - np.transpose(tca, (1, 0, 2, 3))   # tcheck^{vm}_{fx}
        out[8] = 0.5 * (np.einsum("muey,mvfx,uv,xy->ef", tca, tch_ca, G, Th, optimize=True)
                        + np.einsum("umey,vmfx,uv,xy->ef", tac, tch_ac, G, Th, optimize=True))
    if na and 9 in want:   # P(t^{mv}_{ey} t^{mx}_{fu}) Lambda^{uv}_{xy}
        tca = ts[C, A]
        tac = ts[A, C]
        out[9] = (2.0 * np.einsum("mvey,mxfu,uvxy->ef", tca, tca, L, optimize=True)
                  - np.einsum("mvey,xmfu,uvxy->ef", tca, tac, L, optimize=True)
                  - np.einsum("vmey,mxfu,uvxy->ef", tac, tca, L, optimize=True)
                  - np.einsum("vmex,ymfu,uvxy->ef", tac, tac, L, optimize=True))
    if na and 10 in want:   # 1/2 t^{uv}_{ez} t^{xy}_{fw} Theta^w_z Lambda^{uv}_{xy}
        taa = ts[A, A]
        out[10] = 0.5 * np.einsum("uvez,xyfw,wz,uvxy->ef", taa, taa, Th, L, optimize=True)
    if na and 11 in want:   # 1/4 t^{ux}_{ez} tcheck^{vy}_{fw} Gamma^u_v Gamma^x_y Theta^w_z
        # Reading: the printed term carries a plain t on its second factor; the
        # Fock-space evaluation of Eq. A11 requires tcheck there (the printed
        # form misses -1/4 t^{ux}_{ez} t^{yv}_{fw} Gamma^u_v Gamma^x_y Theta^w_z).
        taa = ts[A, A]
        tch = 2.0 * taa - np.transpose(taa, (1, 0, 2, 3))
        out[11] = 0.25 * np.einsum("uxez,vyfw,uv,xy,wz->ef", taa, tch, G, G, Th, optimize=True)
    if na and 12 in want:   # 1/2 P(t^{wv}_{ey} t^{zx}_{fu}) Gamma^w_z Lambda^{uv}_{xy}
        taa = ts[A, A]
        out[12] = 0.5 * (2.0 * np.einsum("wvey,zxfu,wz,uvxy->ef", taa, taa, G, L, optimize=True)
                         - np.einsum("wvey,xzfu,wz,uvxy->ef", taa, taa, G, L, optimize=True)
                         - np.einsum("vwey,zxfu,wz,uvxy->ef", taa, taa, G, L, optimize=True)
                         - np.einsum("vwex,yzfu,wz,uvxy->ef", taa, taa, G, L, optimize=True))
    if na and lambda3 is not None and 13 in want:
        out[13] = dvv_term13(ts[A, A], lambda3)
    return out


def dvv_term13(taa, lambda3):
    """Eq. A12 term 13: t^{uw}_{ez} t^{xy}_{fv} Lambda^{xyz}_{uvw}, with
    taa[u][w][e][z] = t^{uw}_{ez} (active holes u, w; e virtual, z active)."""
    return np.einsum("uwez,xyfv,xyzuvw->ef", taa, taa, lambda3, optimize=True)


def dvv(prob, return_asym=False, lambda3=None):
    """Symmetrised D_vv = 1/2 (D + D^T) of Eq. A12 terms 1-12 (13 with lambda3)."""
    parts = dvv_terms(prob, lambda3=lambda3)
    d = sum(parts.values())
    sym = 0.5 * (d + d.T)
    if return_asym:
        return sym, np.linalg.norm(d - d.T)
    return sym


# --------------------------------------------------------------------------
# Natural orbitals, truncation, recanonicalisation, correction (Sec. 2)
# --------------------------------------------------------------------------
def natural_orbitals(d):
    """Gamma V = n V (Eq. 8), ONs descending.  Each column's component of
    largest magnitude is made positive."""
    w, v = np.linalg.eigh(d)
    order = np.argsort(-w, kind="stable")
    w, v = w[order], v[:, order]
    idx = np.argmax(np.abs(v), axis=0)
    sgn = np.sign(v[idx, np.arange(v.shape[1])])
    sgn[sgn == 0] = 1.0
    return w, v * sgn[None, :]


MODE_PO, MODE_PV, MODE_NKAPPA, MODE_FIXED = 0, 1, 2, 3


def truncate(ons, mode: int, threshold: float, degen_ratio: float = 0.01):
    """Number of kept NOs N' for ONs sorted descending.

    mode 0 (p_o, Eq. 10): smallest N' with sum_{p<=N'} n_p >= p_o/100 * sum_all n_p
    mode 1 (p_v, Eq. 9):  N' = ceil(p_v/100 * N_V)
    mode 2 (n_kappa):     number of ONs >= n_kappa
    mode 3 (fixed):       N' = threshold, rounded and clamped to [0, N_V] (the
                          same N' along a potential energy surface, Sec. 4)
    Then the near-degeneracy widening: while N' < N_V and the next ON differs
    from the last kept one by less than degen_ratio times the larger of the
    two, keep it as well."""
    n = np.asarray(ons, dtype=np.float64)
    nv = len(n)
    if mode == MODE_PO:
        target = threshold / 100.0 * np.sum(n)
        cum = np.cumsum(n)
        hit = np.nonzero(cum >= target)[0]
        k = int(hit[0]) + 1 if len(hit) else nv
    elif mode == MODE_PV:
        k = int(np.ceil(threshold / 100.0 * nv - 1e-12))
    elif mode == MODE_NKAPPA:
        k = int(np.count_nonzero(n >= threshold))
    elif mode == MODE_FIXED:
        k = int(np.rint(min(max(threshold, 0.0), float(nv))))
    else:
        raise ValueError("mode")
    k = max(0, min(nv, k))
    while 0 < k < nv and (n[k - 1] - n[k]) < degen_ratio * max(n[k - 1], n[k]):
        k += 1
    return k


def recanonicalize(prob, no, nkept):
    """Diagonalise the virtual Fock block in the kept NO space.  The VV Fock
    block is diag(eps_v) in the semicanonical basis, so F' = Vk^T diag(eps_v) Vk;
    returns U = Vk W and eps' ascending."""
    ev = particle_eps(prob)[prob.nact:]
    vk = no[:, :nkept]
    fk = vk.T @ (ev[:, None] * vk)
    w, W = np.linalg.eigh(fk)
    return vk @ W, w


def fno_problem(prob, U, eps_new):
    """Same problem with the virtual space rotated to U (nvir x N')."""
    from copy import copy
    p2 = copy(prob)
    na = prob.nact
    Bv = np.einsum("Qhe,ek->Qhk", prob.B[:, :, na:], U, optimize=True)
    p2.B = np.ascontiguousarray(np.concatenate([prob.B[:, :, :na], Bv], axis=2))
    p2.nvir = U.shape[1]
    p2.eps = np.concatenate([prob.eps[: prob.ncore + na], eps_new])
    if prob.f_hp is not None:
        p2.f_hp = np.concatenate([prob.f_hp[:, :na], prob.f_hp[:, na:] @ U], axis=1)
    return p2


def discarded_correction(prob, no, nkept, e_mo=None):
    """Scalar part of Eq. 11: E_vv(MO) - E_vv(FNO).  Returns (dE, E_fno, eps')."""
    if e_mo is None:
        e_mo = e_vv(prob)
    U, eps_new = recanonicalize(prob, no, nkept)
    if nkept == 0:
        return e_mo, 0.0, eps_new
    e_fno = e_vv(fno_problem(prob, U, eps_new))
    return e_mo - e_fno, e_fno, eps_new


def discarded_correction_mr(prob, no, nkept, lambda3=None, e_mo=None):
    """Eq. 11 with the full second-order energy: E^(2)(MO) - E^(2)(FNO), the
    FNO problem being the kept NOs recanonicalised (B, the virtual orbital
    energies and the virtual columns of f_hp rotated; the active particles
    stay).  This carries the active-labelled parts of the correction (the
    doubles with an active particle, the singles) beside the vv part.
    Returns (dE, E_fno, eps')."""
    if e_mo is None:
        e_mo = pt2_energy(prob, lambda3)
    U, eps_new = recanonicalize(prob, no, nkept)
    e_fno = pt2_energy(fno_problem(prob, U, eps_new), lambda3)
    return e_mo - e_fno, e_fno, eps_new


# --------------------------------------------------------------------------
# Particle-particle ladder of Eq. 6 in the truncated virtual basis
# --------------------------------------------------------------------------
def ladder(B_vv, T):
    """The term of C2 = [O2, T2]_2 (Eq. 6) with four virtual indices, whose
    O(N_C^2 N_V^4) cost the FNO truncation cuts by (N_V'/N_V)^4:
        C^{ij}_{ab} = sum_{cd} <ab|cd> T^{ij}_{cd},
        <ab|cd> = (ac|bd) = sum_Q B^Q_{ac} B^Q_{bd}   (DF, Sec. 3).
    B_vv [naux][nv][nv] virtual-virtual factors, T [npairs][nv][nv]
    (T[p][c][d] = T^{ij}_{cd} of hole pair p); returns C [npairs][nv][nv].
    The 4-index integrals are formed explicitly (plain definition)."""
    V = np.einsum("Qac,Qbd->abcd", B_vv, B_vv, optimize=True)
    return np.einsum("abcd,pcd->pab", V, T, optimize=True)


# --------------------------------------------------------------------------
# Natural auxiliary functions (Sec. 4: compression of the auxiliary basis)
# --------------------------------------------------------------------------
def naf(prob, threshold):
    """Natural auxiliary functions of the hole-particle DF factors.

    W_PQ = sum_{i a} B^P_{ia} B^Q_{ia} (i hole, a particle) is diagonalised,
    W = U diag(w) U^T with w descending; the natural auxiliary functions
    are the columns of U with w > threshold, and the compressed factors are
    B'^K_{ia} = sum_Q U_QK B^Q_{ia}.  Returns (B' [k][nh][np], w, U)."""
    nq = prob.naux
    B2 = prob.B.reshape(nq, -1)
    W = B2 @ B2.T
    w, U = np.linalg.eigh(W)
    order = np.argsort(-w, kind="stable")
    w, U = w[order], U[:, order]
    k = int(np.count_nonzero(w > threshold))
    Bp = (U[:, :k].T @ B2).reshape((k,) + prob.B.shape[1:])
    return Bp, w, U


def naf_problem(prob, threshold):
    """The same problem with B replaced by its natural-auxiliary-function
    compression (naux -> the number of kept functions)."""
    from copy import copy
    Bp, _, _ = naf(prob, threshold)
    p2 = copy(prob)
    p2.B = np.ascontiguousarray(Bp)
    p2.naux = Bp.shape[0]
    return p2


def solve(prob, cuts=(98.5,), mode=MODE_PO, degen_ratio=0.01):
    """The whole path: E_vv, D_vv, NOs/ONs, N' per cut, correction per cut."""
    e2 = e_vv(prob)
    d, asym = dvv(prob, return_asym=True)
    ons, no = natural_orbitals(d)
    res = dict(e2=e2, dvv=d, asym=asym, ons=ons, no=no, cuts={})
    for c in cuts:
        k = truncate(ons, mode, c, degen_ratio)
        de, efno, epsn = discarded_correction(prob, no, k, e2)
        res["cuts"][c] = dict(nkept=k, de=de, e_fno=efno, eps_fno=epsn)
    return res
