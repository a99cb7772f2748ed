"""The natural-orbital eigensolver (Eq. 8) behind dsrg_fno_truncate.

Occupation numbers are the eigenvalues of D_vv in descending order and the
natural orbitals its eigenvectors: checked against LAPACK (numpy.linalg.eigh)
on matrices with odd and even sizes, exactly repeated eigenvalues, tight
clusters, a wide spread of magnitudes and already-diagonal input.  Vectors
are compared through the projectors onto the spans of groups of eigenvalues
that are well separated from the rest (the basis inside a degenerate group
is not unique).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2312_07008_gb300 as pkg  # noqa: E402


def solve(D):
    n = D.shape[0]
    d = torch.tensor(D, dtype=torch.float64, device="cuda")
    on = torch.empty(n, dtype=torch.float64, device="cuda")
    no = torch.empty((n, n), dtype=torch.float64, device="cuda")
    pkg.dsrg_fno_truncate(n, d, pkg.MODE_PO, 99.0, 0.01, on, no)
    return on.cpu().numpy(), no.cpu().numpy()


def with_spectrum(rng, lam):
    n = len(lam)
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    return (Q * lam) @ Q.T


def check(D, ons, nos, gap_rel=1e-6, groups=True):
    n = D.shape[0]
    w, U = np.linalg.eigh(D)
    w, U = w[::-1], U[:, ::-1]
    scale = max(np.abs(w).max(), 1e-300)
    # double-float rotations (unit about 2^-48): the rounding error of a
    # sweep grows with n; 1e-12 holds up to n = 1000 and is widened in
    # proportion above (the round-parallel kernel erred by 1.2e-12 at n = 4700)
    tol = 1e-12 * max(1.0, n / 1000.0)
    assert np.all(np.diff(ons) <= 0.0)
    np.testing.assert_allclose(ons, w, rtol=0, atol=tol * scale)
    assert np.abs(nos.T @ nos - np.eye(n)).max() < tol
    assert np.abs((nos * ons) @ nos.T - D).max() < tol * scale
    if not groups:   # large n: the residual and orthogonality above fix the vectors
        return
    # groups separated by relative gaps above gap_rel
    cuts = [0] + [k + 1 for k in range(n - 1) if w[k] - w[k + 1] > gap_rel * scale] + [n]
    for a, b in zip(cuts[:-1], cuts[1:]):
        P = U[:, a:b] @ U[:, a:b].T
        Q = nos[:, a:b] @ nos[:, a:b].T
        # subspace error ~ (rounding of A) / (gap to the rest)
        assert np.abs(P - Q).max() < 1e-14 / gap_rel + 1e-12


@pytest.mark.parametrize("n", [1, 2, 3, 17, 64, 65, 130, 257])
def test_random_spectra(n):
    rng = np.random.default_rng(n)
    X = rng.standard_normal((n, n))
    D = X + X.T
    ons, nos = solve(D)
    check(D, ons, nos)


def test_repeated_and_clustered_eigenvalues():
    rng = np.random.default_rng(5)
    lam = np.concatenate([np.full(7, 2.5), np.full(5, 1e-3), 0.7 + 1e-13 * rng.standard_normal(6),
                          rng.uniform(-1, 1, 45)])
    D = with_spectrum(rng, lam)
    D = 0.5 * (D + D.T)
    ons, nos = solve(D)
    check(D, ons, nos)


def test_wide_magnitude_range_like_occupation_numbers():
    rng = np.random.default_rng(6)
    n = 301
    lam = 10.0 ** rng.uniform(-9, 0.5, n)
    D = with_spectrum(rng, lam)
    D = 0.5 * (D + D.T)
    ons, nos = solve(D)
    check(D, ons, nos)


def test_diagonal_input_needs_no_rotation():
    lam = np.array([3.0, -1.0, 2.0, 0.5, 0.5, 7.0, 0.0])
    ons, nos = solve(np.diag(lam))
    np.testing.assert_array_equal(ons, np.sort(lam)[::-1])
    assert np.abs(np.abs(nos).sum(axis=0) - 1.0).max() == 0.0


def test_grid_barrier_timeout_is_reported_and_the_next_solve_is_clean():
    """Fault injection without a hang: with the grid barrier's spin limit
    lowered to one nap, a multi-block solve (n > 80) has a barrier wait run
    out; the expired block sets the status word, every block leaves, and the
    call returns DSRG_FNO_ERR_TIMEOUT.  The context stays usable: with the
    default limit restored the same call succeeds and matches LAPACK."""
    rng = np.random.default_rng(91)
    D = with_spectrum(rng, np.linspace(2.0, 0.01, 300))
    pkg.dsrg_fno_debug_set_barrier_limit(1)
    try:
        with pytest.raises(pkg.DsrgFnoError) as ei:
            solve(D)
        assert ei.value.status == -5
    finally:
        pkg.dsrg_fno_debug_set_barrier_limit(0)
    ons, nos = solve(D)
    check(D, ons, nos)


@pytest.mark.parametrize("colpair", [True, False], ids=["colpair", "round_parallel"])
@pytest.mark.parametrize("n", [81, 300, 1001])
def test_both_multi_block_kernels_against_lapack(colpair, n):
    """Above the one-block size both Jacobi organisations (column pairs, the
    default; round-parallel over A in global memory) reproduce LAPACK on a
    spectrum with a tight cluster and a wide spread of magnitudes."""
    rng = np.random.default_rng(n + 7)
    lam = np.concatenate([np.geomspace(2.0, 1e-7, n - 6), 0.5 + 1e-9 * np.arange(6)])
    D = with_spectrum(rng, lam)
    pkg.dsrg_fno_debug_set_eig_colpair(colpair)
    try:
        ons, nos = solve(D)
    finally:
        pkg.dsrg_fno_debug_set_eig_colpair(True)
    check(D, ons, nos)


@pytest.mark.parametrize("colpair", [True, False], ids=["colpair", "round_parallel"])
def test_column_pairs_in_several_shared_memory_chunks(colpair):
    """n = 2400: a block holds 8 pairs of a round but shared memory only 4 at
    a time, so each round is rotated in 2 chunks per block."""
    n = 2400
    rng = np.random.default_rng(11)
    lam = np.concatenate([np.geomspace(2.0, 1e-7, n - 6), 0.5 + 1e-9 * np.arange(6)])
    D = with_spectrum(rng, lam)
    pkg.dsrg_fno_debug_set_eig_colpair(colpair)
    try:
        ons, nos = solve(D)
    finally:
        pkg.dsrg_fno_debug_set_eig_colpair(True)
    check(D, ons, nos, groups=False)



def test_density_step_solves_several_matrices_in_one_call():
    """The density step of a pass solves Gamma1 and the two aa blocks of the
    hole 2-RDM together: matrices up to 80 x 80 share one launch, one block
    each; a larger one (91 x 91, the symmetric aa block of 13 active
    orbitals) is solved on its own first."""
    rng = np.random.default_rng(5)
    mats = []
    for n in (10, 91, 55, 1):
        X = rng.standard_normal((n, n))
        mats.append(X + X.T)
    out = pkg.dsrg_fno_debug_eig_batch(mats)
    assert len(out) == len(mats)
    for D, (A, V) in zip(mats, out):
        lam = np.diag(A)
        order = np.argsort(-lam, kind="stable")
        check(D, lam[order], V[:, order])
