"""The fast-form contraction kernel by itself (test hook of the library).

The digit planes of a row reproduce it to the rounding of F = 7 + 8 (k-1)
fraction bits, and the tensor-core product of two planed matrices equals the
float64 product of the rounded operands up to the dropped digit levels.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2312_07008_gb300 as pkg  # noqa: E402

lib = pkg.load()
dp = ctypes.POINTER(ctypes.c_double)


def planes(ks, X):
    R, K = X.shape
    kp = (K + 63) // 64 * 64
    P = np.zeros((ks, R, kp), dtype=np.float32)
    e = np.zeros(R, dtype=np.int32)
    X = np.ascontiguousarray(X)
    st = lib.dsrg_fno_debug_slice_rows(ks, R, K, X.ctypes.data_as(dp), P.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                       e.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
    assert st == 0
    return P, e


def gemm(ks, A, B):
    M, K = A.shape
    N = B.shape[0]
    C = np.zeros((M, N))
    st = lib.dsrg_fno_debug_sliced_gemm(ks, M, N, K, np.ascontiguousarray(A).ctypes.data_as(dp),
                                        np.ascontiguousarray(B).ctypes.data_as(dp), C.ctypes.data_as(dp))
    assert st == 0
    return C


@pytest.mark.parametrize("ks", [3, 4, 5, 6])
def test_digit_planes_reconstruct_rows(ks):
    rng = np.random.default_rng(ks)
    X = rng.standard_normal((37, 150)) * np.exp(rng.uniform(-20, 5, (37, 1)))
    P, e = planes(ks, X)
    assert np.all(np.abs(P) <= 128) and np.all(P == np.round(P))
    w = 2.0 ** (-7 - 8 * np.arange(ks))
    rec = np.einsum("s,srk->rk", w, P[:, :, :150]) * 2.0 ** e[:, None]
    F = 7 + 8 * (ks - 1)
    bound = 2.0 ** (e[:, None] - F - 1) * (1 + 1e-12)
    assert np.all(np.abs(rec - X) <= bound)
    assert np.all(P[:, :, 150:] == 0)


@pytest.mark.parametrize("ks", [3, 4, 5, 6])
def test_sliced_gemm_matches_planed_product(ks):
    rng = np.random.default_rng(10 + ks)
    M, N, K = 300, 157, 1100
    A = rng.standard_normal((M, K))
    B = rng.standard_normal((N, K)) * 1e-3
    C = gemm(ks, A, B)
    PA, ea = planes(ks, A)
    PB, eb = planes(ks, B)
    # level sums of the kept digit products, float64 (exact: integers < 2^53)
    ref = np.zeros((M, N))
    for sa in range(ks):
        for sb in range(ks - sa):
            ref += 2.0 ** (-14 - 8 * (sa + sb)) * (PA[sa, :, :K].astype(np.float64) @ PB[sb, :, :K].T.astype(np.float64))
    ref *= 2.0 ** (ea[:, None] + eb[None, :])
    err = np.abs(C - ref) / (np.abs(ref).max())
    print(ks, "max rel err vs planed product", err.max())
    assert err.max() < 1e-12   # levels >= 3 are accumulated in float32 (rounded)
    exact = A @ B.T
    rel = np.abs(C - exact).max() / np.abs(exact).max()
    print(ks, "vs float64 product", rel)
    # digit rounding (2^-(F+1) of the row maximum) and the dropped levels
    assert rel < [0, 0, 0, 1e-5, 1e-7, 1e-9, 1e-11][ks]


def test_sliced_gemm_exact_at_the_largest_level_sums():
    """Rows whose every digit is +-127: the level sums reach 5 * 192 * 127^2,
    just under 2^24, and must still come out exactly per chunk; the chunks
    are merged in float32 pairs (about 2^-48 relative)."""
    ks = 5
    K = 576
    # x = 127/128 + 127/128 2^-8 + ...  -> every digit 127
    x = sum(127.0 * 2.0 ** (-7 - 8 * s) for s in range(ks))
    A = np.full((130, K), x)
    B = np.full((70, K), -x)
    B[::2] *= -1.0
    C = gemm(ks, A, B)
    PA, ea = planes(ks, A)
    PB, eb = planes(ks, B)
    assert np.all(np.abs(PA[:, :, :K]) == 127)
    ref = np.zeros((130, 70))
    for sa in range(ks):
        for sb in range(ks - sa):
            ref += 2.0 ** (-14 - 8 * (sa + sb)) * (PA[sa, :, :K].astype(np.float64) @ PB[sb, :, :K].T.astype(np.float64))
    ref *= 2.0 ** (ea[:, None] + eb[None, :])
    assert np.max(np.abs(C - ref)) <= 2e-14 * np.max(np.abs(ref))
