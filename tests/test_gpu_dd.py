"""Double-float stages of the fast form (test hooks of the library).

The Eq. A7 regulariser evaluated in double-float arithmetic agrees with the
float64 closed form -expm1(-s Delta^2) / Delta (relative, over the whole range
of x = s Delta^2 including the small-x branch where 1 - exp(-x) cancels), and
the digit planes of double-float rows reproduce hi + lo to the rounding of the
digit grid.
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
fp = ctypes.POINTER(ctypes.c_float)


def regularizer(delta, s):
    delta = np.ascontiguousarray(delta, dtype=np.float64)
    r1 = np.zeros_like(delta)
    y = np.zeros_like(delta)
    st = lib.dsrg_fno_debug_regularizer(len(delta), delta.ctypes.data_as(dp), s, r1.ctypes.data_as(dp),
                                        y.ctypes.data_as(dp))
    assert st == 0
    return r1, y


@pytest.mark.parametrize("s", [0.5, 1.0, 0.1, 7.3])
def test_regularizer_matches_closed_form(s):
    rng = np.random.default_rng(11)
    mag = np.concatenate([
        10.0 ** rng.uniform(-12, 1.5, 4000),
        np.sqrt(np.array([1e-3, 0.999e-3, 1.001e-3, 0.0054, np.log(2.0), 1.0, 39.99, 40.0, 40.01, 60.0]) / s),
        np.sqrt(np.arange(1, 200) / 64.0 / np.log2(np.e) / s),  # table knots n/64
    ])
    delta = mag * rng.choice([-1.0, 1.0], mag.size)
    r1, y = regularizer(delta, s)
    x = s * delta ** 2
    ref_y = np.exp(-x)
    ref_r1 = -np.expm1(-x) / delta
    # double-float products carry ~2^-46 relative error each; a handful of
    # them enter R1, and t = x log2(e) carries an absolute error ~ t 2^-45
    # into y = 2^-t
    assert np.all(np.abs(r1 - ref_r1) <= 1e-13 * np.abs(ref_r1) + 1e-300)
    # y is dropped beyond x = 40 (exp(-40) < 5e-18 against 1 in 1 + y)
    keep = x <= 40.0
    assert np.all(np.abs(y[keep] - ref_y[keep]) <= (1e-13 + 3e-14 * x[keep]) * ref_y[keep])
    assert np.all(y[~keep] <= 5e-18)


def test_regularizer_zero_and_small_delta():
    r1, y = regularizer(np.array([0.0, 1e-20, -1e-15]), 0.5)
    assert r1[0] == 0.0 and y[0] == 1.0
    # R1 -> s Delta for small Delta
    np.testing.assert_allclose(r1[1:], 0.5 * np.array([1e-20, -1e-15]), rtol=1e-12)


@pytest.mark.parametrize("ks", [3, 4, 5])
def test_dd_digit_planes_reconstruct_rows(ks):
    rng = np.random.default_rng(100 + ks)
    R, K = 29, 203
    X = rng.standard_normal((R, K)) * np.exp(rng.uniform(-20, 5, (R, 1)))
    X[3] = 0.0
    X[5, ::3] = 0.0
    hi = X.astype(np.float32)
    lo = (X - hi.astype(np.float64)).astype(np.float32)
    v = hi.astype(np.float64) + lo.astype(np.float64)
    rows = np.ascontiguousarray(np.stack([hi, lo], axis=-1))
    kp = (K + 63) // 64 * 64
    P = np.zeros((ks, R, kp), dtype=np.float32)
    e = np.zeros(R, dtype=np.int32)
    st = lib.dsrg_fno_debug_slice_rows_dd(ks, R, K, rows.ctypes.data_as(fp), P.ctypes.data_as(fp),
                                          e.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
    assert st == 0
    assert np.all(np.abs(P) <= 128) and np.all(P == np.round(P))
    assert np.all(P[:, :, K:] == 0) and np.all(P[:, 3, :] == 0)
    nz = np.abs(v).max(axis=1) > 0
    # row exponent: max |hi| < 2^e <= 2 max |hi|
    mh = np.abs(hi).max(axis=1)
    assert np.all(mh[nz] < 2.0 ** e[nz]) and np.all(2.0 ** e[nz] <= 2 * mh[nz])
    w = 2.0 ** (-7 - 8 * np.arange(ks))
    rec = np.einsum("s,srk->rk", w, P[:, :, :K]) * 2.0 ** e[:, None]
    F = 7 + 8 * (ks - 1)
    bound = 2.0 ** (e[:, None] - F) * (0.5 + 2.0 ** -15)
    assert np.all(np.abs(rec - v) <= bound)
