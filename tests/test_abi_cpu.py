"""CPU checks of the boundary: the library builds, loads and exports every
entry point that include/dsrg_fno.h declares (no compute calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if not h.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", h)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^\s*(?:int|void|int32_t|int64_t|const char\s*\*)\s*(dsrg_fno_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2312_07008_gb300 import build as b
    path = b.build()
    return ctypes.CDLL(path)


def test_header_declares_the_four_calls():
    names = declared_functions()
    for f in ("dsrg_fno_pt2_energy", "dsrg_fno_vv_opdm", "dsrg_fno_truncate", "dsrg_fno_discarded_correction"):
        assert f in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_names_match_header():
    import paper_2312_07008_gb300 as pkg
    assert sorted(pkg.EXPORTED) == declared_functions()


def test_status_strings(lib):
    lib.dsrg_fno_status_string.restype = ctypes.c_char_p
    assert lib.dsrg_fno_status_string(0) == b"ok"
    assert lib.dsrg_fno_status_string(-1) == b"invalid argument"
    assert lib.dsrg_fno_status_string(-99) == b"unknown status"


def test_missing_library_fails_loudly(tmp_path):
    from paper_2312_07008_gb300 import binding
    saved = binding._lib
    binding._lib = None
    try:
        with pytest.raises(ImportError):
            binding.load(str(tmp_path / "nope.so"))
    finally:
        binding._lib = saved


def test_noalloc_rejects_oversize_and_host_pointers_before_any_work():
    """dsrg_fno_truncate_noalloc checks its arguments on the host: nvir above
    the fixed scratch limit, and host (not device) arrays, return
    DSRG_FNO_ERR_ARG with a message to the log callback and no GPU work."""
    import numpy as np

    import paper_2312_07008_gb300 as pkg
    lib = pkg.load()
    msgs = []
    pkg.dsrg_fno_set_log_callback(lambda level, text: msgs.append((level, text)))
    try:
        k = ctypes.c_int32(-7)
        nv = 4
        d = np.eye(nv)
        on = np.zeros(nv)
        no = np.zeros((nv, nv))
        vp = lambda a: ctypes.c_void_p(a.ctypes.data)  # noqa: E731
        st = lib.dsrg_fno_truncate_noalloc(513, vp(d), 0, 98.5, 0.01, vp(on), vp(no), ctypes.byref(k), None)
        assert st == -1
        assert any("512" in t for _, t in msgs), msgs
        st = lib.dsrg_fno_truncate_noalloc(nv, vp(d), 0, 98.5, 0.01, vp(on), vp(no), ctypes.byref(k), None)
        assert st == -1
        assert any("device memory" in t for _, t in msgs), msgs
        assert k.value == -7 and not on.any()
    finally:
        pkg.dsrg_fno_set_log_callback(None)


def test_log_callback_can_be_cleared():
    import paper_2312_07008_gb300 as pkg
    lib = pkg.load()
    msgs = []
    pkg.dsrg_fno_set_log_callback(lambda level, text: msgs.append(text))
    pkg.dsrg_fno_set_log_callback(None)
    k = ctypes.c_int32()
    assert lib.dsrg_fno_truncate_noalloc(600, None, 0, 98.5, 0.01, None, None, ctypes.byref(k), None) == -1
    assert msgs == []


def test_eig_batch_rejects_bad_arguments_before_any_work():
    """The batched density eigensolve's test hook checks its arguments on the
    host: 1 to 4 matrices, sizes in range and non-null arrays."""
    import paper_2312_07008_gb300 as pkg
    lib = pkg.load()
    dp = ctypes.POINTER(ctypes.c_double)
    a = (ctypes.c_double * 4)()
    arr = (dp * 5)(*([ctypes.cast(a, dp)] * 5))
    nul = (dp * 1)()
    dims = lambda *n: (ctypes.c_int32 * len(n))(*n)  # noqa: E731
    assert lib.dsrg_fno_debug_eig_batch(0, dims(2), arr, arr) == -1
    assert lib.dsrg_fno_debug_eig_batch(5, dims(2, 2, 2, 2, 2), arr, arr) == -1
    assert lib.dsrg_fno_debug_eig_batch(1, dims(-1), arr, arr) == -1
    assert lib.dsrg_fno_debug_eig_batch(1, dims(5000), arr, arr) == -1
    assert lib.dsrg_fno_debug_eig_batch(1, dims(2), nul, arr) == -1
    assert lib.dsrg_fno_debug_eig_batch(1, None, arr, arr) == -1


def test_full_energy_calls_reject_bad_arguments_before_any_work():
    """dsrg_fno_pt2_energy_mr and dsrg_fno_discarded_correction_mr check their
    arguments on the host: a null problem, host (not device) arrays in the
    problem, and a null output return DSRG_FNO_ERR_ARG without device work."""
    import numpy as np

    import paper_2312_07008_gb300 as pkg
    from paper_2312_07008_gb300.binding import CProblem
    lib = pkg.load()
    e, ev = ctypes.c_double(7.0), ctypes.c_double(7.0)
    assert lib.dsrg_fno_pt2_energy_mr(None, None, ctypes.byref(e), ctypes.byref(ev), None) == -1
    nc, na, nv, nq = 2, 2, 3, 4
    B = np.zeros((nq, nc + na, na + nv))
    eps = np.zeros(nc + na + nv)
    g1 = np.eye(na)
    l2 = np.zeros((na,) * 4)
    w = (ctypes.c_double * 1)(1.0)
    vp = lambda a: ctypes.c_void_p(a.ctypes.data)  # noqa: E731
    c = CProblem(nc, na, nv, nq, vp(B), vp(eps), vp(g1), vp(l2), None, 1, w, 0.5, 0, 0)
    assert lib.dsrg_fno_pt2_energy_mr(ctypes.byref(c), None, ctypes.byref(e), None, None) == -1
    assert lib.dsrg_fno_pt2_energy_mr(ctypes.byref(c), None, None, None, None) == -1
    no = np.eye(nv)
    de = ctypes.c_double(7.0)
    assert lib.dsrg_fno_discarded_correction_mr(None, None, 1, vp(no), None, ctypes.byref(de), None, None,
                                                None) == -1
    assert lib.dsrg_fno_discarded_correction_mr(ctypes.byref(c), None, 1, vp(no), None, ctypes.byref(de), None,
                                                None, None) == -1
    assert e.value == 7.0 and ev.value == 7.0 and de.value == 7.0
