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
