"""The C-ABI library loads without a GPU and exports every entry point that
include/md.h declares (no compute calls here)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = "".join(open(os.path.join(ROOT, "include", h)).read() for h in ("md.h", "md_spme.h"))
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(md_[a-z_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    from paper_2109_09056_b300 import _native
    lib = ctypes.CDLL(_native.LIB_PATH)
    names = declared_functions()
    assert "md_create" in names and "md_force_backward" in names
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    # the binding gives every declared entry point a signature
    assert set(names) <= set(_native.SIGNATURES)


def test_python_binding_names_match_c_names():
    import paper_2109_09056_b300 as pkg
    for n in declared_functions():
        if n in ("md_last_error", "md_spme_last_error", "md_state_stream_last_error"):
            continue
        assert hasattr(pkg, n), n


def test_params_default_without_gpu():
    import paper_2109_09056_b300 as pkg
    p = pkg.md_params_default()
    assert (p.ntypes, p.rc, p.skin, p.dt, p.rebuild_every) == (1, 2.5, 0.3, 0.005, 20)
    assert p.precision == pkg.MD_MIXED
    assert p.eps[0] == 1.0 and p.sigma[0] == 1.0 and p.mass[0] == 1.0


def test_missing_library_fails_loudly(tmp_path):
    from paper_2109_09056_b300 import _native
    import pytest
    with pytest.raises(ImportError):
        _native.load(str(tmp_path / "nope.so"))
