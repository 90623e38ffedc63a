"""The C-ABI library loads on a machine without a GPU and exports every entry
point that include/fftconv.h declares (no compute calls here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "fftconv.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b([A-Za-z_]\w*)\s*\(", src, flags=re.M)
    return sorted(set(n for n in names if not n.startswith("FC_") and n != "defined"))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("fftconv_plan_create", "fftconv_plan_destroy", "fftconv_apply", "cg_solve",
                 "fc_masked_step"):
        assert must in names


def test_library_exports_every_declared_symbol():
    import __graft_entry__
    lib_path = __graft_entry__._build_module().build()
    lib = ctypes.CDLL(lib_path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, f"not exported: {missing}"


def test_binding_has_the_same_names():
    import paper_1305_3625_b300 as fc
    for n in declared_functions():
        assert hasattr(fc, n), n


def test_version_string_without_gpu():
    import paper_1305_3625_b300 as fc
    assert "sm_103a" in fc.fc_version()


def test_plan_create_rejects_bad_sizes_without_gpu():
    """Argument checks happen before any device call."""
    import paper_1305_3625_b300 as fc
    for L, prec in ((0, 3), (4097, 3), (8, 0), (8, 4)):
        with pytest.raises(fc.FcError) as ei:
            fc.fftconv_plan_create(L, prec)
        assert ei.value.code == fc.FC_EINVAL
