"""The C-ABI library builds, loads without a GPU and exports every function that
include/*.h declares; the binding's signatures name only exported functions."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"\b(sm_[a-z0-9_]+)\s*\([^;{}]*\)\s*;", src):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def libpath():
    from paper_2008_04356_gb300 import build
    return build.build_library()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("sm_init_mesh", "sm_set_motion", "sm_rhs", "sm_step", "sm_set_state", "sm_get_state",
                     "sm_diag", "sm_destroy", "sm_map", "sm_mortar_matrices", "sm_interface"):
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in sorted(declared_functions()) if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_signatures_match_exports(libpath):
    from paper_2008_04356_gb300 import slidemesh
    names = declared_functions()
    for n in slidemesh._SIGS:
        assert n in names, n


def test_status_strings_without_gpu(libpath):
    from paper_2008_04356_gb300 import slidemesh
    L = slidemesh.lib()
    assert L.sm_status_string(0) == b"ok"
    assert L.sm_status_string(-7) == b"unsupported"


def test_invalid_descriptions_are_rejected_before_any_cuda_call(libpath):
    from paper_2008_04356_gb300 import slidemesh, synth
    L = slidemesh.lib()
    h = ctypes.c_void_p()
    p = synth.config_box(N=9)
    assert L.sm_init_mesh(ctypes.byref(slidemesh.mesh_desc(p)), ctypes.byref(h)) == -7
    p = synth.config_box(N=3)
    p.nel_m = (4, 5, 2)                      # interface faces do not match
    assert L.sm_init_mesh(ctypes.byref(slidemesh.mesh_desc(p)), ctypes.byref(h)) == -1
    assert b"interface faces" in L.sm_last_error()
    assert L.sm_init_mesh(None, ctypes.byref(h)) == -1
