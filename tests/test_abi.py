"""The C-ABI library builds, loads without a GPU and exports every function that
include/*.h declares; the binding's signatures name only exported functions."""
import ctypes
import math
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


def _init(L, slidemesh, p):
    h = ctypes.c_void_p()
    rc = L.sm_init_mesh(ctypes.byref(slidemesh.mesh_desc(p)), ctypes.byref(h))
    return rc, L.sm_last_error()


@pytest.mark.parametrize("case", [
    "periodic_cylinder", "periodic_ns", "periodic_bad", "volume_bad", "geom_bad",
    "cone_angle", "cone_axis", "cone_flow", "annular_radius", "annular_flow", "plane_rotation_flow",
])
def test_shape_and_option_checks_without_gpu(libpath, case):
    """Descriptions the library does not build are refused by sm_init_mesh before any CUDA
    call: the second interface off the plane Euler case,
    out-of-range options, and geometry that the annulus and the cone cannot map."""
    from paper_2008_04356_gb300 import slidemesh, synth
    L = slidemesh.lib()
    if case == "periodic_cylinder":
        p = synth.config_cylinder(N=3)
        p.periodic_x = 1
        want, msg = -7, b"periodic x"
    elif case == "periodic_ns":
        p = synth.config_shear_x(N=3)
        p.periodic_x = 1
        want, msg = -7, b"periodic x"
    elif case == "periodic_bad":
        p = synth.config_box(N=3)
        p.periodic_x = 2
        want, msg = -1, b"periodic_x"
    elif case == "volume_bad":
        p = synth.config_box(N=3)
        p.volume = 5
        want, msg = -1, b"volume integral"
    elif case == "geom_bad":
        p = synth.config_box(N=3)
        p.geom = 9
        want, msg = -7, b"geometry"
    elif case == "cone_angle":
        p = synth.config_cone(N=3)
        p.cone_angle = 0.5 * math.pi
        want, msg = -1, b"half-angle"
    elif case == "cone_axis":
        p = synth.config_cone(N=3, n=(-1.0, 0.1, 0.5), s=(0.0, 0.5))
        want, msg = -1, b"off the axis"
    elif case == "cone_flow":
        p = synth.config_cone(N=3)
        p.flow = synth.FLOW_ENTROPY_WAVE
        want, msg = -1, b"cone flows"
    elif case == "annular_radius":
        p = synth.config_annular(N=3, r=(0.0, 1.0))
        want, msg = -1, b"radii"
    elif case == "annular_flow":
        p = synth.config_annular(N=3)
        p.flow = synth.FLOW_MODES
        want, msg = -1, b"annular flows"
    else:
        p = synth.config_box(N=3)
        p.flow = synth.FLOW_RIGID_ROTATION
        want, msg = -1, b"need the cylinder"
    rc, err = _init(L, slidemesh, p)
    assert rc == want, (rc, err)
    assert msg in err, err


@pytest.mark.parametrize("case", ["ns", "cylinder", "split", "periodic", "rotation", "aliased", "null"])
def test_no_alloc_entry_point_checks_without_gpu(libpath, case):
    """sm_rhs_static takes the plane, one-interface, weak-form Euler operator and refuses the
    rest (and malformed calls) before touching the device."""
    from paper_2008_04356_gb300 import slidemesh, synth
    L = slidemesh.lib()
    p = synth.config_box(N=3)
    mo = slidemesh.SmMotion(v=0.5, omega=0.0, delta0=0.0)
    a, b = ctypes.c_void_p(16), ctypes.c_void_p(32)      # never dereferenced: refused first
    want = -7
    if case == "ns":
        p = synth.config_shear_x(N=3)
    elif case == "cylinder":
        p = synth.config_cylinder(N=3)
    elif case == "split":
        p.volume = synth.VOLUME_SPLIT
    elif case == "periodic":
        p.periodic_x = 1
    elif case == "rotation":
        mo = slidemesh.SmMotion(v=0.0, omega=0.4, delta0=0.0)
    elif case == "aliased":
        b, want = a, -1
    else:
        a, want = None, -1
    rc = L.sm_rhs_static(ctypes.byref(slidemesh.mesh_desc(p)), ctypes.byref(mo), 0.0, a, b, None)
    assert rc == want, (rc, L.sm_last_error())


def test_static_rhs_refuses_misaligned_arrays_without_gpu(libpath):
    """sm_rhs_static checks its arrays' 16-byte alignment before any CUDA call (the pointers
    here are never dereferenced)."""
    from paper_2008_04356_gb300 import slidemesh, synth
    L = slidemesh.lib()
    p = synth.config_box(N=3)
    mo = slidemesh.SmMotion(p.v, 0.0, 0.0)
    rc = L.sm_rhs_static(ctypes.byref(slidemesh.mesh_desc(p)), ctypes.byref(mo), 0.0, 0x10008, 0x20000, None)
    assert rc == -1 and b"aligned" in L.sm_last_error()
    rc = L.sm_rhs_static(ctypes.byref(slidemesh.mesh_desc(p)), ctypes.byref(mo), 0.0, 0x10000, 0x20004, None)
    assert rc == -1


@pytest.mark.parametrize("case", ["null_solver", "null_in", "null_out", "count", "nsteps", "dt", "t0", "stride"])
def test_stream_jobs_checks_arguments_without_gpu(libpath, case):
    """sm_stream_jobs refuses malformed calls with SM_ERR_ARG before it touches the solver or
    the device (the solver handle below is never dereferenced)."""
    import math
    from paper_2008_04356_gb300 import slidemesh
    L = slidemesh.lib()
    s, a, b = ctypes.c_void_p(16), ctypes.c_void_p(32), ctypes.c_void_p(48)
    args = dict(s=s, a=a, sa=0, b=b, sb=0, count=2, t0=0.0, dt=1e-3, nsteps=1)
    if case == "null_solver":
        args["s"] = None
    elif case == "null_in":
        args["a"] = None
    elif case == "null_out":
        args["b"] = None
    elif case == "count":
        args["count"] = -1
    elif case == "nsteps":
        args["nsteps"] = 0
    elif case == "dt":
        args["dt"] = 0.0
    elif case == "t0":
        args["t0"] = math.nan
    else:
        args["sa"] = -8
    rc = L.sm_stream_jobs(args["s"], args["a"], args["sa"], args["b"], args["sb"], args["count"], args["t0"],
                          args["dt"], args["nsteps"], None)
    assert rc == -1, (case, rc, L.sm_last_error())


def test_stream_jobs_with_no_jobs_is_a_no_op_without_gpu(libpath):
    from paper_2008_04356_gb300 import slidemesh
    L = slidemesh.lib()
    rc = L.sm_stream_jobs(ctypes.c_void_p(16), ctypes.c_void_p(32), 0, ctypes.c_void_p(48), 0, 0, 0.0, 1e-3, 1, None)
    assert rc == 0
