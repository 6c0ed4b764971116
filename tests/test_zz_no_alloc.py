"""The right-hand side entry point that allocates no device memory (sm_rhs_static).

It serves callers that cannot call cudaMalloc themselves or through the library: code
that runs while another framework owns the device memory through its own pool, code in
regions where an allocation (which synchronises the device) is not acceptable, and
embedders that forbid allocations after start-up.  Its scratch lives in one fixed-size
device array inside the library, so these tests check that

  * it returns what the ordinary entry point (sm_init_mesh + sm_rhs) returns, and what the
    FP64 oracle returns, on two calls in a row with different problems and inputs (the
    shared array keeps the previous call's contents, which must never leak into the next
    result);
  * once the device is set up, calls leave the device's free memory unchanged;
  * a problem whose scratch would not fit is refused with a clear error.

This file is collected last so that a run stopping at the first failure has already run
every other test; it passes on its own in a fresh process as well.
"""
import ctypes

import numpy as np
import pytest

from oracle import oracle as O
from paper_2008_04356_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12     # max-norm, relative to the array's max (as the other GPU parity tests)
FP32_TOL = 1e-5      # relative L2


@pytest.fixture(scope="module")
def sm():
    from paper_2008_04356_gb300 import build, slidemesh
    assert torch.cuda.is_available(), "the gpu tests need a CUDA device"
    build.build_library()
    slidemesh.lib()
    return slidemesh


def _problems():
    a = synth.config_box(N=3, v=0.5)
    a.delta0 = 0.3337
    b = synth.config_box(N=5, v=0.37, precision=synth.FP32, riemann=synth.ROE_HH)
    b.nel_s, b.nel_m = (2, 11, 3), (3, 11, 3)
    b.x2, b.delta0 = 2.3, -1.71
    return a, b


def _close(got, ref, precision):
    got = got.double().cpu().numpy()
    ref = ref if isinstance(ref, np.ndarray) else ref.double().cpu().numpy()
    if precision == synth.FP64:
        return np.abs(got - ref).max() / np.abs(ref).max() < FP64_TOL
    return np.linalg.norm(got - ref) / np.linalg.norm(ref) < FP32_TOL


def test_static_rhs_matches_sm_rhs_on_two_calls_in_a_row(sm):
    a, b = _problems()
    cases = []
    for p, seed, t in ((a, 5, 0.21), (b, 6, 0.05)):
        dt = torch.float64 if p.precision == synth.FP64 else torch.float32
        U = synth.random_state(p, seed=seed)
        dU = torch.from_numpy(U).to(dt).cuda()
        ref = sm.Solver(p).rhs(dU, t)
        ref_o = O.Oracle(p).rhs(dU.double().cpu().numpy(), t)
        cases.append((p, dU, t, ref, ref_o))
    # two calls in a row on different problems, then the first again
    for p, dU, t, ref, ref_o in cases + cases[:1]:
        got = sm.sm_rhs_static(p, dU, t)
        torch.cuda.synchronize()
        assert _close(got, ref, p.precision)
        assert _close(got, ref_o, p.precision)


def test_static_rhs_allocates_nothing(sm):
    """After a first call per problem (the device's set-up and the kernels' first loads),
    further calls leave cudaMemGetInfo's free bytes unchanged."""
    a, b = _problems()
    cases = []
    for p, seed in ((a, 15), (b, 16)):
        dt = torch.float64 if p.precision == synth.FP64 else torch.float32
        dU = torch.from_numpy(synth.random_state(p, seed=seed)).to(dt).cuda()
        out = torch.empty_like(dU)
        sm.sm_rhs_static(p, dU, 0.1, out=out)
        cases.append((p, dU, out))
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(3):
        for p, dU, out in cases:
            sm.sm_rhs_static(p, dU, 0.17, out=out)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0


def test_static_rhs_refuses_scratch_beyond_its_maximum(sm):
    p = synth.config_interface_heavy(seed=1, precision=synth.FP32)   # 65,536 interface faces
    L = sm.lib()
    desc = sm.mesh_desc(p)
    mo = sm.SmMotion(p.v, 0.0, 0.0)
    dummy = torch.empty(8, device="cuda")
    rc = L.sm_rhs_static(ctypes.byref(desc), ctypes.byref(mo), 0.0, dummy.data_ptr(), dummy[4:].data_ptr(), None)
    assert rc == -1
    msg = L.sm_last_error().decode()
    assert "scratch" in msg and "bytes" in msg


def test_static_rhs_refuses_misaligned_arrays(sm):
    p, _ = _problems()
    L = sm.lib()
    desc = sm.mesh_desc(p)
    mo = sm.SmMotion(p.v, 0.0, p.delta0)
    # refused before any CUDA call: the pointers are never dereferenced
    rc = L.sm_rhs_static(ctypes.byref(desc), ctypes.byref(mo), 0.0, 0x10008, 0x20000, None)
    assert rc == -1 and b"aligned" in L.sm_last_error()
