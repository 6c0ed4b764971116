"""The other rotating interface shapes on the GPU against the curvilinear oracle: the plane
annular interface normal to the rotation axis (rotor below the stator) and the conical
interface (rotor inside the cone), both with slip walls and a periodic sector: right-hand
side and interface fluxes (FP64 to 1e-12, FP32 to 1e-5 relative L2), RK steps, conserved
mass and energy, Navier-Stokes with BR1 lifting."""
import copy

import numpy as np
import pytest

from oracle import oracle as O
from paper_2008_04356_gb300 import synth

import fp32_steps as F

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12
FP32_TOL = 1e-5


@pytest.fixture(scope="module")
def sm():
    from paper_2008_04356_gb300 import build, slidemesh
    assert torch.cuda.is_available(), "the gpu tests need a CUDA device"
    build.build_library()
    slidemesh.lib()
    return slidemesh


def rel_max(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def rel_l2(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def dev(U, dt=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(U)).to(dt).cuda()


def annulus(N, riemann=synth.RUSANOV, prec=synth.FP64, phi0=0.913, flow="pulse", nel=(2, 9, 3)):
    """Uneven element counts: 2 axial layers per block, 9 angular, 3 radial."""
    p = synth.config_annular(N=N, nel=nel, omega=0.4, phi0=phi0, flow=flow, precision=prec)
    p.riemann = riemann
    return p


def cone(N, riemann=synth.RUSANOV, prec=synth.FP64, phi0=0.913, flow="pulse", nel=(2, 9, 3)):
    """Half-angle 0.6 rad; 2 normal layers per block, 9 angular, 3 along the generator."""
    p = synth.config_cone(N=N, nel=nel, omega=0.4, phi0=phi0, alpha=0.6, flow=flow, precision=prec)
    p.riemann = riemann
    return p


SHAPES = {"annular": annulus, "cone": cone}


def check_rhs(sm, p, seed, t, tol=FP64_TOL):
    o = O.Oracle(p)
    U = synth.random_state(p, seed=seed)
    ref = o.rhs(U, t)
    s = sm.Solver(p)
    got = s.rhs(dev(U), t).cpu().numpy()
    assert rel_max(got, ref) < tol
    Fs, Fm = s.interface(dev(U), t)
    Fs_ref, Fm_ref = o.interface_fluxes(U, t)
    assert rel_max(Fs.cpu().numpy(), Fs_ref) < tol
    assert rel_max(Fm.cpu().numpy(), Fm_ref) < tol
    s.close()


@pytest.mark.parametrize("shape", ["annular", "cone"])
@pytest.mark.parametrize("riemann", [synth.RUSANOV, synth.ROE_HH])
@pytest.mark.parametrize("N", [1, 2, 3, 4, 5, 6, 7])
def test_shape_rhs_fp64(sm, N, riemann, shape):
    # phi0 + omega t beyond the sector angle: stator faces are seen through periodic wraps
    check_rhs(sm, SHAPES[shape](N, riemann), 140 + N, 0.37)


@pytest.mark.parametrize("shape", ["annular", "cone"])
@pytest.mark.parametrize("t", [0.0, 0.5, 3.1])
def test_shape_rhs_across_wraps(sm, t, shape):
    check_rhs(sm, SHAPES[shape](3, phi0=0.0, nel=(2, 8, 2)), 17, t)


@pytest.mark.parametrize("shape", ["annular", "cone"])
@pytest.mark.parametrize("N", [3, 7])
def test_shape_rhs_fp32(sm, N, shape):
    p = SHAPES[shape](N)
    o = O.Oracle(p)
    U = synth.random_state(p, seed=150 + N)
    ref = o.rhs(U, 0.37)
    p32 = copy.deepcopy(p)
    p32.precision = synth.FP32
    s = sm.Solver(p32)
    got = s.rhs(dev(U, torch.float32), 0.37).cpu().numpy()
    s.close()
    assert rel_l2(got, ref) < FP32_TOL


@pytest.mark.parametrize("shape", ["annular", "cone"])
@pytest.mark.parametrize("N", [2, 5])
def test_shape_steps(sm, N, shape):
    p = SHAPES[shape](N, flow="pulse")
    o = O.Oracle(p)
    U0 = o.init_state()
    dt = 0.5 * synth.cfl_dt(p)
    Uo, Go = U0.copy(), np.zeros_like(U0)
    o.step(Uo, Go, 0.0, dt, 4)
    s = sm.Solver(p)
    s.init_state()
    U_init, _ = s.get_state()
    assert rel_max(U_init.cpu().numpy(), U0) < 1e-13
    s.step(dt, 4)
    Ug, t = s.get_state()
    assert abs(t - 4 * dt) < 1e-15
    assert rel_max(Ug.cpu().numpy(), Uo) < FP64_TOL
    # mass and energy: slip walls and the periodic sector keep them (to rounding)
    d = s.diag()
    t0 = o.totals(U0)
    for v in (0, 4):
        assert abs(d["totals"][v] - t0[v]) < 1e-12 * abs(t0[v])
    s.close()
    p32 = copy.deepcopy(p)
    p32.precision = synth.FP32
    s32 = sm.Solver(p32)
    err = F.check_fp32_steps(s32, o, F.perturbed(U0, seed=110 + N), dt, 4)
    print("FP32 increment rel L2 %.2e" % err)
    s32.close()


@pytest.mark.parametrize("shape", ["annular", "cone"])
def test_shape_zero_rotation_is_conforming(sm, shape):
    p = SHAPES[shape](3, phi0=0.0)
    p.v = 0.0
    U = dev(synth.random_state(p, seed=3))
    a = sm.Solver(p).rhs(U, 0.0).cpu().numpy()
    p.interface_conforming = 1
    b = sm.Solver(p).rhs(U, 0.0).cpu().numpy()
    assert rel_max(a, b) < 1e-13


@pytest.mark.parametrize("shape", ["annular", "cone"])
@pytest.mark.parametrize("N", [2, 4])
def test_shape_ns_fp64(sm, N, shape):
    p = SHAPES[shape](N, riemann=synth.ROE_HH)
    p.physics, p.mu = synth.NAVIER_STOKES, 0.01
    check_rhs(sm, p, 160 + N, 0.21)
