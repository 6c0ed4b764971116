"""Curvilinear kernels on the GPU against the curvilinear oracle: the plane box through
general metrics and the rotating cylindrical sliding interface (FP64 to 1e-12, FP32 to
1e-5 relative L2): right-hand side, interface fluxes, RK steps, conserved totals."""
import copy
import math

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


def plane(N, riemann=synth.RUSANOV, prec=synth.FP64):
    p = synth.config_box(N=N, v=0.37, riemann=riemann, precision=prec)
    p.nel_s, p.nel_m, p.x2, p.delta0 = (2, 7, 3), (3, 7, 3), 2.3, 0.3337
    p.geom = synth.GEOM_PLANE_CURVILINEAR
    return p


def cylinder(N, riemann=synth.RUSANOV, prec=synth.FP64, phi0=0.913, flow="pulse", nel=(2, 9, 2)):
    p = synth.config_cylinder(N=N, nel=nel, omega=0.4, phi0=phi0, flow=flow, precision=prec)
    p.riemann = riemann
    return p


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


@pytest.mark.parametrize("riemann", [synth.RUSANOV, synth.ROE_HH])
@pytest.mark.parametrize("N", [1, 2, 3, 5, 7])
def test_plane_curvilinear_rhs_fp64(sm, N, riemann):
    check_rhs(sm, plane(N, riemann), 30 + N, 0.11)


@pytest.mark.parametrize("riemann", [synth.RUSANOV, synth.ROE_HH])
@pytest.mark.parametrize("N", [1, 2, 3, 4, 5, 6, 7])
def test_cylinder_rhs_fp64(sm, N, riemann):
    # phi0 + omega t beyond the sector angle: stator faces are seen through periodic wraps
    check_rhs(sm, cylinder(N, riemann), 40 + N, 0.37)


@pytest.mark.parametrize("t", [0.0, 0.5, 3.1])
def test_cylinder_rhs_across_wraps(sm, t):
    check_rhs(sm, cylinder(3, phi0=0.0, nel=(2, 8, 2)), 7, t)


@pytest.mark.parametrize("N", [3, 7])
def test_cylinder_rhs_fp32(sm, N):
    p = cylinder(N)
    o = O.Oracle(p)
    U = synth.random_state(p, seed=50 + N)
    ref = o.rhs(U, 0.37)
    p32 = copy.deepcopy(p)
    p32.precision = synth.FP32
    got = sm.Solver(p32).rhs(dev(U, torch.float32), 0.37).cpu().numpy()
    assert rel_l2(got, ref) < FP32_TOL


@pytest.mark.parametrize("N", [2, 5])
def test_cylinder_steps(sm, N):
    p = cylinder(N, flow="pulse")
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
    p32 = copy.deepcopy(p)
    p32.precision = synth.FP32
    s32 = sm.Solver(p32)
    err = F.check_fp32_steps(s32, o, F.perturbed(U0, seed=70 + N), dt, 4)
    print("FP32 increment rel L2 %.2e" % err)
    s32.close()
    # mass and energy: slip walls and the periodic sector keep them (to rounding)
    d = s.diag()
    t0 = o.totals(U0)
    for v in (0, 4):
        assert abs(d["totals"][v] - t0[v]) < 1e-12 * abs(t0[v])


def test_cylinder_free_stream_level(sm):
    p = cylinder(5, flow="free")
    o = O.Oracle(p)
    U = o.init_state()
    ref = o.rhs(U, 0.37)
    got = sm.Solver(p).rhs(dev(U), 0.37).cpu().numpy()
    # the curved interface's free-stream error (not zero: the paper guarantees free-stream
    # preservation on plane interfaces), identical on both sides to rounding
    assert np.abs(got - ref).max() < 1e-11
    assert np.abs(ref).max() < 1e-6


def test_cylinder_zero_rotation_is_conforming(sm):
    p = cylinder(3, phi0=0.0)
    p.v = 0.0
    U = dev(synth.random_state(p, seed=3))
    a = sm.Solver(p).rhs(U, 0.0).cpu().numpy()
    p.interface_conforming = 1
    b = sm.Solver(p).rhs(U, 0.0).cpu().numpy()
    assert rel_max(a, b) < 1e-13


def ns(p, mu=0.01):
    p.physics, p.mu = synth.NAVIER_STOKES, mu
    return p


@pytest.mark.parametrize("geom", ["plane", "cylinder"])
@pytest.mark.parametrize("N", [1, 2, 4, 7])
def test_curvilinear_ns_fp64(sm, N, geom):
    p = ns(plane(N) if geom == "plane" else cylinder(N))
    o = O.Oracle(p)
    U = synth.random_state(p, seed=60 + N)
    t = 0.37
    s = sm.Solver(p)
    g = s.gradients(dev(U), t).cpu().numpy()
    assert rel_max(g, o.lifting(U, t)) < FP64_TOL
    check_rhs(sm, p, 60 + N, t)


@pytest.mark.parametrize("N", [3, 5])
def test_cylinder_ns_steps(sm, N):
    p = ns(cylinder(N, flow="pulse"))
    o = O.Oracle(p)
    U0 = o.init_state()
    dt = 0.5 * synth.cfl_dt(p)
    Uo, Go = U0.copy(), np.zeros_like(U0)
    o.step(Uo, Go, 0.0, dt, 3)
    s = sm.Solver(p)
    s.set_state(U0, 0.0)
    s.step(dt, 3)
    Ug, _ = s.get_state()
    assert rel_max(Ug.cpu().numpy(), Uo) < FP64_TOL
    p32 = copy.deepcopy(p)
    p32.precision = synth.FP32
    s32 = sm.Solver(p32)
    err = F.check_fp32_steps(s32, o, F.perturbed(U0, seed=80 + N), dt, 3)
    print("FP32 increment rel L2 %.2e" % err)
    s32.close()


@pytest.mark.parametrize("physics", ["euler", "ns"])
@pytest.mark.parametrize("riemann", [synth.RUSANOV, synth.ROE_HH])
def test_cylinder_fp32_n7_rhs_and_steps(sm, riemann, physics):
    """FP32 at N = 7 (the benchmark's degree, built for two CTAs per SM): the right-hand side
    and three RK steps (first-stage and later-stage kernels) against the FP64 oracle."""
    p = cylinder(7, riemann)
    if physics == "ns":
        p = ns(p)
    o = O.Oracle(p)
    U = synth.random_state(p, seed=90 + riemann)
    ref = o.rhs(U, 0.37)
    p32 = copy.deepcopy(p)
    p32.precision = synth.FP32
    s32 = sm.Solver(p32)
    got = s32.rhs(dev(U, torch.float32), 0.37).cpu().numpy()
    assert rel_l2(got, ref) < FP32_TOL
    dt = 0.5 * synth.cfl_dt(p)
    err = F.check_fp32_steps(s32, o, F.perturbed(o.init_state(), seed=95 + riemann), dt, 3)
    print("FP32 increment rel L2 %.2e" % err)
    s32.close()


@pytest.mark.slow
def test_cylinder_full_size_sampled(sm):
    """The 2 x 24x48x16 cylinder at N = 7 (18.9 M DOF) in the benchmark's launch
    configuration: sampled elements (walls, interface, periodic ends, interior) of the GPU
    RHS against the oracle element by element (Euler; FP64 1e-12, FP32 1e-5 rel L2)."""
    p = synth.config_cylinder(N=7, nel=(24, 48, 16), omega=0.4, phi0=0.913, flow="pulse")
    o = O.Oracle(p)
    U = synth.random_state(p, seed=77)
    rng = np.random.default_rng(5)
    nx, ny, nz = 24, 48, 16
    pick = [(b, ix, iy, iz) for b in (0, 1) for ix in (0, nx - 1) for iy in (0, ny - 1) for iz in (0, nz - 1)]
    pick += [(int(rng.integers(2)), int(rng.integers(nx)), int(rng.integers(ny)), int(rng.integers(nz))) for _ in range(16)]
    elems = np.array([b * nx * ny * nz + ix + nx * (iy + ny * iz) for b, ix, iy, iz in pick], dtype=np.int64)
    t = 0.37
    ref = o.rhs_elements(U, t, elems)
    got = sm.Solver(p).rhs(dev(U), t).cpu().numpy()[elems]
    assert rel_max(got, ref) < FP64_TOL
    p32 = copy.deepcopy(p)
    p32.precision = synth.FP32
    got32 = sm.Solver(p32).rhs(dev(U, torch.float32), t).cpu().numpy()[elems]
    assert rel_l2(got32, ref) < FP32_TOL
