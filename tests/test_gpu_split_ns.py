"""The split form with Navier-Stokes physics on the GPU (Sec. 3.1: Pirozzoli's split form for
the advective terms, BR1 lifting for the viscous ones, Roe with the Harten-Hyman fix: the
scheme of the paper's computations) against the FP64 CPU oracle, through the C-ABI.

The oracle evaluates the strong form literally (2 D F# over every pair, the surface term
F* - F_adv(U), the viscous flux in the weak form); the kernel folds the advective surface
correction into Ds = 2 D - M^-1 B and contracts the viscous flux with Dhat beside it.  Bars:
FP64 1e-12 relative (max norm), FP32 1e-5 relative L2 (steps by increments, fp32_steps).
"""
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
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def split_ns_box(N, riemann=synth.ROE_HH, prec=synth.FP64, ny=7, delta0=0.3337, mu=0.02):
    """Ragged two-block box (element counts that fill no whole CTA), sub-face offset."""
    p = synth.config_box(N=N, v=0.37, precision=prec, riemann=riemann)
    p.nel_s, p.nel_m, p.x2, p.delta0 = (2, ny, 3), (3, ny, 3), 2.3, delta0
    p.physics, p.mu, p.Pr, p.Rgas = synth.NAVIER_STOKES, mu, 0.72, 1.0
    p.volume = synth.VOLUME_SPLIT
    return p


def dev(U, dt=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(U)).to(dt).cuda()


@pytest.mark.parametrize("riemann", [synth.RUSANOV, synth.ROE_HH])
@pytest.mark.parametrize("N", range(1, 8))
def test_split_ns_rhs_fp64(sm, N, riemann):
    p = split_ns_box(N, riemann)
    o = O.Oracle(p)
    U = synth.random_state(p, seed=500 + N)
    ref = o.rhs(U, 0.11)
    s = sm.Solver(p)
    Ut = s.rhs(dev(U), 0.11).cpu().numpy()
    s.close()
    assert rel_max(Ut, ref) < FP64_TOL


@pytest.mark.parametrize("riemann", [synth.RUSANOV, synth.ROE_HH])
def test_split_ns_rhs_fp32(sm, riemann):
    for N in (1, 3, 5, 7):
        p = split_ns_box(N, riemann, prec=synth.FP32)
        U = synth.random_state(p, seed=520 + N).astype(np.float32)
        ref = O.Oracle(p).rhs(U.astype(np.float64), 0.3)
        s = sm.Solver(p)
        Ut = s.rhs(dev(U, torch.float32), 0.3).cpu().numpy()
        s.close()
        assert rel_l2(Ut, ref) < FP32_TOL, N


@pytest.mark.parametrize("riemann", [synth.RUSANOV, synth.ROE_HH])
def test_split_ns_shear_closed_form_on_gpu(sm, riemann):
    """rho = p = const, v = (0, 0, w(x)), w quadratic: residual (0, 0, 0, mu w'', mu (w'^2 + w w''))."""
    p = synth.config_shear_x(N=3, v=0.41, mu=0.03)
    p.riemann, p.delta0, p.volume = riemann, 0.2718, synth.VOLUME_SPLIT
    o = O.Oracle(p)
    U = o.init_state()
    X = o.coords(0.0)[:, 0]
    w0, w1, w2 = p.fpar[2:5]
    w, dw, d2w = w0 + X * (w1 + X * w2), w1 + 2 * w2 * X, 2 * w2
    expect = np.zeros_like(U)
    expect[:, 3] = p.mu * d2w
    expect[:, 4] = p.mu * (dw * dw + w * d2w)
    s = sm.Solver(p)
    Ut = s.rhs(dev(U), 0.0).cpu().numpy()
    s.close()
    assert np.abs(Ut - expect).max() < 1e-11


def test_split_ns_zero_viscosity_and_zero_displacement(sm):
    """mu = 0 gives the split Euler operator; zero displacement the conforming mesh (to
    rounding: the GPU paths inline their flux arithmetic in different kernels)."""
    p = split_ns_box(3, mu=0.0)
    U = dev(synth.random_state(p, seed=531))
    e = split_ns_box(3)
    e.physics, e.mu = synth.EULER, 0.0
    a = sm.Solver(p).rhs(U, 0.1).cpu().numpy()
    b = sm.Solver(e).rhs(U, 0.1).cpu().numpy()
    assert rel_max(a, b) < 1e-13
    q = split_ns_box(3, delta0=0.0)
    q.v = 0.0
    c = sm.Solver(q).rhs(U, 0.0).cpu().numpy()
    q.interface_conforming = 1
    d = sm.Solver(q).rhs(U, 0.0).cpu().numpy()
    assert rel_max(c, d) < 1e-13


@pytest.mark.parametrize("N", [2, 5])
def test_split_ns_steps_fp64_and_fp32(sm, N):
    p = split_ns_box(N)
    o = O.Oracle(p)
    U0 = o.init_state()
    dt = synth.cfl_dt(p)
    Uo, Go = U0.copy(), np.zeros_like(U0)
    o.step(Uo, Go, 0.0, dt, 6)
    s = sm.Solver(p)
    s.set_state(U0, 0.0)
    s.step(dt, 2)
    s.step(dt, 4)
    Ug, _ = s.get_state()
    s.close()
    assert rel_max(Ug.cpu().numpy(), Uo) < FP64_TOL
    s32 = sm.Solver(split_ns_box(N, prec=synth.FP32))
    err = F.check_fp32_steps(s32, o, F.perturbed(U0, seed=540 + N), dt, 6)
    s32.close()
    print("N=%d: FP32 increment rel L2 %.2e" % (N, err))


# ------------------------------------------------------------------ curved elements
def curved(name, N, riemann=synth.ROE_HH, prec=synth.FP64, mu=0.01):
    """The rotating shapes (and the plane box through general metrics) with the split form and
    Navier-Stokes physics."""
    if name == "cylinder":
        p = synth.config_cylinder(N=N, nel=(2, 9, 2), omega=0.4, phi0=0.913, precision=prec)
    elif name == "annular":
        p = synth.config_annular(N=N, nel=(2, 9, 3), omega=0.4, phi0=0.913, precision=prec)
    elif name == "cone":
        p = synth.config_cone(N=N, nel=(2, 9, 3), omega=0.4, phi0=0.913, alpha=0.6, precision=prec)
    else:
        p = synth.config_box(N=N, v=0.37, precision=prec)
        p.nel_s, p.nel_m, p.x2, p.delta0 = (2, 7, 3), (3, 7, 3), 2.3, 0.3337
        p.geom = synth.GEOM_PLANE_CURVILINEAR
    p.riemann, p.volume = riemann, synth.VOLUME_SPLIT
    p.physics, p.mu = synth.NAVIER_STOKES, mu
    return p


@pytest.mark.parametrize("name", ["cylinder", "annular", "cone", "plane"])
@pytest.mark.parametrize("riemann", [synth.RUSANOV, synth.ROE_HH])
@pytest.mark.parametrize("N", [1, 2, 3, 5, 7])
def test_curved_split_ns_rhs_fp64(sm, N, riemann, name):
    p = curved(name, N, riemann)
    U = synth.random_state(p, seed=560 + N)
    ref = O.Oracle(p).rhs(U, 0.37)
    s = sm.Solver(p)
    got = s.rhs(dev(U), 0.37).cpu().numpy()
    s.close()
    assert rel_max(got, ref) < FP64_TOL


@pytest.mark.parametrize("name", ["cylinder", "annular", "cone"])
def test_curved_split_ns_rhs_fp32(sm, name):
    for N in (3, 6, 7):
        p = curved(name, N)
        U = synth.random_state(p, seed=570 + N)
        ref = O.Oracle(p).rhs(U, 0.37)
        s = sm.Solver(curved(name, N, prec=synth.FP32))
        got = s.rhs(dev(U, torch.float32), 0.37).cpu().numpy()
        s.close()
        assert rel_l2(got, ref) < FP32_TOL, N


@pytest.mark.parametrize("name", ["cylinder", "cone"])
def test_curved_split_ns_steps_and_conservation(sm, name):
    """FP64 steps against the oracle; mass and energy kept by the closed rotating shape (slip
    walls, adiabatic, periodic sector); FP32 steps by increments."""
    p = curved(name, 3)
    p.flow = synth.FLOW_AXIAL_PULSE if name == "cylinder" else p.flow
    o = O.Oracle(p)
    U0 = o.init_state()
    dt = 0.5 * synth.cfl_dt(p)
    Uo, Go = U0.copy(), np.zeros_like(U0)
    o.step(Uo, Go, 0.0, dt, 4)
    s = sm.Solver(p)
    s.set_state(U0, 0.0)
    s.step(dt, 4)
    Ug, _ = s.get_state()
    d = s.diag()
    s.close()
    assert rel_max(Ug.cpu().numpy(), Uo) < FP64_TOL
    t0 = o.totals(U0)
    for v in (0, 4):
        assert abs(d["totals"][v] - t0[v]) < 1e-12 * abs(t0[v])
    q = curved(name, 3, prec=synth.FP32)
    q.flow = p.flow
    s32 = sm.Solver(q)
    err = F.check_fp32_steps(s32, o, F.perturbed(U0, seed=580), dt, 4)
    s32.close()
    print("%s: FP32 increment rel L2 %.2e" % (name, err))
