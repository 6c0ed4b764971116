"""Navier-Stokes with BR1 lifting on the GPU against the oracle (FP64 1e-12, FP32 1e-5):
lifted gradients, interface fluxes with the viscous mortar mean, the full right-hand side,
the closed-form shear residual, and RK steps."""
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


def ns_box(N, riemann=synth.RUSANOV, prec=synth.FP64, ny=7, delta0=0.3337):
    p = synth.config_box(N=N, v=0.37, precision=prec, riemann=riemann)
    p.nel_s, p.nel_m, p.x2, p.delta0 = (2, ny, 3), (3, ny, 3), 2.3, delta0
    p.physics, p.mu, p.Pr, p.Rgas = synth.NAVIER_STOKES, 0.02, 0.72, 1.0
    return p


def dev(U, dt=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(U)).to(dt).cuda()


@pytest.mark.parametrize("N", [1, 2, 3, 5, 7])
def test_gradients_fp64(sm, N):
    p = ns_box(N)
    U = synth.random_state(p, seed=40 + N)
    ref = O.Oracle(p).lifting(U, 0.07)
    g = sm.Solver(p).gradients(dev(U), 0.07).cpu().numpy()
    assert rel_max(g, ref) < FP64_TOL


@pytest.mark.parametrize("riemann", [synth.RUSANOV, synth.ROE_HH])
@pytest.mark.parametrize("N", [1, 3, 4, 7])
def test_interface_and_rhs_fp64(sm, N, riemann):
    p = ns_box(N, riemann)
    o = O.Oracle(p)
    U = synth.random_state(p, seed=50 + N)
    Fs_ref, Fm_ref = o.interface_fluxes(U, 0.11)
    ref = o.rhs(U, 0.11)
    s = sm.Solver(p)
    Fs, Fm = s.interface(dev(U), 0.11)
    Ut = s.rhs(dev(U), 0.11).cpu().numpy()
    assert rel_max(Fs.cpu().numpy(), Fs_ref) < FP64_TOL
    assert rel_max(Fm.cpu().numpy(), Fm_ref) < FP64_TOL
    assert rel_max(Ut, ref) < FP64_TOL


def test_shear_closed_form_on_gpu(sm):
    p = synth.config_shear_x(N=3, v=0.41, mu=0.03)
    p.delta0 = 0.2718
    o = O.Oracle(p)
    U = o.init_state()
    X = o.coords(0.0)[:, 0]
    w0, w1, w2 = p.fpar[2:5]
    w, dw, d2w = w0 + X * (w1 + X * w2), w1 + 2 * w2 * X, 2 * w2
    expect = np.zeros_like(U)
    expect[:, 3] = p.mu * d2w
    expect[:, 4] = p.mu * (dw * dw + w * d2w)
    Ut = sm.Solver(p).rhs(dev(U), 0.0).cpu().numpy()
    assert np.abs(Ut - expect).max() < 1e-11


@pytest.mark.parametrize("N", [2, 5])
def test_ns_steps_fp64_and_fp32(sm, N):
    p = ns_box(N)
    o = O.Oracle(p)
    U0 = o.init_state()
    dt = synth.cfl_dt(p)
    Uo, Go = U0.copy(), np.zeros_like(U0)
    o.step(Uo, Go, 0.0, dt, 6)
    s = sm.Solver(p)
    s.set_state(U0, 0.0)
    s.step(dt, 6)
    Ug, _ = s.get_state()
    assert rel_max(Ug.cpu().numpy(), Uo) < FP64_TOL
    p32 = ns_box(N, prec=synth.FP32)
    s32 = sm.Solver(p32)
    err = F.check_fp32_steps(s32, o, F.perturbed(U0, seed=130 + N), dt, 6)
    print("FP32 increment rel L2 %.2e" % err)
    s32.close()


def test_ns_zero_displacement_and_euler_limit(sm):
    p = ns_box(3, delta0=0.0)
    p.v = 0.0
    U = dev(synth.random_state(p, seed=61))
    a = sm.Solver(p).rhs(U, 0.0)
    p.interface_conforming = 1
    b = sm.Solver(p).rhs(U, 0.0)
    assert rel_max(a.cpu().numpy(), b.cpu().numpy()) < 1e-14
    q = ns_box(3)
    q.mu = 0.0
    e = synth.config_box(N=3, v=0.37)
    e.nel_s, e.nel_m, e.x2, e.delta0 = q.nel_s, q.nel_m, q.x2, q.delta0
    V = dev(synth.random_state(q, seed=62))
    assert rel_max(sm.Solver(q).rhs(V, 0.1).cpu().numpy(), sm.Solver(e).rhs(V, 0.1).cpu().numpy()) < 1e-13
