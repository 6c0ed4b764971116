"""The split form on curved elements on the GPU against the curvilinear oracle (Sec. 3.1, the
split formulation with Pirozzoli's flux through averaged metric terms): the rotating
cylindrical, annular and conical interfaces and the plane box through general metrics;
right-hand side (FP64 to 1e-12, FP32 to 1e-5 relative L2), RK steps, conserved mass and
energy."""
import copy
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2008_04356_gb300 import synth

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


def shape(name, N, riemann=synth.ROE_HH, prec=synth.FP64):
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
    return p


@pytest.mark.parametrize("name", ["cylinder", "annular", "cone", "plane"])
@pytest.mark.parametrize("riemann", [synth.RUSANOV, synth.ROE_HH])
@pytest.mark.parametrize("N", [1, 2, 3, 5, 7])
def test_curved_split_rhs_fp64(sm, N, riemann, name):
    p = shape(name, N, riemann)
    U = synth.random_state(p, seed=240 + N)
    ref = O.Oracle(p).rhs(U, 0.37)
    s = sm.Solver(p)
    got = s.rhs(dev(U), 0.37).cpu().numpy()
    s.close()
    assert rel_max(got, ref) < FP64_TOL


@pytest.mark.parametrize("name", ["cylinder", "annular", "cone"])
def test_curved_split_rhs_fp32(sm, name):
    for N in (3, 6, 7):
        p = shape(name, N)
        U = synth.random_state(p, seed=250 + N)
        ref = O.Oracle(p).rhs(U, 0.37)
        q = copy.deepcopy(p)
        q.precision = synth.FP32
        s = sm.Solver(q)
        got = s.rhs(dev(U, torch.float32), 0.37).cpu().numpy()
        s.close()
        assert rel_l2(got, ref) < FP32_TOL, N


@pytest.mark.parametrize("name", ["cylinder", "cone"])
def test_curved_split_steps(sm, name):
    p = shape(name, 3)
    p.flow = synth.FLOW_AXIAL_PULSE if name == "cylinder" else p.flow
    o = O.Oracle(p)
    U0 = o.init_state()
    dt = 0.5 * synth.cfl_dt(p)
    Uo, Go = U0.copy(), np.zeros_like(U0)
    o.step(Uo, Go, 0.0, dt, 4)
    s = sm.Solver(p)
    s.init_state()
    s.step(dt, 4)
    Ug, _ = s.get_state()
    d = s.diag()
    s.close()
    assert rel_max(Ug.cpu().numpy(), Uo) < FP64_TOL
    t0 = o.totals(U0)
    for v in (0, 4):
        assert abs(d["totals"][v] - t0[v]) < 1e-12 * abs(t0[v])


@pytest.mark.slow
@pytest.mark.parametrize("name", ["annular", "cone"])
def test_curved_split_full_size_sampled(sm, name):
    """The 2 x 24x48x16 annulus or cone at N = 7 (18.9 M DOF) with the split form and Roe/HH,
    the benchmark's launch configuration: sampled elements (walls, interface, periodic ends,
    interior) of the GPU RHS against the oracle element by element, FP64 to 1e-12 and FP32 to
    1e-5 relative L2."""
    if name == "cone":
        p = synth.config_cone(N=7, nel=(24, 48, 16), omega=0.4, phi0=0.913, alpha=math.pi / 6, flow="pulse")
    else:
        p = synth.config_annular(N=7, nel=(24, 48, 16), omega=0.4, phi0=0.913, flow="pulse")
    p.riemann, p.volume = synth.ROE_HH, synth.VOLUME_SPLIT
    o = O.Oracle(p)
    U = synth.random_state(p, seed=78)
    rng = np.random.default_rng(6)
    nx, ny, nz = 24, 48, 16
    pick = [(b, ix, iy, iz) for b in (0, 1) for ix in (0, nx - 1) for iy in (0, ny - 1) for iz in (0, nz - 1)]
    pick += [(int(rng.integers(2)), int(rng.integers(nx)), int(rng.integers(ny)), int(rng.integers(nz))) for _ in range(16)]
    elems = np.array([b * nx * ny * nz + ix + nx * (iy + ny * iz) for b, ix, iy, iz in pick], dtype=np.int64)
    t = 0.37
    ref = o.rhs_elements(U, t, elems)
    s = sm.Solver(p)
    got = s.rhs(dev(U), t).cpu().numpy()[elems]
    s.close()
    assert rel_max(got, ref) < FP64_TOL
    p32 = copy.deepcopy(p)
    p32.precision = synth.FP32
    s = sm.Solver(p32)
    got32 = s.rhs(dev(U, torch.float32), t).cpu().numpy()[elems]
    s.close()
    assert rel_l2(got32, ref) < FP32_TOL
