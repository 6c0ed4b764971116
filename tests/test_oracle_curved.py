"""Pins of the curvilinear oracle operator (cylindrical sliding interface, Sec. 3.3; curved
elements through the metric terms of Sec. 3.1, Eq. transformed_equation).

* the plane box written through general metrics equals the Cartesian operator (which the
  other oracle tests pin) for the RHS, interface fluxes, lifting and RK steps;
* the curl-form metrics satisfy the discrete metric identities, converge to the analytic
  metrics of the cylinder map, and the rotor's rotated metrics equal those of a mesh
  built rotated;
* free stream: preserved to rounding on the conforming cylinder; on the curved sliding
  interface it is not guaranteed (the paper ensures it for plane interfaces only) and its
  error converges spectrally with N;
* rigid rotation about the axis (a steady Euler solution): the residual equals the exact
  mesh-following derivative, spectrally in N, on static and rotating meshes;
* Navier-Stokes rigid rotation: the energy rate is the closed form 2 k Omega^2 / R away
  from the (adiabatic) walls;
* mass and energy totals of the RHS vanish (slip walls, periodic sector);
* zero rotation reproduces the conforming mesh.
"""
import copy
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2008_04356_gb300 import synth


def rel(a, b):
    return np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(b).max(), 1e-300)


def curvilinear(p):
    q = copy.deepcopy(p)
    q.geom = synth.GEOM_PLANE_CURVILINEAR
    return q


def box(N, riemann=synth.RUSANOV, ns=False):
    p = synth.config_box(N=N, v=0.37, riemann=riemann)
    p.nel_s, p.nel_m, p.x2, p.delta0 = (2, 5, 3), (3, 5, 3), 2.3, 0.1337
    if ns:
        p.physics, p.mu = synth.NAVIER_STOKES, 0.02
    return p


@pytest.mark.parametrize("riemann", [synth.RUSANOV, synth.ROE_HH])
@pytest.mark.parametrize("N", [1, 2, 3, 5])
def test_plane_through_metrics_equals_cartesian(N, riemann):
    p = box(N, riemann)
    a, b = O.Oracle(p), O.Oracle(curvilinear(p))
    U = synth.random_state(p, seed=11 + N)
    Ja, J = a.metrics(0.0)
    Jb, Jc = b.metrics(0.0)
    assert np.abs(Ja - Jb).max() < 1e-12 * np.abs(Ja).max()
    assert np.abs(J - Jc).max() < 1e-12 * np.abs(J).max()
    assert rel(b.rhs(U, 0.11), a.rhs(U, 0.11)) < 1e-12
    for fa, fb in zip(a.interface_fluxes(U, 0.11), b.interface_fluxes(U, 0.11)):
        assert rel(fb, fa) < 1e-12


@pytest.mark.parametrize("N", [2, 4])
def test_plane_through_metrics_equals_cartesian_ns(N):
    p = box(N, ns=True)
    a, b = O.Oracle(p), O.Oracle(curvilinear(p))
    U = synth.random_state(p, seed=21 + N)
    assert rel(b.lifting(U, 0.07), a.lifting(U, 0.07)) < 1e-12
    assert rel(b.rhs(U, 0.07), a.rhs(U, 0.07)) < 1e-12
    U0 = a.init_state()
    Ua, Ga, Ub, Gb = U0.copy(), np.zeros_like(U0), U0.copy(), np.zeros_like(U0)
    dt = synth.cfl_dt(p)
    a.step(Ua, Ga, 0.0, dt, 3)
    b.step(Ub, Gb, 0.0, dt, 3)
    assert rel(Ub, Ua) < 1e-12


def ddir(D, d, f):
    """derivative along reference direction d of nodal data f[..., k, j, i]"""
    if d == 0:
        return np.einsum("il,...kjl->...kji", D, f)
    if d == 1:
        return np.einsum("jl,...klx->...kjx", D, f)
    return np.einsum("kl,...ljx->...kjx", D, f)


@pytest.mark.parametrize("N", [1, 3, 6])
def test_cylinder_metric_identities(N):
    p = synth.config_cylinder(N=N, nel=(2, 6, 2), omega=0.4, phi0=0.05)
    o = O.Oracle(p)
    x, _ = O.lgl(N)
    D = O.dmatrix(N, x)
    for t in (0.0, 0.7):
        Ja, _ = o.metrics(t)
        Jr = Ja.reshape(o.E, 3, 3, N + 1, N + 1, N + 1)
        ident = sum(ddir(D, i, Jr[:, i]) for i in range(3))
        assert np.abs(ident).max() < 1e-13 * np.abs(Ja).max() * np.abs(D).max()


def test_cylinder_metrics_converge_to_the_analytic_map():
    errs = []
    for N in (1, 2, 3, 4, 5, 6):
        p = synth.config_cylinder(N=N, nel=(2, 8, 2), omega=0.0)
        o = O.Oracle(p)
        Ja, J = o.metrics(0.0)
        X = o.coords(0.0)
        r, th = np.hypot(X[:, 0], X[:, 1]), np.arctan2(X[:, 1], X[:, 0])
        hr, hth, hz = 0.25 / 2, (math.pi / 4) / 8, 0.5 / 2
        eth = np.stack([-np.sin(th), np.cos(th), 0 * th], 1)
        er = np.stack([np.cos(th), np.sin(th), 0 * th], 1)
        ez = np.stack([0 * th, 0 * th, 1 + 0 * th], 1)
        e = max(np.abs(Ja[:, 0] - hz * hr / 4 * eth).max() / (hz * hr / 4),
                np.abs(Ja[:, 1] - hr * hth * r[:, None] / 4 * ez).max() / (hr * hth / 4),
                np.abs(Ja[:, 2] - hth * hz * r[:, None] / 4 * er).max() / (hth * hz / 4),
                np.abs(J - hth * hz * hr * r / 8).max() / (hth * hz * hr / 8))
        errs.append(e)
    assert all(errs[k + 1] < errs[k] for k in range(len(errs) - 1))
    assert errs[-1] < 1e-9


def test_rotor_metrics_equal_a_mesh_built_rotated():
    phi = 0.2345
    p = synth.config_cylinder(N=3, nel=(2, 6, 2), omega=0.5, phi0=0.0)
    q = synth.config_cylinder(N=3, nel=(2, 6, 2), omega=0.0, phi0=0.0)
    q.y0, q.y1 = phi, phi + p.y1
    a, b = O.Oracle(p), O.Oracle(q)
    t = phi / 0.5
    rot = slice(0, a.E // 2)
    Ja, J = a.metrics(t)
    Jb, Jc = b.metrics(0.0)
    assert np.abs(Ja[rot] - Jb[rot]).max() < 1e-14
    assert np.abs(J[rot] - Jc[rot]).max() < 1e-14
    assert np.abs(a.coords(t)[rot] - b.coords(0.0)[rot]).max() < 1e-14


def test_cylinder_free_stream():
    # conforming cylinder: preserved to rounding (discrete metric identities)
    p = synth.config_cylinder(N=4, nel=(2, 8, 2), flow="free", omega=0.0)
    p.interface_conforming = 1
    o = O.Oracle(p)
    assert np.abs(o.rhs(o.init_state(), 0.0)).max() < 1e-9
    # curved sliding interface: error at the interface elements, spectrally small in N
    errs = []
    for N in (2, 3, 4, 5):
        p = synth.config_cylinder(N=N, nel=(2, 8, 2), flow="free", omega=0.4, phi0=0.013)
        o = O.Oracle(p)
        errs.append(np.abs(o.rhs(o.init_state(), 0.0)).max())
    assert all(errs[k + 1] < 0.2 * errs[k] for k in range(3)), errs
    assert errs[-1] < 1e-6


def mesh_following(o, U, X, omega, Omega, rho=1.0):
    """d/dt of the rigid rotation state at nodes turning with the rotor: the momentum
    vector turns with angular speed omega, rho and p stay."""
    ex = np.zeros_like(U)
    if omega != 0.0:
        rot = slice(0, o.E // 2)
        ex[rot, 1] = -rho * Omega * omega * X[rot, 0]
        ex[rot, 2] = -rho * Omega * omega * X[rot, 1]
    return ex


@pytest.mark.parametrize("omega", [0.0, 0.4])
def test_rigid_rotation_residual_converges(omega):
    errs = []
    for N in (2, 3, 4, 5):
        p = synth.config_cylinder(N=N, nel=(2, 8, 2), flow="rotation", omega=omega, phi0=0.013)
        p.fpar = (1.0, 1.0, 0.4)
        o = O.Oracle(p)
        U = o.exact_state(0.0)
        errs.append(np.abs(o.rhs(U, 0.0) - mesh_following(o, U, o.coords(0.0), omega, 0.4)).max())
    assert all(errs[k + 1] < 0.5 * errs[k] for k in range(3)), errs
    assert errs[-1] < 1e-6


def test_ns_rigid_rotation_heat_conduction_closed_form():
    errs, gerrs = [], []
    for N in (3, 4, 5):
        p = synth.config_cylinder(N=N, nel=(3, 8, 2), flow="rotation", omega=0.4, phi0=0.013,
                                  physics=synth.NAVIER_STOKES)
        p.fpar, p.mu = (1.0, 1.0, 0.4), 0.01
        o = O.Oracle(p)
        U = o.exact_state(0.0)
        ex = mesh_following(o, U, o.coords(0.0), 0.4, 0.4)
        k = p.mu * p.gamma * p.Rgas / ((p.gamma - 1.0) * p.Pr)
        ex[:, 4] = 2.0 * k * 0.4 ** 2 / p.Rgas
        # elements at the interface, away from the adiabatic walls
        nx = 3
        ids = [e for e in range(o.E) if (e < o.E // 2 and e % nx == nx - 1) or (e >= o.E // 2 and (e - o.E // 2) % nx == 0)]
        errs.append(np.abs(o.rhs(U, 0.0) - ex)[ids].max())
        # lifted gradients of (rho, u, v, w, p) = (1, -Omega y, Omega x, 0, p0 + Omega^2 r^2 / 2)
        X = o.coords(0.0)
        g = o.lifting(U, 0.0).reshape(o.E, 3, 5, -1)
        ge = np.zeros_like(g)
        ge[:, 1, 1] = -0.4
        ge[:, 0, 2] = 0.4
        ge[:, 0, 4] = 0.16 * X[:, 0]
        ge[:, 1, 4] = 0.16 * X[:, 1]
        gerrs.append(np.abs(g - ge)[ids].max())
    assert errs[1] < 0.05 * errs[0] and errs[2] < errs[1], errs
    assert errs[-1] < 1e-6
    assert gerrs[1] < 0.05 * gerrs[0] and gerrs[2] < 0.05 * gerrs[1] and gerrs[-1] < 1e-6, gerrs


@pytest.mark.parametrize("ns", [False, True])
def test_cylinder_mass_and_energy_conserved(ns):
    p = synth.config_cylinder(N=3, nel=(2, 8, 2), flow="pulse", omega=0.4, phi0=0.013,
                              physics=synth.NAVIER_STOKES if ns else synth.EULER)
    if ns:
        p.mu = 0.01
    o = O.Oracle(p)
    U = synth.random_state(p, seed=5)
    tot = o.totals(o.rhs(U, 0.3))
    scale = o.totals(np.abs(o.rhs(U, 0.3)))
    assert abs(tot[0]) < 1e-13 * scale[0] and abs(tot[4]) < 1e-13 * scale[4]
    Fs, Fm = o.interface_fluxes(U, 0.3)
    ss, sm = o.face_flux_sums(Fs, Fm)
    for v in (0, 4):
        assert abs(ss[v] + sm[v]) < 1e-13 * (abs(ss[v]) + abs(sm[v]) + 1e-30)


@pytest.mark.parametrize("ns", [False, True])
def test_cylinder_zero_rotation_is_conforming(ns):
    p = synth.config_cylinder(N=3, nel=(2, 6, 2), flow="pulse", omega=0.0, phi0=0.0,
                              physics=synth.NAVIER_STOKES if ns else synth.EULER)
    if ns:
        p.mu = 0.01
    U = synth.random_state(p, seed=9)
    a = O.Oracle(p).rhs(U, 0.0)
    p.interface_conforming = 1
    b = O.Oracle(p).rhs(U, 0.0)
    assert rel(a, b) < 1e-12
