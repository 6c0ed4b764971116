"""Pins of the curvilinear oracle on the conical sliding interface about the rotation axis
(the "rotation with a conical interface" geometry of Sec. 3.3's overview figure): a rotor
inside the cone, the stator outside, slip walls at the ends of the generator and of the
normal coordinate, periodic angular sector.

* the curl-form metrics satisfy the discrete metric identities, and J converges spectrally
  to the analytic rho (h_theta / 2) (h_s / 2) (h_n / 2) of the map;
* a state at rest is preserved to rounding at the conforming instant; off it its error
  converges spectrally with N;
* rigid rotation about the axis (a steady Euler solution): the residual equals the exact
  mesh-following derivative, spectrally in N, on static and rotating meshes;
* mass and energy totals of the RHS vanish (closed domain), and the interface flux sums of
  mass and energy cancel;
* zero rotation reproduces the conforming mesh.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2008_04356_gb300 import synth


def rel(a, b):
    return np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(b).max(), 1e-300)


def mesh_following(o, U, X, omega, Omega, rho=1.0):
    ex = np.zeros_like(U)
    if omega != 0.0:
        rot = slice(0, o.E // 2)
        ex[rot, 1] = -rho * Omega * omega * X[rot, 0]
        ex[rot, 2] = -rho * Omega * omega * X[rot, 1]
    return ex


@pytest.mark.parametrize("alpha", [math.pi / 6, 1.1])
def test_cone_metric_identities(alpha):
    N = 3
    p = synth.config_cone(N=N, nel=(2, 6, 2), omega=0.4, phi0=0.05, alpha=alpha)
    o = O.Oracle(p)
    x, _ = O.lgl(N)
    Dm = O.dmatrix(N, x)
    np_ = N + 1
    for t in (0.0, 0.7):
        Ja, J = o.metrics(t)
        Jr = Ja.reshape(o.E, 3, 3, np_, np_, np_)
        s = (np.einsum("al,enkjl->enkja", Dm, Jr[:, 0]) + np.einsum("al,enklb->enkab", Dm, Jr[:, 1])
             + np.einsum("al,enljb->enajb", Dm, Jr[:, 2]))
        assert np.abs(s).max() < 1e-13 * np.abs(Ja).max() * np.abs(Dm).max()
        assert J.min() > 0.0


def test_cone_jacobian_converges_to_the_analytic_map():
    errs = []
    for N in (2, 3, 4, 5, 6):
        p = synth.config_cone(N=N, nel=(2, 6, 2), omega=0.0)
        o = O.Oracle(p)
        _, J = o.metrics(0.0)
        X = o.coords(0.0)
        r = np.hypot(X[:, 0], X[:, 1])
        exact = r * (p.y1 - p.y0) / p.nel_s[1] * (p.z1 - p.z0) / p.nel_s[2] * (p.x1 - p.x0) / p.nel_s[0] / 8.0
        errs.append(np.abs(J - exact).max() / exact.max())
    assert all(errs[k + 1] < 0.2 * errs[k] for k in range(4)), errs
    assert errs[-1] < 1e-8


def test_cone_rest_state_at_the_conforming_instant():
    p = synth.config_cone(N=4, nel=(2, 8, 2), omega=0.0, phi0=0.0, flow="rest")
    o = O.Oracle(p)
    assert np.abs(o.rhs(o.init_state(), 0.0)).max() < 1e-11


@pytest.mark.parametrize("omega,phi0", [(0.0, 0.137), (0.4, 0.013)])
def test_cone_rest_state_error_converges(omega, phi0):
    errs = []
    for N in (2, 3, 4, 5):
        p = synth.config_cone(N=N, nel=(2, 8, 2), omega=omega, phi0=phi0, flow="rest")
        o = O.Oracle(p)
        errs.append(np.abs(o.rhs(o.init_state(), 0.0)).max())
    assert all(errs[k + 1] < 0.3 * errs[k] for k in range(3)), errs
    assert errs[-1] < 1e-5


@pytest.mark.parametrize("omega", [0.0, 0.4])
def test_cone_rigid_rotation_residual_converges(omega):
    errs = []
    for N in (2, 3, 4, 5):
        p = synth.config_cone(N=N, nel=(2, 8, 2), flow="rotation", omega=omega, phi0=0.013)
        p.fpar = (1.0, 1.0, 0.4)
        o = O.Oracle(p)
        U = o.exact_state(0.0)
        errs.append(np.abs(o.rhs(U, 0.0) - mesh_following(o, U, o.coords(0.0), omega, 0.4)).max())
    assert all(errs[k + 1] < 0.5 * errs[k] for k in range(3)), errs
    assert errs[-1] < 1e-5


def test_cone_mass_and_energy_conserved():
    p = synth.config_cone(N=3, nel=(2, 8, 2), flow="pulse", omega=0.4, phi0=0.013)
    o = O.Oracle(p)
    U = synth.random_state(p, seed=5)
    Ut = o.rhs(U, 0.3)
    tot = o.totals(Ut)
    scale = o.totals(np.abs(Ut))
    assert abs(tot[0]) < 1e-13 * scale[0] and abs(tot[4]) < 1e-13 * scale[4]
    Fs, Fm = o.interface_fluxes(U, 0.3)
    ss, sm = o.face_flux_sums(Fs, Fm)
    for v in (0, 4):
        assert abs(ss[v] + sm[v]) < 1e-13 * (abs(ss[v]) + abs(sm[v]) + 1e-30)
        assert abs(ss[v]) > 1e-6


def test_cone_zero_rotation_is_conforming():
    p = synth.config_cone(N=3, nel=(2, 6, 2), flow="pulse", omega=0.0, phi0=0.0)
    U = synth.random_state(p, seed=9)
    a = O.Oracle(p).rhs(U, 0.0)
    p.interface_conforming = 1
    b = O.Oracle(p).rhs(U, 0.0)
    assert rel(a, b) < 1e-12
