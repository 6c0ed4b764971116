"""Pins of the oracle's Navier-Stokes terms (Sec. 2, Eqs. stress_tensor and heat_flux; BR1
lifting of Sec. 3.1; gradients projected onto the mortars, Sec. 3.2).

* the viscous flux against closed forms (Couette stress, Fourier heat flux);
* BR1 lifting exact for polynomial fields, across the sliding interface;
* the residual of the shear flow rho = p = const, v = (0, 0, w(x)), w quadratic, equals the
  closed form (0, 0, 0, mu w'', mu (w'^2 + w w'')) for N >= 3;
* mu = 0 reduces to the Euler operator bit for bit; zero displacement reproduces the
  conforming mesh bit for bit; interface flux sums of both sides cancel.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2008_04356_gb300 import synth

G = 1.4


def cons(rho, u, p):
    u = np.asarray(u, float)
    return np.array([rho, *(rho * u), p / (G - 1) + 0.5 * rho * u @ u])


def test_viscous_flux_closed_forms():
    mu, Pr, R = 0.02, 0.72, 287.0
    rho, u, p = 1.2, np.array([0.3, -0.1, 0.2]), 1.0e5
    g = np.zeros((3, 5))
    a = 4.0
    g[1, 1] = a                        # du/dy = a (Couette)
    F = O.viscous_flux(cons(rho, u, p), g.ravel(), mu, Pr, R, G)
    assert np.allclose(F[1, 1], mu * a) and np.allclose(F[0, 2], mu * a)      # tau_xy = tau_yx
    assert np.allclose(F[0, 1], 0.0) and np.allclose(F[1, 2], 0.0)
    assert np.allclose(F[1, 4], mu * a * u[0]) and np.allclose(F[0, 4], mu * a * u[1])
    # dilatation: du/dx = b gives tau_xx = 4/3 mu b, tau_yy = tau_zz = -2/3 mu b
    g = np.zeros((3, 5))
    g[0, 1] = 3.0
    F = O.viscous_flux(cons(rho, u, p), g.ravel(), mu, Pr, R, G)
    assert np.allclose([F[0, 1], F[1, 2], F[2, 3]], [4 / 3 * mu * 3, -2 / 3 * mu * 3, -2 / 3 * mu * 3])
    # heat flux: with u = 0 and dp/dz = c at constant rho, dT/dz = c/(rho R): F_z energy = k dT/dz
    g = np.zeros((3, 5))
    g[2, 4] = 50.0
    F = O.viscous_flux(cons(rho, np.zeros(3), p), g.ravel(), mu, Pr, R, G)
    k = mu * G * R / ((G - 1) * Pr)
    assert np.allclose(F[2, 4], k * 50.0 / (rho * R)) and np.allclose(F[:, :4], 0.0)


@pytest.mark.parametrize("N", [2, 3, 5])
def test_lifting_exact_for_polynomial_field(N):
    p = synth.config_shear_x(N=N, v=0.37)
    p.delta0 = 0.123
    o = O.Oracle(p)
    U = o.init_state()
    g = o.lifting(U, 0.0)
    X = o.coords(0.0)
    w0, w1, w2 = p.fpar[2:5]
    expect = np.zeros_like(g)
    expect[:, 0, 3, :] = w1 + 2 * w2 * X[:, 0]       # d w / dx
    assert np.abs(g - expect).max() < 1e-12


@pytest.mark.parametrize("riemann", [synth.RUSANOV, synth.ROE_HH])
@pytest.mark.parametrize("N", [3, 4])
def test_ns_residual_closed_form_shear(N, riemann):
    p = synth.config_shear_x(N=N, v=0.41, mu=0.03)
    p.riemann, p.delta0 = riemann, 0.2718
    o = O.Oracle(p)
    U = o.init_state()
    Ut = o.rhs(U, 0.0)
    X = o.coords(0.0)[:, 0]
    w0, w1, w2 = p.fpar[2:5]
    w, dw, d2w = w0 + X * (w1 + X * w2), w1 + 2 * w2 * X, 2 * w2
    expect = np.zeros_like(Ut)
    expect[:, 3] = p.mu * d2w
    expect[:, 4] = p.mu * (dw * dw + w * d2w)
    assert np.abs(Ut - expect).max() < 1e-11


def test_ns_with_zero_viscosity_is_euler():
    p = synth.config_box(N=3)
    p.delta0 = 0.31
    U = synth.random_state(p, seed=8)
    e = O.Oracle(p).rhs(U, 0.1)
    p.physics, p.mu = synth.NAVIER_STOKES, 0.0
    n = O.Oracle(p).rhs(U, 0.1)
    assert np.array_equal(e, n)


@pytest.mark.parametrize("riemann", [synth.RUSANOV, synth.ROE_HH])
def test_ns_zero_displacement_is_conforming(riemann):
    p = synth.config_box(N=3, v=0.0, riemann=riemann)
    p.physics, p.mu = synth.NAVIER_STOKES, 0.02
    U = synth.random_state(p, seed=12)
    a = O.Oracle(p).rhs(U, 0.05)
    p.interface_conforming = 1
    b = O.Oracle(p).rhs(U, 0.05)
    assert np.array_equal(a, b)


def test_ns_interface_flux_sums_cancel():
    p = synth.config_box(N=4)
    p.physics, p.mu, p.delta0 = synth.NAVIER_STOKES, 0.02, 0.777
    o = O.Oracle(p)
    U = synth.random_state(p, seed=13)
    Fs, Fm = o.interface_fluxes(U, 0.0)
    ss, sm = o.face_flux_sums(Fs, Fm)
    assert np.all(np.abs(ss + sm) < 1e-12 * (1 + np.abs(ss)))
