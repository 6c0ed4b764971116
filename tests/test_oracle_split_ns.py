"""Pins of the oracle's split form with Navier-Stokes physics (Sec. 3.1: the split formulation
with Pirozzoli's flux for the advective terms, BR1 lifting for the viscous ones; the paper's
production scheme).  The viscous flux keeps the weak form and the face flux carries the BR1
viscous mean, so:

* the shear flow rho = p = const, v = (0, 0, w(x)) with w quadratic has the closed-form
  residual (0, 0, 0, mu w'', mu (w'^2 + w w'')), as for the weak form;
* mu = 0 gives the split Euler operator bit for bit, zero displacement the conforming mesh;
* with the central two-point flux the split form is the weak form (summation by parts), on
  the sliding box and on the rotating cylinder, annulus and cone;
* kinetic-energy balance: for a face-continuous state at constant pressure whose velocity
  vanishes on the Dirichlet faces, the semi-discrete kinetic-energy rate equals minus the
  discrete viscous dissipation sum J w tau(grad v) : grad v of the lifted gradients (the
  advective part preserves kinetic energy, the BR1 terms telescope); the weak form does not
  meet it;
* mass and energy totals of the residual vanish on the closed rotating geometries.
"""
import copy
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2008_04356_gb300 import synth

G = 1.4


def ns(p, mu=0.01):
    p.physics, p.mu = synth.NAVIER_STOKES, mu
    return p


def shapes(N=3, omega=0.4, phi0=0.3):
    return {
        "cylinder": synth.config_cylinder(N=N, nel=(2, 8, 2), omega=omega, phi0=phi0),
        "annular": synth.config_annular(N=N, nel=(2, 8, 2), omega=omega, phi0=phi0),
        "cone": synth.config_cone(N=N, nel=(2, 8, 2), omega=omega, phi0=phi0),
    }


@pytest.mark.parametrize("riemann", [synth.RUSANOV, synth.ROE_HH])
@pytest.mark.parametrize("N", [3, 4])
def test_split_ns_residual_closed_form_shear(N, riemann):
    p = synth.config_shear_x(N=N, v=0.41, mu=0.03)
    p.riemann, p.delta0, p.volume = riemann, 0.2718, synth.VOLUME_SPLIT
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


def test_split_ns_with_zero_viscosity_is_split_euler():
    p = synth.config_box(N=3, riemann=synth.ROE_HH)
    p.delta0, p.volume = 0.31, synth.VOLUME_SPLIT
    U = synth.random_state(p, seed=8)
    e = O.Oracle(p).rhs(U, 0.1)
    p.physics, p.mu = synth.NAVIER_STOKES, 0.0
    n = O.Oracle(p).rhs(U, 0.1)
    assert np.array_equal(e, n)


@pytest.mark.parametrize("riemann", [synth.RUSANOV, synth.ROE_HH])
def test_split_ns_zero_displacement_is_conforming(riemann):
    p = ns(synth.config_box(N=3, v=0.0, riemann=riemann), 0.02)
    p.volume = synth.VOLUME_SPLIT
    U = synth.random_state(p, seed=12)
    a = O.Oracle(p).rhs(U, 0.05)
    p.interface_conforming = 1
    b = O.Oracle(p).rhs(U, 0.05)
    assert np.array_equal(a, b)


@pytest.mark.parametrize("riemann", [synth.RUSANOV, synth.ROE_HH])
@pytest.mark.parametrize("N", [2, 4])
def test_central_split_ns_is_the_weak_ns_on_the_sliding_box(N, riemann):
    p = ns(synth.config_box(N=N, v=0.37, riemann=riemann))
    p.nel_s, p.nel_m, p.delta0 = (2, 7, 3), (3, 7, 3), 0.3337
    U = synth.random_state(p, seed=N)
    weak = O.Oracle(p).rhs(U, 0.11)
    q = copy.deepcopy(p)
    q.volume = 2
    central = O.Oracle(q).rhs(U, 0.11)
    assert np.abs(central - weak).max() < 1e-13 * np.abs(weak).max()


@pytest.mark.parametrize("shape", ["cylinder", "annular", "cone"])
def test_central_curved_split_ns_is_the_curved_weak_ns(shape):
    p = ns(shapes()[shape])
    U = synth.random_state(p, seed=5)
    weak = O.Oracle(p).rhs(U, 0.2)
    p.volume = 2
    central = O.Oracle(p).rhs(U, 0.2)
    assert np.abs(central - weak).max() < 1e-13 * np.abs(weak).max()


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5, 6, 7])
def test_split_ns_kinetic_energy_balance(N):
    rates = {}
    for vol in (synth.VOLUME_SPLIT, synth.VOLUME_WEAK):
        p = ns(synth.config_box(N=N, v=0.5, riemann=synth.ROE_HH), 0.02)
        p.flow, p.fpar, p.delta0, p.volume = synth.FLOW_CONSTANT, (1.0, 0.0, 0.0, 0.0, 1.0), 0.0, vol
        o = O.Oracle(p)
        X = o.coords(0.0)
        x, y, z = X[:, 0], X[:, 1], X[:, 2]
        rng = np.random.default_rng(7 + N)
        # vanishes on the Dirichlet faces x = x0, x2, where the state is the Dirichlet state
        wall = np.sin(math.pi * (x - p.x0) / (p.x2 - p.x0))

        def field(amp):
            f = np.zeros_like(x)
            for _ in range(3):
                kx, ky, kz = rng.integers(1, 3), rng.integers(-2, 3), rng.integers(-2, 3)
                f += amp * rng.uniform(0.3, 1.0) * np.sin(math.pi * kx * x + 2 * math.pi * ky * y
                                                           + 2 * math.pi * kz * z + rng.uniform(0, 2 * math.pi))
            return f

        rho = 1.0 + wall * field(0.1)
        u, v, w = wall * field(0.2), wall * field(0.2), wall * field(0.2)
        U = np.stack([rho, rho * u, rho * v, rho * w, 1.0 / (G - 1) + 0.5 * rho * (u * u + v * v + w * w)], axis=1)
        Ut = o.rhs(U, 0.0)
        g = o.lifting(U, 0.0)                         # (E, 3, 5, nn): d(prim c)/dx_a
        L = np.transpose(g[:, :, 1:4, :], (0, 2, 1, 3))  # L[:, b, a] = d v_b / d x_a
        div = L[:, 0, 0] + L[:, 1, 1] + L[:, 2, 2]
        tau = p.mu * (L + np.transpose(L, (0, 2, 1, 3)) - (2.0 / 3.0) * div[:, None, None] * np.eye(3)[None, :, :, None])
        dissipation = (tau * L).sum(axis=(1, 2))
        ke = u * Ut[:, 1] + v * Ut[:, 2] + w * Ut[:, 3] - 0.5 * (u * u + v * v + w * w) * Ut[:, 0]
        F = np.zeros_like(Ut)
        F[:, 0], F[:, 1], F[:, 2] = ke, dissipation, np.abs(ke)
        t = o.totals(F)
        rates[vol] = abs(t[0] + t[1]) / t[2]
    assert rates[synth.VOLUME_SPLIT] < 1e-13
    if N <= 5:
        assert rates[synth.VOLUME_WEAK] > 1e-7


@pytest.mark.parametrize("shape", ["cylinder", "annular", "cone"])
def test_curved_split_ns_conserves_mass_and_energy(shape):
    p = ns(shapes()[shape])
    p.volume, p.riemann = synth.VOLUME_SPLIT, synth.ROE_HH
    o = O.Oracle(p)
    Ut = o.rhs(synth.random_state(p, seed=6), 0.1)
    tot, scale = o.totals(Ut), o.totals(np.abs(Ut))
    assert abs(tot[0]) < 1e-13 * scale[0] and abs(tot[4]) < 1e-13 * scale[4]
