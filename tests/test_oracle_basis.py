"""Pins of the oracle's 1-D basis (Sec. 3.1: LGL collocation, Lagrange basis, D, mass).

Closed forms and textbook identities only; nothing here re-types the oracle's formulas.
"""
import math

import numpy as np
import numpy.polynomial.legendre as npleg
import pytest

from oracle import oracle as O


def test_lgl_closed_forms():
    x, w = O.lgl(1)
    assert np.array_equal(x, [-1.0, 1.0]) and np.allclose(w, [1.0, 1.0], atol=1e-15)
    x, w = O.lgl(2)
    assert np.allclose(x, [-1.0, 0.0, 1.0], atol=1e-15)
    assert np.allclose(w, [1 / 3, 4 / 3, 1 / 3], atol=1e-15)
    x, w = O.lgl(3)
    r = 1 / math.sqrt(5)
    assert np.allclose(x, [-1, -r, r, 1], atol=1e-15)
    assert np.allclose(w, [1 / 6, 5 / 6, 5 / 6, 1 / 6], atol=1e-15)
    x, w = O.lgl(4)
    r = math.sqrt(3 / 7)
    assert np.allclose(x, [-1, -r, 0, r, 1], atol=1e-15)
    assert np.allclose(w, [1 / 10, 49 / 90, 32 / 45, 49 / 90, 1 / 10], atol=1e-15)


@pytest.mark.parametrize("N", range(1, 8))
def test_lgl_exactness(N):
    x, w = O.lgl(N)
    assert abs(w.sum() - 2.0) < 1e-14
    for k in range(0, 2 * N):           # exact through degree 2N-1
        exact = 2.0 / (k + 1) if k % 2 == 0 else 0.0
        assert abs(np.dot(w, x ** k) - exact) < 1e-14
    k = 2 * N                           # and not beyond: the rule really is Lobatto
    assert abs(np.dot(w, x ** k) - 2.0 / (k + 1)) > 1e-6
    # interior nodes are the roots of P_N'
    dPN = npleg.legder([0] * N + [1])
    assert np.allclose(npleg.legval(x[1:-1], dPN), 0.0, atol=1e-13)


@pytest.mark.parametrize("N", range(1, 8))
def test_gl_matches_numpy_and_exactness(N):
    x, w = O.gl(N)
    xr, wr = npleg.leggauss(N + 1)
    assert np.allclose(x, xr, atol=1e-15) and np.allclose(w, wr, atol=1e-15)
    for k in range(0, 2 * N + 2):       # exact through degree 2N+1
        exact = 2.0 / (k + 1) if k % 2 == 0 else 0.0
        assert abs(np.dot(w, x ** k) - exact) < 1e-14


@pytest.mark.parametrize("N", range(1, 8))
def test_lagrange_cardinal_and_reproduction(N):
    x, _ = O.lgl(N)
    for i in range(N + 1):
        assert np.array_equal(O.lagrange(N, x, x[i]), np.eye(N + 1)[i])
    rng = np.random.default_rng(N)
    c = rng.standard_normal(N + 1)               # random degree-N polynomial
    for t in rng.uniform(-1, 1, 7):
        l = O.lagrange(N, x, t)
        assert abs(l.sum() - 1.0) < 1e-13
        assert abs(np.dot(l, np.polyval(c, x)) - np.polyval(c, t)) < 1e-12


@pytest.mark.parametrize("N", range(1, 8))
def test_dmatrix(N):
    x, w = O.lgl(N)
    D = O.dmatrix(N, x)
    for k in range(1, N + 1):                    # D x^k = k x^(k-1)
        assert np.allclose(D @ x ** k, k * x ** (k - 1), atol=1e-12)
    assert np.allclose(D.sum(axis=1), 0.0, atol=1e-12)
    Q = np.diag(w) @ D                           # summation-by-parts
    Bnd = np.zeros((N + 1, N + 1))
    Bnd[0, 0], Bnd[N, N] = -1.0, 1.0
    assert np.allclose(Q + Q.T, Bnd, atol=1e-13)


@pytest.mark.parametrize("N", range(1, 8))
def test_mass_exact_matches_legendre_closed_form(N):
    # M = V^-T diag(2/(2k+1)) V^-1 with V_ik = P_k(x_i) (Legendre Vandermonde)
    x, _ = O.lgl(N)
    V = npleg.legvander(x, N)
    Vi = np.linalg.inv(V)
    Mref = Vi.T @ np.diag([2.0 / (2 * k + 1) for k in range(N + 1)]) @ Vi
    assert np.allclose(O.mass_exact(N), Mref, atol=1e-13)
