"""Pins of the oracle's mortar operators (Sec. 3.2, Eqs. proj_M, proj_S,
projection_domain_mortar, projection_mortar_domain; Sec. 3.3 conforming instants).

Checked against: direct interpolation (the forward L2 projection is exact for equal N),
polynomial reproduction both ways, the discrete conservation identity, and the closed
form B = J M^-1 P^T M built here from a Legendre-Vandermonde mass matrix.
"""
import numpy as np
import numpy.polynomial.legendre as npleg
import pytest

from oracle import oracle as O


def bary_interp_matrix(nodes, pts):
    """L[j, i] = ell_i(pts[j]) via the barycentric formula (independent of the oracle)."""
    n = len(nodes)
    lam = np.array([1.0 / np.prod([nodes[i] - nodes[k] for k in range(n) if k != i]) for i in range(n)])
    L = np.zeros((len(pts), n))
    for j, x in enumerate(pts):
        d = x - nodes
        hit = np.where(d == 0.0)[0]
        if len(hit):
            L[j, hit[0]] = 1.0
            continue
        t = lam / d
        L[j] = t / t.sum()
    return L


def legendre_mass(nodes):
    N = len(nodes) - 1
    Vi = np.linalg.inv(npleg.legvander(nodes, N))
    return Vi.T @ np.diag([2.0 / (2 * k + 1) for k in range(N + 1)]) @ Vi


SIGMAS = [-0.9, -0.37, 0.0, 0.2, 0.71, 0.999]


@pytest.mark.parametrize("N", range(1, 8))
@pytest.mark.parametrize("sigma", SIGMAS)
def test_forward_is_interpolation(N, sigma):
    x, _ = O.lgl(N)
    P_lo, P_hi, _, _ = O.mortar_mats(N, sigma)
    z = x
    assert np.allclose(P_lo, bary_interp_matrix(x, -1 + (1 + sigma) / 2 * (z + 1)), atol=1e-13)
    assert np.allclose(P_hi, bary_interp_matrix(x, sigma + (1 - sigma) / 2 * (z + 1)), atol=1e-13)


@pytest.mark.parametrize("N", range(1, 8))
@pytest.mark.parametrize("sigma", SIGMAS)
def test_backward_closed_form(N, sigma):
    x, _ = O.lgl(N)
    M = legendre_mass(x)
    P_lo, P_hi, B_lo, B_hi = O.mortar_mats(N, sigma)
    Mi = np.linalg.inv(M)
    assert np.allclose(B_lo, (1 + sigma) / 2 * Mi @ P_lo.T @ M, atol=1e-12)
    assert np.allclose(B_hi, (1 - sigma) / 2 * Mi @ P_hi.T @ M, atol=1e-12)


@pytest.mark.parametrize("N", range(1, 8))
@pytest.mark.parametrize("sigma", SIGMAS)
def test_polynomials_projected_exactly_both_ways(N, sigma):
    x, _ = O.lgl(N)
    P_lo, P_hi, B_lo, B_hi = O.mortar_mats(N, sigma)
    rng = np.random.default_rng(N)
    c = rng.standard_normal(N + 1)
    f = lambda t: np.polyval(c, t)                   # a degree-N polynomial on the face
    xi_lo = -1 + (1 + sigma) / 2 * (x + 1)
    xi_hi = sigma + (1 - sigma) / 2 * (x + 1)
    assert np.allclose(P_lo @ f(x), f(xi_lo), atol=1e-13)
    assert np.allclose(P_hi @ f(x), f(xi_hi), atol=1e-13)
    # back: mortar data sampled from one degree-N polynomial returns that polynomial
    assert np.allclose(B_lo @ f(xi_lo) + B_hi @ f(xi_hi), f(x), atol=1e-12)


@pytest.mark.parametrize("N", range(1, 8))
@pytest.mark.parametrize("sigma", SIGMAS)
def test_back_projection_is_conservative(N, sigma):
    """sum_i w_i (B_lo a + B_hi b)_i = J_lo sum w a + J_hi sum w b (Sec. 3.2: the unweighted
    L2 projection conserves the integral; LGL integrates degree-N data exactly)."""
    x, w = O.lgl(N)
    _, _, B_lo, B_hi = O.mortar_mats(N, sigma)
    rng = np.random.default_rng(7 * N)
    for _ in range(5):
        a, b = rng.standard_normal(N + 1), rng.standard_normal(N + 1)
        lhs = w @ (B_lo @ a + B_hi @ b)
        rhs = (1 + sigma) / 2 * (w @ a) + (1 - sigma) / 2 * (w @ b)
        assert abs(lhs - rhs) < 1e-14 * (1 + abs(rhs)) * 10


@pytest.mark.parametrize("N", range(1, 8))
def test_conforming_instants_are_identity(N):
    I = np.eye(N + 1)
    P_lo, P_hi, B_lo, B_hi = O.mortar_mats(N, -1.0)
    assert np.array_equal(P_hi, I) and np.array_equal(B_hi, I) and np.array_equal(B_lo, 0 * I)
    P_lo, P_hi, B_lo, B_hi = O.mortar_mats(N, 1.0)
    assert np.array_equal(P_lo, I) and np.array_equal(B_lo, I) and np.array_equal(B_hi, 0 * I)
    # and the limit is continuous: sigma -> -1 approaches the identity
    P_lo, P_hi, B_lo, B_hi = O.mortar_mats(N, -1.0 + 1e-12)
    assert np.allclose(P_hi, I, atol=1e-9) and np.allclose(B_hi, I, atol=1e-9)
