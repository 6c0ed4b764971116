"""Pins of the oracle's time integration (Sec. 3.1: Carpenter-Kennedy low-storage RK4).

The 2N-storage recurrence G = A_k G + dt f(t + c_k dt, U); U += B_k G is written here in
its generic form and run on scalar ODEs: fourth order on y' = lambda y, exact on
y' = t^3 (quadrature order conditions pin the stage times c_k), and orc_step itself is
fourth order in time on a flow that DGSEM resolves exactly in space.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2008_04356_gb300 import synth


def lsrk(f, y0, t0, dt, nsteps):
    A, B, c = O.lsrk_coeffs()
    y, t = y0, t0
    for _ in range(nsteps):
        g = 0.0
        for k in range(5):
            g = A[k] * g + dt * f(t + c[k] * dt, y)
            y = y + B[k] * g
        t = t + dt
    return y


def test_stage_times_and_quadrature_exactness():
    A, B, c = O.lsrk_coeffs()
    assert A[0] == 0.0 and c[0] == 0.0
    for deg in range(4):                     # y' = t^deg integrates exactly for deg <= 3
        y = lsrk(lambda t, y: t ** deg, 0.0, 0.3, 0.2, 1)
        exact = (0.5 ** (deg + 1) - 0.3 ** (deg + 1)) / (deg + 1)
        assert abs(y - exact) < 1e-15
    # degree 4 is not exact: the pin above really constrains the stage times
    y = lsrk(lambda t, y: t ** 4, 0.0, 0.3, 0.2, 1)
    assert abs(y - (0.5 ** 5 - 0.3 ** 5) / 5) > 1e-12


def test_fourth_order_on_linear_ode():
    lam = -1.3 + 0.7j
    errs = []
    for n in (8, 16, 32):
        y = lsrk(lambda t, y: lam * y, 1.0 + 0j, 0.0, 1.0 / n, n)
        errs.append(abs(y - np.exp(lam)))
    orders = [np.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert all(abs(o - 4.0) < 0.15 for o in orders), orders


@pytest.mark.parametrize("riemann", [synth.RUSANOV, synth.ROE_HH])
def test_orc_step_fourth_order_in_time(riemann):
    """Density polynomial in x (flow 3, cubic) advected at constant velocity: DGSEM is
    exact in space on it, so the error against the exact solution is the time error of
    orc_step alone (stage times, time-dependent boundary data and displacement included),
    which must fall as dt^4."""
    p = synth.config_poly_x(N=3, v=0.37)
    p.riemann, p.delta0 = riemann, 0.093
    p.fpar = (1.0, 0.3, -0.2, 0.15, 0.6, 0.2, -0.1, 1.0)
    o = O.Oracle(p)
    T, errs = 0.24, []
    for n in (6, 12, 24):
        U = o.init_state()
        G = np.zeros_like(U)
        t = o.step(U, G, 0.0, T / n, n)
        assert abs(t - T) < 1e-15
        errs.append(np.abs(U - o.exact_state(t)).max())
    orders = [np.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert all(abs(o_ - 4.0) < 0.2 for o_ in orders), (errs, orders)
