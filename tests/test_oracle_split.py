"""Pins of the oracle's split-form volume integral (Sec. 3.1: the split formulation with
Pirozzoli's flux, used with Roe's solver and the Harten-Hyman fix for all of the paper's
computations).

* the two-point flux is consistent with the ALE flux of Sec. 2 (Eq. fluxes_written_out)
  and symmetric in its two states;
* its momentum part meets the kinetic-energy-preservation condition
  F#_m = {{v}} F#_rho + {{p}} n, and the assembled operator preserves the kinetic energy
  of a face-continuous state at constant pressure on the fully periodic box (the central
  flux does not);
* with the central two-point flux the split form is the weak form (summation by parts of
  the LGL derivative), which the weak-form pins already fix;
* for an entropy wave (constant velocity and pressure) the mass and momentum fluxes are
  linear in the state, so those components equal the weak form's, the energy does not;
* free-stream preservation and discrete conservation on the sliding mesh;
* zero displacement reproduces the conforming mesh bit for bit;
* order N+1 convergence for the translating entropy wave.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2008_04356_gb300 import synth

G = 1.4


def _random_states(seed, count):
    rng = np.random.default_rng(seed)
    rho = rng.uniform(0.6, 1.6, count)
    vel = rng.uniform(-0.7, 0.7, (count, 3))
    p = rng.uniform(0.5, 1.5, count)
    E = p / (G - 1) + 0.5 * rho * (vel ** 2).sum(1)
    return np.column_stack([rho, rho[:, None] * vel, E])


def _prims(U):
    rho = U[0]
    v = U[1:4] / rho
    p = (G - 1) * (U[4] - 0.5 * rho * v @ v)
    return rho, v, p


NORMALS = [np.array([1.0, 0.0, 0.0]), np.array([0.0, 1.0, 0.0]), np.array([0.0, 0.0, 1.0]),
           np.array([0.6, -0.48, 0.64])]


@pytest.mark.parametrize("kind", [0, 1])
def test_two_point_flux_consistent_with_ale_flux(kind):
    S = _random_states(1, 40)
    for k, U in enumerate(S):
        n = NORMALS[k % 4]
        vgn = 0.37 * (k % 3 - 1)
        F2 = O.two_point_flux(kind, U, U, n, vgn, G)
        F = O.euler_flux(U, n, vgn, G)
        assert np.allclose(F2, F, rtol=1e-14, atol=1e-14)


@pytest.mark.parametrize("kind", [0, 1])
def test_two_point_flux_symmetric(kind):
    S = _random_states(2, 40)
    for k in range(0, 40, 2):
        n, vgn = NORMALS[k % 4], 0.21
        assert np.array_equal(O.two_point_flux(kind, S[k], S[k + 1], n, vgn, G),
                              O.two_point_flux(kind, S[k + 1], S[k], n, vgn, G))


def test_pirozzoli_flux_kinetic_energy_condition():
    S = _random_states(3, 40)
    for k in range(0, 40, 2):
        n, vgn = NORMALS[k % 4], -0.3 + 0.03 * k
        F = O.two_point_flux(0, S[k], S[k + 1], n, vgn, G)
        (_, vL, pL), (_, vR, pR) = _prims(S[k]), _prims(S[k + 1])
        vm, pm = 0.5 * (vL + vR), 0.5 * (pL + pR)
        assert np.allclose(F[1:4], vm * F[0] + pm * n, rtol=0, atol=1e-14)
        # the central flux does not meet it: the condition is a property of this flux
        Fc = O.two_point_flux(1, S[k], S[k + 1], n, vgn, G)
        assert np.abs(Fc[1:4] - (vm * Fc[0] + pm * n)).max() > 1e-6


def _periodic_smooth_state(o, seed):
    """A state continuous across every face of the fully periodic box (x closed through the
    second interface, the conforming instant), with constant pressure: smooth periodic
    density and velocity with random wave numbers and phases, evaluated at the nodes."""
    X = o.coords(0.0)
    x, y, z = X[:, 0], X[:, 1], X[:, 2]
    rng = np.random.default_rng(seed)

    def field(amp):
        f = np.zeros_like(x)
        for _ in range(4):
            kx, ky, kz = rng.integers(1, 3), rng.integers(-2, 3), rng.integers(-2, 3)
            f += amp * rng.uniform(0.3, 1.0) * np.sin(np.pi * kx * x + 2 * np.pi * ky * y + 2 * np.pi * kz * z
                                                       + rng.uniform(0, 2 * np.pi))
        return f

    rho = 1.0 + field(0.1)
    u, v, w = field(0.2), field(0.2), field(0.2)
    U = np.stack([rho, rho * u, rho * v, rho * w, 1.0 / (G - 1) + 0.5 * rho * (u * u + v * v + w * w)], axis=1)
    return U, (u, v, w)


@pytest.mark.parametrize("riemann", [synth.RUSANOV, synth.ROE_HH])
@pytest.mark.parametrize("N", [1, 2, 3, 4, 5, 6, 7])
def test_split_form_preserves_kinetic_energy(N, riemann):
    """Kinetic-energy preservation of the assembled split-form operator (the reason for
    Pirozzoli's split, Sec. 3.1): on a fully periodic box with a state that is continuous
    across every face (so every Riemann solver returns the central flux) and constant
    pressure, the semi-discrete kinetic-energy rate sum J w (v . dm/dt - |v|^2/2 drho/dt)
    vanishes to rounding.  The central two-point flux (the weak form) does not preserve it
    on the same state, so the check can tell the two apart."""
    rates = {}
    for vol in (synth.VOLUME_SPLIT, 2):
        p = synth.config_box(N=N, v=0.5, riemann=riemann)
        p.periodic_x, p.volume, p.delta0 = 1, vol, 0.0
        o = O.Oracle(p)
        U, (u, v, w) = _periodic_smooth_state(o, 10 + N)
        Ut = o.rhs(U, 0.0)
        xg, wg = O.lgl(N)
        W = (wg[None, None, :] * wg[None, :, None] * wg[:, None, None]).reshape(-1)
        Es = p.nel_s[0] * p.nel_s[1] * p.nel_s[2]
        hx = np.where(np.arange(p.nelem) < Es, (p.x1 - p.x0) / p.nel_s[0], (p.x2 - p.x1) / p.nel_m[0])
        J = hx * (p.y1 - p.y0) / p.nel_s[1] * (p.z1 - p.z0) / p.nel_s[2] / 8.0
        terms = (J[:, None] * W[None, :]) * (u * Ut[:, 1] + v * Ut[:, 2] + w * Ut[:, 3]
                                             - 0.5 * (u * u + v * v + w * w) * Ut[:, 0])
        rates[vol] = abs(terms.sum()) / np.abs(terms).sum()
    assert rates[synth.VOLUME_SPLIT] < 1e-13
    assert rates[2] > 1e-7


@pytest.mark.parametrize("riemann", [synth.RUSANOV, synth.ROE_HH])
@pytest.mark.parametrize("N", [1, 2, 3, 5])
def test_central_split_form_is_the_weak_form(N, riemann):
    p = synth.config_box(N=N)
    p.delta0, p.riemann = 0.2121, riemann
    U = synth.random_state(p, seed=N + 10)
    weak = O.Oracle(p).rhs(U, 0.13)
    p.volume = 2
    split_central = O.Oracle(p).rhs(U, 0.13)
    assert np.abs(split_central - weak).max() < 1e-13 * np.abs(weak).max()


@pytest.mark.parametrize("N", [2, 4])
def test_split_form_of_an_entropy_wave(N):
    """u and p constant: the mass and momentum two-point fluxes are linear in the state
    (central), the energy flux {{rho}}{{w}}{{H}} is not."""
    p = synth.config_box(N=N, v=0.43)
    p.delta0 = 0.071
    o = O.Oracle(p)
    U = o.init_state()
    weak = o.rhs(U, 0.0)
    p.volume = synth.VOLUME_SPLIT
    split = O.Oracle(p).rhs(U, 0.0)
    scale = np.abs(weak).max()
    # rounding only: the residual is a small difference of flux terms about 10x larger
    assert np.abs(split[:, 0:4] - weak[:, 0:4]).max() < 1e-12 * scale
    assert np.abs(split[:, 4] - weak[:, 4]).max() > 1e-6 * scale


@pytest.mark.parametrize("N", [1, 3, 5, 7])
def test_split_free_stream_preserved(N):
    p = synth.config_box(N=N, flow="free", v=0.37)
    p.delta0, p.volume, p.riemann = 0.011, synth.VOLUME_SPLIT, synth.ROE_HH
    o = O.Oracle(p)
    U = o.init_state()
    U0 = U.copy()
    G2 = np.zeros_like(U)
    o.step(U, G2, 0.0, synth.cfl_dt(p), 100)
    assert np.abs(U - U0).max() < 1e-13


@pytest.mark.parametrize("riemann", [synth.RUSANOV, synth.ROE_HH])
def test_split_zero_displacement_is_conforming_mesh(riemann):
    p = synth.config_box(N=3, v=0.0)
    p.riemann, p.volume = riemann, synth.VOLUME_SPLIT
    U = synth.random_state(p, seed=5)
    Ut_slide = O.Oracle(p).rhs(U, 0.2)
    p.interface_conforming = 1
    assert np.array_equal(Ut_slide, O.Oracle(p).rhs(U, 0.2))


def test_split_total_residual_equals_boundary_flux():
    """The two-point volume terms telescope: the totals change only through the weak
    Dirichlet faces x = 0 and x = 2 (conforming and mortar faces cancel)."""
    p = synth.config_box(N=3)
    p.flow, p.fpar, p.delta0 = synth.FLOW_MODES, (1.0, 0.1, 0.0, 0.0, 1.0), 0.2121
    p.volume = synth.VOLUME_SPLIT
    o = O.Oracle(p)
    U = synth.random_state(p, seed=21)
    tot = o.totals(o.rhs(U, 0.0))
    x, w = O.lgl(3)
    np_, ny, nz = 4, 4, 2
    sJ = 0.25 * 0.5 / 4
    rho, u, pr = 1.0, np.array([0.1, 0.0, 0.0]), 1.0
    bg = np.array([rho, rho * u[0], 0.0, 0.0, pr / (G - 1) + 0.5 * rho * u @ u])
    n = np.array([1.0, 0.0, 0.0])
    bflux = np.zeros(5)
    for iz in range(nz):
        for iy in range(ny):
            for blk, ix, k, left in ((0, 0, 0, True), (1, 3, 3, False)):
                e = blk * 32 + ix + 4 * (iy + ny * iz)
                for j in range(np_):
                    for i in range(np_):
                        uin = U[e, :, i + np_ * (j + np_ * k)]
                        f = -O.riemann(0, bg, uin, n, 0.0, G) if left else O.riemann(0, uin, bg, n, 0.0, G)
                        bflux += w[i] * w[j] * sJ * f
    assert np.allclose(tot, -bflux, atol=1e-13)


def _wave_error(N, k, T, riemann):
    p = synth.config_box(N=N, k=k, v=0.5, riemann=riemann)
    p.volume = synth.VOLUME_SPLIT
    o = O.Oracle(p)
    U = o.init_state()
    G2 = np.zeros_like(U)
    dt = min(synth.cfl_dt(p), 0.1 * (1.0 / k) ** ((N + 1) / 4.0))
    nsteps = int(np.ceil(T / dt))
    t = o.step(U, G2, 0.0, T / nsteps, nsteps)
    return o.l2_error_rho(U, t)


def test_split_convergence_order_entropy_wave():
    errs = [_wave_error(3, k, 0.21, synth.ROE_HH) for k in (4, 8)]
    order = np.log2(errs[0] / errs[1])
    assert order > 3.5, (errs, order)
