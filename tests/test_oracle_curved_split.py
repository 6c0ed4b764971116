"""Pins of the oracle's split form on curved elements (Sec. 3.1, the split formulation with
Pirozzoli's flux, on the curvilinear geometries): the contravariant two-point flux takes
Pirozzoli's products with the averaged metric vector {{Ja^d}} of its two nodes and the
averaged normal grid speed {{Ja^d . v^g}}.

* the plane box through general metrics gives the Cartesian split form (pinned separately);
* with the central two-point flux {{Ja . F - (Ja . v^g) U}} the curved split form is the
  curved weak form (summation by parts of the LGL derivative), on all rotating shapes;
* a state at rest stays at rest on the conforming cylinder (metric identities);
* mass and energy totals of the residual vanish on the closed rotating geometries;
* rigid rotation: the residual converges spectrally to the mesh-following derivative;
* kinetic-energy preservation of the assembled operator (the property Pirozzoli's split is
  chosen for) on every rotating shape, rotor moving or not: see the test's docstring.
"""
import copy
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2008_04356_gb300 import synth


def shapes(N=3, omega=0.4, phi0=0.3, flow="pulse"):
    return {
        "cylinder": synth.config_cylinder(N=N, nel=(2, 8, 2), omega=omega, phi0=phi0, flow=flow),
        "annular": synth.config_annular(N=N, nel=(2, 8, 2), omega=omega, phi0=phi0, flow=flow if flow != "free" else "rest"),
        "cone": synth.config_cone(N=N, nel=(2, 8, 2), omega=omega, phi0=phi0, flow=flow if flow != "free" else "rest"),
    }


@pytest.mark.parametrize("riemann", [synth.RUSANOV, synth.ROE_HH])
@pytest.mark.parametrize("N", [2, 4])
def test_plane_through_metrics_equals_cartesian_split(N, riemann):
    p = synth.config_box(N=N, v=0.37, riemann=riemann)
    p.nel_s, p.nel_m, p.x2, p.delta0, p.volume = (2, 7, 3), (3, 7, 3), 2.3, 0.3337, synth.VOLUME_SPLIT
    U = synth.random_state(p, seed=N)
    a = O.Oracle(p).rhs(U, 0.11)
    q = copy.deepcopy(p)
    q.geom = synth.GEOM_PLANE_CURVILINEAR
    b = O.Oracle(q).rhs(U, 0.11)
    assert np.abs(a - b).max() < 1e-13 * np.abs(a).max()


@pytest.mark.parametrize("shape", ["cylinder", "annular", "cone"])
def test_central_curved_split_is_the_curved_weak_form(shape):
    p = shapes()[shape]
    U = synth.random_state(p, seed=5)
    weak = O.Oracle(p).rhs(U, 0.2)
    p.volume = 2
    central = O.Oracle(p).rhs(U, 0.2)
    assert np.abs(central - weak).max() < 1e-13 * np.abs(weak).max()
    p.volume = synth.VOLUME_SPLIT
    assert np.abs(O.Oracle(p).rhs(U, 0.2) - weak).max() > 1e-6 * np.abs(weak).max()


def test_curved_split_rest_state_on_the_conforming_cylinder():
    p = synth.config_cylinder(N=4, nel=(2, 8, 2), omega=0.0, flow="free")
    p.fpar, p.interface_conforming, p.volume = (1.0, 0.0, 0.0, 0.0, 1.0), 1, synth.VOLUME_SPLIT
    o = O.Oracle(p)
    assert np.abs(o.rhs(o.init_state(), 0.0)).max() < 1e-11


@pytest.mark.parametrize("shape", ["cylinder", "annular", "cone"])
def test_curved_split_conserves_mass_and_energy(shape):
    p = shapes()[shape]
    p.volume = synth.VOLUME_SPLIT
    o = O.Oracle(p)
    Ut = o.rhs(synth.random_state(p, seed=6), 0.1)
    tot, scale = o.totals(Ut), o.totals(np.abs(Ut))
    assert abs(tot[0]) < 1e-13 * scale[0] and abs(tot[4]) < 1e-13 * scale[4]


def test_curved_split_rigid_rotation_converges():
    errs = []
    for N in (2, 3, 4, 5):
        p = synth.config_cylinder(N=N, nel=(2, 8, 2), flow="rotation", omega=0.4, phi0=0.013)
        p.fpar, p.volume = (1.0, 1.0, 0.4), synth.VOLUME_SPLIT
        o = O.Oracle(p)
        U = o.exact_state(0.0)
        X = o.coords(0.0)
        ex = np.zeros_like(U)
        rot = slice(0, o.E // 2)
        ex[rot, 1] = -0.16 * X[rot, 0]
        ex[rot, 2] = -0.16 * X[rot, 1]
        errs.append(np.abs(o.rhs(U, 0.0) - ex).max())
    assert all(errs[k + 1] < 0.5 * errs[k] for k in range(3)), errs
    assert errs[-1] < 1e-5


def _ke_state(p, o, seed):
    """Density and velocity continuous across every face at the conforming instant, with
    constant pressure and a velocity that vanishes on every slip wall (so that the mirror
    state equals the state whatever the discrete wall normal): periodic in the sector angle
    (and in z on the cylinder), random wave numbers and phases."""
    X = o.coords(0.0)
    x, y, z = X[:, 0], X[:, 1], X[:, 2]
    r, th = np.hypot(x, y), np.arctan2(y, x)
    if p.geom == synth.GEOM_CYLINDER:
        wall, per = np.sin(math.pi * (r - p.x0) / (p.x2 - p.x0)), 2 * math.pi * z / (p.z1 - p.z0)
    elif p.geom == synth.GEOM_ANNULAR:
        wall = np.sin(math.pi * (r - p.z0) / (p.z1 - p.z0)) * np.sin(math.pi * (z - p.x0) / (p.x2 - p.x0))
        per = 0.0 * z
    else:
        sa, ca = math.sin(p.cone_angle), math.cos(p.cone_angle)
        s_, n_ = r * sa + z * ca, r * ca - z * sa
        wall = np.sin(math.pi * (s_ - p.z0) / (p.z1 - p.z0)) * np.sin(math.pi * (n_ - p.x0) / (p.x2 - p.x0))
        per = 0.0 * z
    rng = np.random.default_rng(seed)
    sector = p.y1 - p.y0

    def field(amp):
        f = np.zeros_like(x)
        for _ in range(3):
            kt, kz, kr = rng.integers(-2, 3), rng.integers(-2, 3), rng.integers(1, 3)
            f += amp * rng.uniform(0.3, 1.0) * np.sin(2 * math.pi * kt * th / sector + kz * per + kr * r
                                                       + rng.uniform(0, 2 * math.pi))
        return f

    rho = 1.0 + field(0.1)
    vr, vt, vz = wall * field(0.2), wall * field(0.2), wall * field(0.2)
    u, v, w = vr * np.cos(th) - vt * np.sin(th), vr * np.sin(th) + vt * np.cos(th), vz
    U = np.stack([rho, rho * u, rho * v, rho * w, 1.0 / (p.gamma - 1) + 0.5 * rho * (u * u + v * v + w * w)], axis=1)
    return U, (u, v, w)


@pytest.mark.parametrize("omega", [0.0, 0.4])
@pytest.mark.parametrize("N", [1, 2, 3, 5, 7])
@pytest.mark.parametrize("shape", ["cylinder", "annular", "cone"])
def test_curved_split_preserves_kinetic_energy(shape, N, omega):
    """With a face-continuous state at constant pressure whose velocity vanishes on the slip
    walls (every Riemann solver then returns the central flux), the semi-discrete
    kinetic-energy rate sum J w (v . dm/dt - |v|^2/2 drho/dt) of the curved split form
    vanishes to rounding, with the rotor at rest or turning (the ALE terms included).  The
    central two-point flux, i.e. the curved weak form, does not preserve it on the same
    state (checked where its defect is well above rounding, N <= 5)."""
    rates = {}
    for vol in (synth.VOLUME_SPLIT, 2):
        p = shapes(N=N, omega=omega, phi0=0.0, flow="free")[shape]
        p.volume, p.riemann = vol, synth.ROE_HH
        o = O.Oracle(p)
        U, (u, v, w) = _ke_state(p, o, seed=5 + N)
        Ut = o.rhs(U, 0.0)
        integrand = u * Ut[:, 1] + v * Ut[:, 2] + w * Ut[:, 3] - 0.5 * (u * u + v * v + w * w) * Ut[:, 0]
        F = np.zeros_like(Ut)
        F[:, 0], F[:, 1] = integrand, np.abs(integrand)
        t = o.totals(F)                  # quadrature sums of the integrand and of its magnitude
        rates[vol] = abs(t[0]) / t[1]
    assert rates[synth.VOLUME_SPLIT] < 1e-12
    if N <= 5:
        assert rates[2] > 1e-8
