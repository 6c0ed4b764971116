"""Pins of the oracle's split form on curved elements (Sec. 3.1, the split formulation with
Pirozzoli's flux, on the curvilinear geometries): the contravariant two-point flux takes
Pirozzoli's products with the averaged metric vector {{Ja^d}} of its two nodes and the
averaged normal grid speed {{Ja^d . v^g}}.

* the plane box through general metrics gives the Cartesian split form (pinned separately);
* with the central two-point flux {{Ja . F - (Ja . v^g) U}} the curved split form is the
  curved weak form (summation by parts of the LGL derivative), on all rotating shapes;
* a state at rest stays at rest on the conforming cylinder (metric identities);
* mass and energy totals of the residual vanish on the closed rotating geometries;
* rigid rotation: the residual converges spectrally to the mesh-following derivative.
"""
import copy

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
