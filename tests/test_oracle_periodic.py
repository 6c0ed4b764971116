"""Pins of the oracle with two sliding interfaces (several interfaces, Sec. 4.3: the
interface is the outermost key of the mortar ordering).  With x periodic the moving block's
face x = x2 meets the static block's face x = x0 in a second plane sliding interface, with
the same displacement as the first; the domain is closed (periodic in x, y and z).

* discrete conservation: the totals of the residual vanish (no boundary flux), for the weak
  and the split volume integral, any displacement;
* the mortar flux sums of each interface cancel between its two sides;
* zero displacement reproduces the fully periodic conforming mesh bit for bit;
* free-stream preservation over 100 steps;
* order N+1 convergence for the translating entropy wave, which is periodic in x.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2008_04356_gb300 import synth


def periodic_box(N=3, k=None, v=0.5, delta0=0.2121, riemann=synth.RUSANOV, volume=synth.VOLUME_WEAK,
                 flow="wave"):
    p = synth.config_box(N=N, k=k, v=v, riemann=riemann, flow=flow)
    p.delta0, p.volume, p.periodic_x = delta0, volume, 1
    return p


@pytest.mark.parametrize("volume", [synth.VOLUME_WEAK, synth.VOLUME_SPLIT])
@pytest.mark.parametrize("riemann", [synth.RUSANOV, synth.ROE_HH])
@pytest.mark.parametrize("delta0", [0.0, 0.2121, 1.37, -0.61])
def test_closed_domain_conserves_totals(delta0, riemann, volume):
    p = periodic_box(N=3, delta0=delta0, riemann=riemann, volume=volume)
    o = O.Oracle(p)
    U = synth.random_state(p, seed=41)
    Ut = o.rhs(U, 0.07)
    tot = o.totals(Ut)
    assert np.abs(tot).max() < 1e-13 * np.abs(Ut).max()
    assert np.abs(Ut).max() > 1.0            # the residual itself is not small


@pytest.mark.parametrize("riemann", [synth.RUSANOV, synth.ROE_HH])
def test_both_interfaces_flux_sums_cancel(riemann):
    p = periodic_box(N=4, delta0=0.3337, riemann=riemann)
    o = O.Oracle(p)
    U = synth.random_state(p, seed=9)
    Fs, Fm = o.interface_fluxes(U, 0.0)
    assert Fs.shape[0] == 2
    for k in range(2):
        ss, sm = o.face_flux_sums(Fs[k], Fm[k])
        assert np.all(np.abs(ss + sm) < 1e-13 * max(1.0, np.abs(Fs[k]).sum() / Fs[k].size * 8))
        assert np.abs(ss).max() > 1e-3
    # the two interfaces see different traces: their fluxes differ
    assert np.abs(Fs[0] - Fs[1]).max() > 1e-3


@pytest.mark.parametrize("volume", [synth.VOLUME_WEAK, synth.VOLUME_SPLIT])
@pytest.mark.parametrize("riemann", [synth.RUSANOV, synth.ROE_HH])
def test_zero_displacement_is_fully_periodic_conforming_mesh(riemann, volume):
    p = periodic_box(N=3, v=0.0, delta0=0.0, riemann=riemann, volume=volume)
    U = synth.random_state(p, seed=5)
    Ut_slide = O.Oracle(p).rhs(U, 0.2)
    p.interface_conforming = 1
    assert np.array_equal(Ut_slide, O.Oracle(p).rhs(U, 0.2))


@pytest.mark.parametrize("N", [1, 3, 5])
def test_free_stream_preserved_two_interfaces(N):
    p = periodic_box(N=N, v=0.37, delta0=0.011, flow="free", riemann=synth.ROE_HH)
    o = O.Oracle(p)
    U = o.init_state()
    U0 = U.copy()
    G2 = np.zeros_like(U)
    o.step(U, G2, 0.0, synth.cfl_dt(p), 100)
    assert np.abs(U - U0).max() < 1e-13


def _wave_error(N, k, T, riemann, volume):
    p = periodic_box(N=N, k=k, v=0.5, delta0=0.0, riemann=riemann, volume=volume)
    o = O.Oracle(p)
    U = o.init_state()
    G2 = np.zeros_like(U)
    dt = min(synth.cfl_dt(p), 0.1 * (1.0 / k) ** ((N + 1) / 4.0))
    nsteps = int(np.ceil(T / dt))
    t = o.step(U, G2, 0.0, T / nsteps, nsteps)
    return o.l2_error_rho(U, t)


@pytest.mark.parametrize("volume", [synth.VOLUME_WEAK, synth.VOLUME_SPLIT])
def test_convergence_order_two_interfaces(volume):
    errs = [_wave_error(3, k, 0.21, synth.ROE_HH, volume) for k in (4, 8)]
    order = np.log2(errs[0] / errs[1])
    assert order > 3.5, (errs, order)
