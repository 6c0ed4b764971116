"""The exactness and convergence sweep through the CUDA path: the box [0,2] x [0,1]^2 split
at x = 1 by the plane sliding interface, the right block moving along +y at v = 0.5, N = 1..7
and k^3 elements per block (k = 4 .. 32).

* Free stream (rho = 1, u = (0.5, 0.2, 0.1), p = 1) is kept to 1e-13 (FP64) / 1e-5 (FP32)
  over 10 steps on every mesh (Sec. 3.3: plane interfaces preserve it), the interface
  fluxes of both sides cancel (discrete conservation of the mortar projection, Sec. 3.2),
  and the conserved totals do not drift.
* The translating entropy wave converges at order N + 1 in FP64 (errors measured against
  the closed-form solution, dt small enough that the time error is negligible), and the FP32
  path follows the same errors down to its precision floor.
* FP32 against the FP64 oracle on the sweep meshes (k = 4, 8): step increments from
  perturbed states at 1e-5 relative L2 (fp32_steps).

Errors and orders are printed (pytest -s) for the record.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2008_04356_gb300 import synth

import fp32_steps as F

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

T_END = 0.21         # v T / l = 0.105 k: the moving block never ends on a whole face
KS = {1: (4, 8, 16, 32), 2: (4, 8, 16, 32), 3: (4, 8, 16, 32), 4: (4, 8, 16), 5: (4, 8, 16), 6: (4, 8, 16),
      7: (4, 8, 16)}


@pytest.fixture(scope="module")
def sm():
    from paper_2008_04356_gb300 import build, slidemesh
    assert torch.cuda.is_available(), "the gpu tests need a CUDA device"
    build.build_library()
    slidemesh.lib()
    return slidemesh


@pytest.mark.parametrize("N", range(1, 8))
def test_free_stream_and_conservation_sweep(sm, N):
    for k in (4, 8, 16, 32):
        for prec, tol in ((synth.FP64, 1e-13), (synth.FP32, 1e-5)):
            p = synth.config_box(N=N, k=k, flow="free", v=0.5, precision=prec)
            p.delta0 = 0.0137
            sol = sm.Solver(p)
            sol.init_state()
            U0, _ = sol.get_state()
            U0 = U0.clone()
            tot0 = np.array(sol.diag()["totals"])
            sol.step(synth.cfl_dt(p), 10)
            U1, _ = sol.get_state()
            d = sol.diag()
            sol.close()
            dev = (U1 - U0).abs().max().item()
            ss, sm_ = np.array(d["iface_sum_static"]), np.array(d["iface_sum_moving"])
            drift = np.abs(np.array(d["totals"]) - tot0).max() / np.abs(tot0).max()
            print("N=%d k=%2d %s: free-stream deviation %.2e, interface sums %.2e, totals drift %.2e"
                  % (N, k, "fp64" if prec == synth.FP64 else "fp32", dev, np.abs(ss + sm_).max(), drift))
            assert dev < tol
            assert np.all(np.abs(ss + sm_) <= tol * (1.0 + np.abs(ss)))
            assert drift < (1e-13 if prec == synth.FP64 else 1e-6)


def wave_errors(sm, N, k, prec):
    """L2 error of the density against the closed-form entropy wave at T_END."""
    p = synth.config_box(N=N, k=k, v=0.5, precision=prec, riemann=synth.ROE_HH)
    h = 1.0 / k
    dt = min(synth.cfl_dt(p), 0.1 * h ** ((N + 1) / 4.0))
    nsteps = int(math.ceil(T_END / dt))
    dt = T_END / nsteps
    sol = sm.Solver(p)
    sol.init_state()
    sol.step(dt, nsteps)
    U, t = sol.get_state()
    sol.close()
    q = synth.config_box(N=N, k=k, v=0.5, riemann=synth.ROE_HH)
    return O.Oracle(q).l2_error_rho(U.double().cpu().numpy(), t)


@pytest.mark.parametrize("N", range(1, 8))
def test_convergence_order_sweep(sm, N):
    ks = KS[N]
    e64 = [wave_errors(sm, N, k, synth.FP64) for k in ks]
    e32 = [wave_errors(sm, N, k, synth.FP32) for k in ks]
    o64 = [math.log2(e64[i] / e64[i + 1]) for i in range(len(ks) - 1)]
    o32 = [math.log2(e32[i] / e32[i + 1]) for i in range(len(ks) - 1)]
    print("N=%d k=%s\n  fp64 L2 %s orders %s\n  fp32 L2 %s orders %s"
          % (N, ks, ["%.3e" % e for e in e64], ["%.2f" % o for o in o64],
             ["%.3e" % e for e in e32], ["%.2f" % o for o in o32]))
    # order N + 1 on the finest pair of meshes (to within half an order)
    assert o64[-1] > N + 1 - 0.5, (e64, o64)
    # the FP32 path has the FP64 path's error down to its precision floor: FP32 rounding of
    # the state over the finest meshes' 300 - 640 steps (5.5e-6 measured at N = 3, k = 32)
    for a, b in zip(e32, e64):
        assert a < 1.05 * b + 2e-5, (e32, e64)


@pytest.mark.parametrize("N", range(1, 8))
def test_fp32_increments_against_the_oracle_sweep(sm, N):
    for k in (4, 8):
        p = synth.config_box(N=N, k=k, v=0.5, precision=synth.FP32)
        o = O.Oracle(p)
        sol = sm.Solver(p)
        err = F.check_fp32_steps(sol, o, F.perturbed(o.init_state(), seed=300 + 10 * N + k), synth.cfl_dt(p), 3)
        sol.close()
        print("N=%d k=%d: FP32 increment rel L2 against the oracle %.2e" % (N, k, err))
