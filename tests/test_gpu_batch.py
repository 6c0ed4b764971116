"""Batched stepping and the serving loop on the GPU.

* batched FP32 steps agree with the same solves stepped one at a time (FP32 tolerance,
  1e-5 relative L2) and with the FP64 oracle;
* a solve's result does not depend on the batch it is in, nor on the launch shapes the
  autotuner picks (the same kernels do the same arithmetic per element): bit for bit;
* the server admits by slots and HBM budget, overlaps solves, and each result is the same
  alone and in the mix.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2008_04356_gb300 import synth

import fp32_steps as F

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FP32_TOL = 1e-5


@pytest.fixture(scope="module")
def sm():
    from paper_2008_04356_gb300 import build, slidemesh
    assert torch.cuda.is_available(), "the gpu tests need a CUDA device"
    build.build_library()
    slidemesh.lib()
    return slidemesh


def rel_l2(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def problems():
    a = synth.config_box(N=3, precision=synth.FP32)
    b = synth.config_box(N=5, v=0.37, precision=synth.FP32, riemann=synth.ROE_HH)
    b.nel_s, b.nel_m, b.x2, b.delta0 = (2, 11, 3), (3, 11, 3), 2.3, 0.41
    c = synth.config_box(N=3, k=4, v=-0.8, precision=synth.FP32)
    c.delta0 = -0.137
    d = synth.config_interface_heavy(seed=4, precision=synth.FP32, nz=4, ny=16, nx=2, N=3)
    return [a, b, c, d]


def fresh(sm, p):
    s = sm.Solver(p)
    s.init_state()
    return s


def test_batch_matches_one_at_a_time_and_oracle(sm):
    """Batched steps from perturbed initial states (fp32_steps): the same as each solve
    stepped alone, and every solve's increment against the FP64 oracle at 1e-5."""
    ps = problems()
    dts = [synth.cfl_dt(p) for p in ps]
    oracles = [O.Oracle(p) for p in ps]
    U0s = [F.perturbed(o.init_state(), seed=140 + k) for k, o in enumerate(oracles)]
    batched = []
    for p, U0 in zip(ps, U0s):
        s = sm.Solver(p)
        s.set_state(U0.astype(np.float32), 0.0)
        batched.append(s)
    bt = sm.Batch(batched, dts)
    bt.step(3)
    bt.step(4)
    for p, dt, s, o, U0 in zip(ps, dts, batched, oracles, U0s):
        alone = sm.Solver(p)
        alone.set_state(U0.astype(np.float32), 0.0)
        alone.step(dt, 7)
        ub, tb = s.get_state()
        ua, ta = alone.get_state()
        assert abs(tb - ta) < 1e-15
        assert rel_l2(ub.cpu().numpy(), ua.cpu().numpy()) < FP32_TOL
        Uo, Go = U0.copy(), np.zeros_like(U0)
        o.step(Uo, Go, 0.0, dt, 7)
        err = F.increment_error(U0, ub.cpu().numpy(), Uo)
        print("N=%d: batched increment rel L2 %.2e" % (p.N, err))
        assert err < F.INCREMENT_TOL


def test_result_independent_of_batch_and_launch_shapes(sm):
    ps = problems()
    dts = [synth.cfl_dt(p) for p in ps]
    alone = fresh(sm, ps[1])
    b1 = sm.Batch([alone], [dts[1]])
    b1.step(5)
    mix = [fresh(sm, p) for p in ps]
    b2 = sm.Batch(mix, dts)
    b2.autotune()
    shapes = b2.shapes()
    assert {s["N"] for s in shapes} == {3, 5}
    b2.step(5)
    ua, _ = alone.get_state()
    um, _ = mix[1].get_state()
    assert torch.equal(ua, um)


def _stream(seed=0, n=8):
    rng = np.random.default_rng(seed)
    reqs = []
    for k in range(n):
        N = int(rng.choice([3, 5]))
        kk = int(rng.choice([3, 4, 6]))
        p = synth.config_box(N=N, k=kk, v=float(rng.uniform(0.1, 1.0)), precision=synth.FP32)
        p.delta0 = float(rng.uniform(-0.5, 0.5))
        reqs.append((p, synth.cfl_dt(p), int(rng.integers(5, 25))))
    return reqs


def test_server_results_same_alone_and_in_the_mix(sm):
    reqs = _stream(seed=1)
    srv = sm.Server(hbm_budget_bytes=8 << 30, max_slots=16)
    tickets = [srv.submit(p, dt, n, keep_state=True) for p, dt, n in reqs]
    srv.wait(300)
    mixed = [srv.poll(t) for t in tickets]
    st = srv.stats()
    srv.close()
    assert all(r["status"] == 0 for r in mixed)
    assert st["completed"] == len(reqs) and st["max_concurrent"] > 1
    for (p, dt, n), r in zip(reqs, mixed):
        alone_srv = sm.Server(hbm_budget_bytes=8 << 30, max_slots=1)
        t = alone_srv.submit(p, dt, n, keep_state=True)
        alone_srv.wait(120)
        ra = alone_srv.poll(t)
        alone_srv.close()
        assert ra["state"] == r["state"]                 # bit for bit
        assert abs(ra["sim_time"] - n * dt) < 1e-12
        # and the one-solve path
        s = fresh(sm, p)
        s.step(dt, n)
        u1, _ = s.get_state()
        um = np.frombuffer(r["state"], dtype=np.float32)
        assert rel_l2(um, u1.cpu().numpy().ravel()) < FP32_TOL


def test_server_admission_by_budget_and_slots(sm):
    reqs = _stream(seed=2, n=6)
    need = max(3 * p.ndof * 5 * 4 for p, _, _ in reqs)
    budget = int(2.2 * need) + (1 << 21)
    srv = sm.Server(hbm_budget_bytes=budget, max_slots=3)
    for p, dt, n in reqs:
        srv.submit(p, dt, n)
    srv.wait(300)
    st = srv.stats()
    assert st["completed"] == 6 and st["failed"] == 0
    assert st["peak_bytes"] <= budget and st["max_concurrent"] <= 3
    big = synth.config_interface_heavy(seed=1, precision=synth.FP32)
    with pytest.raises(sm.SlidemeshError):
        srv.submit(big, 1e-4, 1)                          # could never fit this budget
    srv.close()


def test_server_fp64_requests_match_sm_step(sm):
    p = synth.config_box(N=3)
    dt = synth.cfl_dt(p)
    srv = sm.Server(hbm_budget_bytes=4 << 30, max_slots=4)
    t = srv.submit(p, dt, 9, keep_state=True)
    srv.wait(120)
    r = srv.poll(t)
    srv.close()
    s = fresh(sm, p)
    s.step(dt, 9)
    u, _ = s.get_state()
    assert np.frombuffer(r["state"], dtype=np.float64).tobytes() == u.cpu().numpy().tobytes()


def test_server_runs_slow_solves_beside_the_batch(sm):
    """FP64 requests step on streams of their own, beside the FP32 batch: every result is
    the one-solve result bit for bit, and short FP32 requests submitted together with a long
    FP64 one finish before it."""
    long_p = synth.config_box(N=5, k=6)                      # FP64, 2 x 6^3 elements
    long_dt, long_n = synth.cfl_dt(long_p), 400
    short = _stream(seed=3, n=4)
    srv = sm.Server(hbm_budget_bytes=8 << 30, max_slots=8)
    t_long = srv.submit(long_p, long_dt, long_n, keep_state=True)
    t_short = [srv.submit(p, dt, n, keep_state=True) for p, dt, n in short]
    srv.wait(300)
    r_long = srv.poll(t_long)
    r_short = [srv.poll(t) for t in t_short]
    srv.close()
    assert r_long["status"] == 0 and all(r["status"] == 0 for r in r_short)
    assert r_long["steps"] == long_n
    assert max(r["t_done"] for r in r_short) < r_long["t_done"]
    s = fresh(sm, long_p)
    s.step(long_dt, long_n)
    u, _ = s.get_state()
    assert np.frombuffer(r_long["state"], dtype=np.float64).tobytes() == u.cpu().numpy().tobytes()
    for (p, dt, n), r in zip(short, r_short):
        alone = sm.Server(hbm_budget_bytes=8 << 30, max_slots=1)
        t = alone.submit(p, dt, n, keep_state=True)
        alone.wait(120)
        ra = alone.poll(t)
        alone.close()
        assert ra["state"] == r["state"]
