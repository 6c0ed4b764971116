"""Failure handling of the serving loop, with the failure made on the host (no GPU fault):

* a request whose initial data is not finite (a NaN density in its flow parameters) ends
  with SM_ERR_NONFINITE, while the solves stepped in the same batched launches (or beside it,
  when it runs outside the batch) complete with exactly the state they reach alone;
* malformed requests (degree outside 1..7, non-positive time step, a request that can never
  fit the memory budget) are refused at submission with their status, and the server keeps
  serving;
* checkpoint and resume (state and time through the C-ABI) continue a solve bit for bit.
"""
import copy

import numpy as np
import pytest

from paper_2008_04356_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SM_ERR_ARG, SM_ERR_OOM, SM_ERR_NONFINITE = -1, -2, -4


@pytest.fixture(scope="module")
def sm():
    from paper_2008_04356_gb300 import build, slidemesh
    assert torch.cuda.is_available(), "the gpu tests need a CUDA device"
    build.build_library()
    slidemesh.lib()
    return slidemesh


def requests():
    reqs = []
    for k, (N, kk, v) in enumerate(((3, 4, 0.5), (5, 3, 0.8), (3, 6, 0.3))):
        p = synth.config_box(N=N, k=kk, v=v, precision=synth.FP32)
        p.delta0 = 0.1 * k
        reqs.append((p, synth.cfl_dt(p), 6 + 3 * k))
    return reqs


def test_nonfinite_request_is_isolated(sm):
    reqs = requests()
    bad = copy.deepcopy(reqs[0][0])
    bad.fpar = (float("nan"),) + tuple(bad.fpar[1:])      # NaN density in the initial data
    srv = sm.Server(hbm_budget_bytes=4 << 30, max_slots=8)
    tickets = [srv.submit(p, dt, n, keep_state=True) for p, dt, n in reqs]
    tbad = srv.submit(bad, reqs[0][1], reqs[0][2])
    srv.wait(300)
    res = [srv.poll(t) for t in tickets]
    rbad = srv.poll(tbad)
    st = srv.stats()
    srv.close()
    assert rbad["status"] == SM_ERR_NONFINITE
    assert all(r["status"] == 0 for r in res)
    assert st["completed"] + st["failed"] == len(reqs) + 1 and st["failed"] >= 1
    for (p, dt, n), r in zip(reqs, res):
        alone = sm.Server(hbm_budget_bytes=4 << 30, max_slots=1)
        t = alone.submit(p, dt, n, keep_state=True)
        alone.wait(120)
        ra = alone.poll(t)
        alone.close()
        assert ra["state"] == r["state"]                   # bit for bit
        assert np.all(np.isfinite(np.frombuffer(r["state"], dtype=np.float32)))


def test_nonfinite_solo_request_is_isolated(sm):
    """The same for a request outside the batch (FP64, on a stream of its own): its NaN ends
    it with SM_ERR_NONFINITE and the batched FP32 solves beside it are unaffected."""
    reqs = requests()
    bad = synth.config_box(N=3)                               # FP64
    dt_bad = synth.cfl_dt(bad)
    bad.fpar = (float("nan"),) + tuple(bad.fpar[1:])
    srv = sm.Server(hbm_budget_bytes=4 << 30, max_slots=8)
    tbad = srv.submit(bad, dt_bad, 12)
    tickets = [srv.submit(p, dt, n, keep_state=True) for p, dt, n in reqs]
    srv.wait(300)
    rbad = srv.poll(tbad)
    res = [srv.poll(t) for t in tickets]
    srv.close()
    assert rbad["status"] == SM_ERR_NONFINITE
    assert all(r["status"] == 0 for r in res)
    for (p, dt, n), r in zip(reqs, res):
        alone = sm.Server(hbm_budget_bytes=4 << 30, max_slots=1)
        t = alone.submit(p, dt, n, keep_state=True)
        alone.wait(120)
        ra = alone.poll(t)
        alone.close()
        assert ra["state"] == r["state"]                   # bit for bit


def test_malformed_requests_are_refused_and_serving_continues(sm):
    (p, dt, n), = requests()[:1]
    srv = sm.Server(hbm_budget_bytes=1 << 30, max_slots=2)
    q = copy.deepcopy(p)
    q.N = 9
    with pytest.raises(sm.SlidemeshError) as ei:
        srv.submit(q, dt, n)
    assert ei.value.status == SM_ERR_ARG
    with pytest.raises(sm.SlidemeshError) as ei:
        srv.submit(p, 0.0, n)
    assert ei.value.status == SM_ERR_ARG
    big = synth.config_interface_heavy(seed=1, precision=synth.FP32)
    with pytest.raises(sm.SlidemeshError) as ei:
        srv.submit(big, 1e-4, 1)                            # never fits 1 GiB
    assert ei.value.status == SM_ERR_OOM
    t = srv.submit(p, dt, n)
    srv.wait(120)
    r = srv.poll(t)
    srv.close()
    assert r["status"] == 0


@pytest.mark.parametrize("prec", [synth.FP64, synth.FP32])
def test_checkpoint_resume_is_bit_exact(sm, prec):
    """A solve checkpointed with sm_get_state after 3 steps and resumed in a new solver with
    sm_set_state (state and time; the RK register restarts every step) continues bit for bit
    like the uninterrupted solve."""
    p = synth.config_box(N=3, v=0.43, precision=prec)
    p.delta0 = 0.21
    dt = synth.cfl_dt(p)
    a = sm.Solver(p)
    a.init_state()
    a.step(dt, 7)
    ua, ta = a.get_state()
    b = sm.Solver(p)
    b.init_state()
    b.step(dt, 3)
    ub, tb = b.get_state()
    ck = (ub.cpu().clone(), tb)
    b.close()
    c = sm.Solver(p)
    c.set_state(ck[0].numpy(), ck[1])
    c.step(dt, 4)
    uc, tc = c.get_state()
    assert tc == ta
    assert torch.equal(uc.cpu(), ua.cpu())
    a.close()
    c.close()
