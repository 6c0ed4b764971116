"""sm_stream_jobs: independent jobs streamed from host memory through one solver, with the
host-to-device and device-to-host copies overlapping the steps.  Each job's result must be
bit-identical to sm_set_state + sm_step + sm_get_state on the same input (the same kernels
in the same order on the same values), whatever the number of jobs, with one reused input or
one per job, and with one reused output or one per job; the solver keeps the last job's
state and time."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2008_04356_gb300 import synth

import fp32_steps as F

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sm():
    from paper_2008_04356_gb300 import build, slidemesh
    assert torch.cuda.is_available(), "the gpu tests need a CUDA device"
    build.build_library()
    slidemesh.lib()
    return slidemesh


def job_inputs(p, sol, count, seed):
    """count distinct states (smooth field plus seeded noise) in pinned host memory."""
    U0 = O.Oracle(p).init_state()
    xs = [F.perturbed(U0, seed=seed + i, amp=0.05) for i in range(count)]
    host = torch.empty((count,) + tuple(sol.shape()), dtype=sol.torch_dtype).pin_memory()
    for i, x in enumerate(xs):
        host[i].copy_(torch.from_numpy(x.astype(sol.dtype_np)).reshape(tuple(sol.shape())))
    return host


def one_at_a_time(sol, host_in, t0, dt, nsteps):
    outs = []
    t = None
    for i in range(host_in.shape[0]):
        sol.set_state(host_in[i], t0)
        sol.step(dt, nsteps)
        U, t = sol.get_state(out=torch.empty_like(host_in[i]))
        outs.append(U.clone())
    return torch.stack(outs), t


@pytest.mark.parametrize("prec", [synth.FP32, synth.FP64])
@pytest.mark.parametrize("count", [1, 3])
def test_streamed_jobs_equal_one_at_a_time(sm, prec, count):
    p = synth.config_box(N=3, v=0.5, precision=prec)
    sol = sm.Solver(p)
    dt, nsteps, t0 = synth.cfl_dt(p), 2, 0.125
    host_in = job_inputs(p, sol, count, seed=900 + 10 * count + prec)
    ref, t_ref = one_at_a_time(sol, host_in, t0, dt, nsteps)
    out = torch.zeros_like(host_in).pin_memory()
    sol.stream_jobs(host_in, out, t0, dt, nsteps)
    for i in range(count):
        assert torch.equal(out[i], ref[i]), i
    U_last, t_last = sol.get_state(out=torch.empty_like(host_in[0]))
    assert torch.equal(U_last, ref[-1])
    assert t_last == t_ref
    sol.close()


def test_streamed_jobs_reuse_one_input_and_one_output(sm):
    """in_stride 0: every job starts from the same state; out_stride 0: each result overwrites
    the last.  Four jobs, each must reproduce the single run."""
    p = synth.config_box(N=5, v=0.5, precision=synth.FP32)
    sol = sm.Solver(p)
    dt, nsteps, t0 = synth.cfl_dt(p), 3, 0.0
    host_in = job_inputs(p, sol, 1, seed=950)
    ref, _ = one_at_a_time(sol, host_in, t0, dt, nsteps)
    out_all = torch.zeros((4,) + tuple(sol.shape()), dtype=sol.torch_dtype).pin_memory()
    sol.stream_jobs(host_in[0], out_all, t0, dt, nsteps, count=4)
    for i in range(4):
        assert torch.equal(out_all[i], ref[0]), i
    out_one = torch.zeros_like(host_in[0]).pin_memory()
    sol.stream_jobs(host_in[0], out_one, t0, dt, nsteps, count=4)
    assert torch.equal(out_one, ref[0])
    sol.close()


def test_streamed_jobs_match_the_oracle(sm):
    """The streamed FP32 steps against the FP64 oracle by increments (the FP32 step bar)."""
    p = synth.config_box(N=3, v=0.5, precision=synth.FP32)
    o = O.Oracle(p)
    sol = sm.Solver(p)
    dt, nsteps = synth.cfl_dt(p), 2
    U0 = F.perturbed(o.init_state(), seed=977)
    host_in = torch.from_numpy(U0.astype(np.float32)).reshape(tuple(sol.shape())).pin_memory()
    out = torch.zeros_like(host_in).pin_memory()
    sol.stream_jobs(host_in, out, 0.0, dt, nsteps, count=2)
    U = U0.copy()
    G = np.zeros_like(U)
    o.step(U, G, 0.0, dt, nsteps)
    err = F.increment_error(U0, out.double().numpy().reshape(U0.shape), U)
    assert err < F.INCREMENT_TOL, err
    sol.close()


def test_streamed_jobs_on_the_rotating_cylinder_with_navier_stokes(sm):
    """The same bit-equality on the curved, rotating, Navier-Stokes path (lifting kernels in
    every stage), two distinct jobs."""
    p = synth.config_cylinder(N=3, precision=synth.FP32, physics=synth.NAVIER_STOKES)
    sol = sm.Solver(p)
    dt, nsteps, t0 = synth.cfl_dt(p), 2, 0.0
    sol.init_state()
    U0, _ = sol.get_state(out=torch.empty(tuple(sol.shape()), dtype=sol.torch_dtype))
    host_in = torch.stack([U0, U0 * torch.tensor([1.0, 1.02, 1.0, 0.98, 1.01]).view(1, 5, 1)]).contiguous().pin_memory()
    ref, t_ref = one_at_a_time(sol, host_in, t0, dt, nsteps)
    out = torch.zeros_like(host_in).pin_memory()
    sol.stream_jobs(host_in, out, t0, dt, nsteps)
    assert torch.equal(out[0], ref[0]) and torch.equal(out[1], ref[1])
    assert not torch.equal(out[0], out[1])
    sol.close()
