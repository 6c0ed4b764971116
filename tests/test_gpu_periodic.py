"""GPU parity with two sliding interfaces (periodic x: the moving block's face x = x2 meets
the static block's face x = x0; several interfaces, Sec. 4.3) against the FP64 oracle,
through the C-ABI.  The GPU solves the second interface as the x-mirrored first one (traces
with the x-momentum negated, fluxes mirrored back); the oracle evaluates it directly in
canonical orientation.  Bars: FP64 1e-12 relative (max norm), FP32 1e-5 relative L2.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2008_04356_gb300 import synth

import fp32_steps as F

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12
FP32_TOL = 1e-5


@pytest.fixture(scope="module")
def sm():
    from paper_2008_04356_gb300 import build, slidemesh
    assert torch.cuda.is_available(), "the gpu tests need a CUDA device"
    build.build_library()
    slidemesh.lib()
    return slidemesh


def rel_max(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def rel_l2(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def to_dev(U, dtype):
    return torch.from_numpy(np.ascontiguousarray(U)).to(dtype).cuda()


def periodic_box(N, riemann, volume=synth.VOLUME_WEAK, ny=11, nz=3, nx=(2, 3), delta0=0.3337, v=0.37,
                 prec=synth.FP64, flow="wave"):
    p = synth.config_box(N=N, v=v, precision=prec, riemann=riemann, flow=flow)
    p.nel_s, p.nel_m = (nx[0], ny, nz), (nx[1], ny, nz)
    p.x2 = 2.3
    p.delta0, p.volume, p.periodic_x = delta0, volume, 1
    return p


@pytest.mark.parametrize("volume", [synth.VOLUME_WEAK, synth.VOLUME_SPLIT])
@pytest.mark.parametrize("riemann", [synth.RUSANOV, synth.ROE_HH])
@pytest.mark.parametrize("N", [1, 2, 3, 4, 5, 6, 7])
def test_periodic_rhs_fp64_random_state(sm, N, riemann, volume):
    p = periodic_box(N, riemann, volume)
    U = synth.random_state(p, seed=277 + N)
    ref = O.Oracle(p).rhs(U, 0.123)
    sol = sm.Solver(p)
    Ut = sol.rhs(to_dev(U, torch.float64), 0.123).cpu().numpy()
    sol.close()
    assert rel_max(Ut, ref) < FP64_TOL


def test_periodic_single_element_blocks(sm):
    """One element along x per block: each element carries both interfaces."""
    p = periodic_box(3, synth.ROE_HH, nx=(1, 1), delta0=1.61)
    U = synth.random_state(p, seed=3)
    ref = O.Oracle(p).rhs(U, 0.05)
    sol = sm.Solver(p)
    Ut = sol.rhs(to_dev(U, torch.float64), 0.05).cpu().numpy()
    sol.close()
    assert rel_max(Ut, ref) < FP64_TOL


@pytest.mark.parametrize("volume", [synth.VOLUME_WEAK, synth.VOLUME_SPLIT])
def test_periodic_rhs_fp32_vs_oracle(sm, volume):
    for N in (2, 3, 5, 7):
        p = periodic_box(N, synth.ROE_HH, volume, prec=synth.FP32)
        U = synth.random_state(p, seed=331 + N).astype(np.float32)
        ref = O.Oracle(p).rhs(U.astype(np.float64), 0.3)
        sol = sm.Solver(p)
        Ut = sol.rhs(to_dev(U, torch.float32), 0.3).cpu().numpy()
        sol.close()
        assert rel_l2(Ut, ref) < FP32_TOL, N


@pytest.mark.parametrize("volume", [synth.VOLUME_WEAK, synth.VOLUME_SPLIT])
@pytest.mark.parametrize("N", [3, 4])
def test_periodic_step_fp64_with_rhs_between(sm, N, volume):
    """Steps through the compact traces of both interfaces (written by the element kernel),
    with an sm_rhs call of another state in between (it overwrites the second interface's
    traces, which the next step gathers again)."""
    p = periodic_box(N, synth.ROE_HH, volume, delta0=0.91)
    o = O.Oracle(p)
    U0 = o.init_state()
    dt = synth.cfl_dt(p)
    Uo, Go = U0.copy(), np.zeros_like(U0)
    t_ref = o.step(Uo, Go, 0.0, dt, 7)
    sol = sm.Solver(p)
    sol.set_state(U0, 0.0)
    sol.step(dt, 3)
    other = to_dev(synth.random_state(p, seed=8), torch.float64)
    sol.rhs(other, 0.4)
    torch.cuda.synchronize()
    sol.step(dt, 4)
    Ug, tg = sol.get_state()
    sol.close()
    assert tg == t_ref
    assert rel_max(Ug.cpu().numpy(), Uo) < FP64_TOL


@pytest.mark.parametrize("N", [3, 5, 7])
def test_periodic_step_fp32_ragged_tiles(sm, N):
    """FP32 steps: 37 faces along the sliding direction (ragged interface tiles), the moving
    block crossing several faces; both interfaces through the FP32 interface kernel; the
    increments against the oracle (fp32_steps)."""
    p = periodic_box(N, synth.RUSANOV, ny=37, nz=2, delta0=1.93, v=0.9, prec=synth.FP32)
    o = O.Oracle(p)
    sol = sm.Solver(p)
    err = F.check_fp32_steps(sol, o, F.perturbed(o.init_state(), seed=60 + N), synth.cfl_dt(p), 6, pieces=[2, 4])
    print("N=%d: increment rel L2 %.2e" % (N, err))
    sol.close()


@pytest.mark.parametrize("volume", [synth.VOLUME_WEAK, synth.VOLUME_SPLIT])
def test_periodic_closed_domain_conservation_gpu(sm, volume):
    """No boundary flux: the totals of the FP64 residual vanish to rounding."""
    p = periodic_box(4, synth.ROE_HH, volume, delta0=1.37)
    U = synth.random_state(p, seed=41)
    sol = sm.Solver(p)
    Ut = sol.rhs(to_dev(U, torch.float64), 0.07).cpu().numpy()
    sol.close()
    _, w = O.lgl(4)
    W = np.einsum("k,j,i->kji", w, w, w).ravel()
    Es = p.nel_s[0] * p.nel_s[1] * p.nel_s[2]
    hx = np.where(np.arange(Ut.shape[0]) < Es, (p.x1 - p.x0) / p.nel_s[0], (p.x2 - p.x1) / p.nel_m[0])
    J = hx * (p.y1 - p.y0) / p.nel_s[1] * (p.z1 - p.z0) / p.nel_s[2] / 8.0
    tot = np.einsum("e,evn,n->v", J, Ut, W)
    assert np.abs(tot).max() < 1e-13 * np.abs(Ut).max()


@pytest.mark.parametrize("N", [1, 4, 7])
def test_periodic_free_stream_gpu(sm, N):
    for prec, tol in ((synth.FP64, 1e-13), (synth.FP32, 1e-5)):
        p = periodic_box(N, synth.ROE_HH, delta0=0.011, prec=prec, flow="free")
        sol = sm.Solver(p)
        sol.init_state()
        U0, _ = sol.get_state()
        U0 = U0.clone()
        sol.step(synth.cfl_dt(p), 50)
        U1, _ = sol.get_state()
        sol.close()
        assert (U1 - U0).abs().max().item() < tol, (N, prec)


def test_periodic_zero_displacement_is_conforming(sm):
    for prec, dt, tol in ((synth.FP64, torch.float64, 1e-14), (synth.FP32, torch.float32, 1e-6)):
        for riemann in (synth.RUSANOV, synth.ROE_HH):
            p = periodic_box(3, riemann, v=0.0, delta0=0.0, prec=prec)
            U = to_dev(synth.random_state(p, seed=5), dt)
            a = sm.Solver(p).rhs(U, 0.2)
            p.interface_conforming = 1
            b = sm.Solver(p).rhs(U, 0.2)
            torch.cuda.synchronize()
            assert rel_max(a.cpu().numpy(), b.cpu().numpy()) < tol, (prec, riemann)


def test_periodic_rejected_where_unsupported(sm):
    p = synth.config_shear_x(N=3)
    p.periodic_x = 1
    with pytest.raises(sm.SlidemeshError):
        sm.Solver(p)
    p = periodic_box(3, synth.RUSANOV, prec=synth.FP32)
    s1 = sm.Solver(p)
    with pytest.raises(sm.SlidemeshError):
        sm.Batch([s1], [1e-3])
    s1.close()


def test_periodic_interface_heavy_full_size_sampled(sm):
    """2 x 4 x 256 x 256 elements closed in x (2 x 65,536 interface face pairs), N = 5, FP32,
    Rusanov: the launch configuration of the benchmark's two-interface leg; sampled elements,
    among them both interfaces' layers, against the oracle."""
    p = synth.config_interface_heavy(seed=1, precision=synth.FP32)
    p.periodic_x = 1
    E, nn = p.nelem, (p.N + 1) ** 3
    iz_s = [0, 129, 255]
    slabs = sorted({(iz + d) % 256 for iz in iz_s for d in (-1, 0, 1)})
    per_slab = 4 * 256
    Uh = torch.empty((E, 5, nn), dtype=torch.float32, pin_memory=True)
    chunk = 16 * per_slab
    lo = np.array([0.8, -0.3, -0.3, -0.3, 2.3])[None, :, None]
    hi = np.array([1.2, 0.3, 0.3, 0.3, 2.7])[None, :, None]
    for e0 in range(0, E, chunk):
        e1 = min(E, e0 + chunk)
        vals = synth.uniform(23, (e1 - e0) * 5 * nn, offset=e0 * 5 * nn).reshape(e1 - e0, 5, nn)
        Uh[e0:e1] = torch.from_numpy((lo + (hi - lo) * vals).astype(np.float32))
    sol = sm.Solver(p)
    t = 0.0321
    Ut = sol.rhs(Uh.cuda(), t)
    torch.cuda.synchronize()
    U64 = np.zeros((E, 5, nn))
    Es = p.nelem // 2
    for blk in (0, 1):
        for iz in slabs:
            a = blk * Es + iz * per_slab
            U64[a:a + per_slab] = Uh[a:a + per_slab].numpy().astype(np.float64)
    rng = np.random.default_rng(11)
    elems = []
    for blk in (0, 1):
        for iz in iz_s:
            for ix in (0, 3):                 # both interface layers of each block
                for iy in rng.choice(256, 5, replace=False):
                    elems.append(blk * Es + ix + 4 * (int(iy) + 256 * iz))
    elems = np.array(sorted(set(elems)))
    ref = O.Oracle(p).rhs_elements(U64, t, elems)
    got = Ut[torch.from_numpy(elems).cuda()].cpu().numpy()
    sol.close()
    assert rel_l2(got, ref) < FP32_TOL
    assert rel_max(got, ref) < 1e-4
