"""GPU parity of the split-form volume integral (Sec. 3.1, the split formulation with
Pirozzoli's two-point flux) against the FP64 CPU oracle, through the C-ABI.

The oracle evaluates the strong form literally (2 D_il F#(U_i, U_l) over every l, then the
surface term F* - F(U) at the face nodes); the kernel folds the surface correction into the
operator Ds = 2D - M^-1 B, skips its zero diagonal and evaluates each pair flux once for both
of its nodes.  Bars as for the weak form: FP64 1e-12 relative (max norm), FP32 1e-5 relative
L2, free stream to 1e-13 (FP64).
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


def split_box(N, riemann, ny=11, nz=3, nx=(2, 3), delta0=0.3337, v=0.37, prec=synth.FP64):
    """Ragged two-block box: element counts that fill no whole CTA (N = 1..4 pack 32, 8, 4, 2
    elements per CTA), a moving block of another width, a sub-face offset."""
    p = synth.config_box(N=N, v=v, precision=prec, riemann=riemann)
    p.nel_s, p.nel_m = (nx[0], ny, nz), (nx[1], ny, nz)
    p.x2 = 2.3
    p.delta0 = delta0
    p.volume = synth.VOLUME_SPLIT
    return p


@pytest.mark.parametrize("riemann", [synth.RUSANOV, synth.ROE_HH])
@pytest.mark.parametrize("N", range(1, 8))
def test_split_rhs_fp64_random_state(sm, N, riemann):
    p = split_box(N, riemann)
    U = synth.random_state(p, seed=177 + N)
    ref = O.Oracle(p).rhs(U, 0.123)
    sol = sm.Solver(p)
    Ut = sol.rhs(to_dev(U, torch.float64), 0.123).cpu().numpy()
    sol.close()
    assert rel_max(Ut, ref) < FP64_TOL


@pytest.mark.parametrize("N", [2, 5])
def test_split_rhs_fp64_smooth_wave(sm, N):
    p = synth.config_box(N=N)
    p.delta0, p.volume, p.riemann = 0.1234, synth.VOLUME_SPLIT, synth.ROE_HH
    o = O.Oracle(p)
    U = o.exact_state(0.05)
    ref = o.rhs(U, 0.05)
    sol = sm.Solver(p)
    Ut = sol.rhs(to_dev(U, torch.float64), 0.05).cpu().numpy()
    sol.close()
    # a smooth residual is a small difference of flux terms |U| (|v| + c) / h: relative to those
    vel, c = synth.wave_speed_bounds(p)
    scale = np.abs(U).max() * (max(vel) + abs(p.v) + c) / 0.25
    assert np.abs(Ut - ref).max() / scale < FP64_TOL


@pytest.mark.parametrize("riemann", [synth.RUSANOV, synth.ROE_HH])
def test_split_rhs_fp32_vs_oracle(sm, riemann):
    for N in (1, 3, 5, 7):
        p = split_box(N, riemann, prec=synth.FP32)
        U = synth.random_state(p, seed=131 + N).astype(np.float32)
        ref = O.Oracle(p).rhs(U.astype(np.float64), 0.3)
        Ut = sm.Solver(p).rhs(to_dev(U, torch.float32), 0.3).cpu().numpy()
        assert rel_l2(Ut, ref) < FP32_TOL, N


@pytest.mark.parametrize("N", [1, 3, 4, 7])
def test_split_step_fp64_ragged(sm, N):
    p = split_box(N, synth.ROE_HH, delta0=0.91)
    o = O.Oracle(p)
    U0 = o.init_state()
    dt = synth.cfl_dt(p)
    Uo, Go = U0.copy(), np.zeros_like(U0)
    t_ref = o.step(Uo, Go, 0.0, dt, 7)
    sol = sm.Solver(p)
    sol.set_state(U0, 0.0)
    sol.step(dt, 3)
    sol.step(dt, 4)
    Ug, tg = sol.get_state()
    sol.close()
    assert tg == t_ref
    assert rel_max(Ug.cpu().numpy(), Uo) < FP64_TOL


def test_split_step_fp64_box_100_steps(sm):
    """The 8x4x2 box, N = 3, moving block at v = 0.5, entropy wave, 100 steps, Roe/HH."""
    p = synth.config_box(N=3, riemann=synth.ROE_HH)
    p.volume = synth.VOLUME_SPLIT
    o = O.Oracle(p)
    U0 = o.init_state()
    dt = synth.cfl_dt(p)
    Uo, Go = U0.copy(), np.zeros_like(U0)
    o.step(Uo, Go, 0.0, dt, 100)
    sol = sm.Solver(p)
    sol.set_state(U0, 0.0)
    sol.step(dt, 100)
    Ug, _ = sol.get_state()
    sol.close()
    assert rel_max(Ug.cpu().numpy(), Uo) < FP64_TOL


@pytest.mark.parametrize("N", [3, 5])
def test_split_step_fp32_vs_oracle(sm, N):
    p = split_box(N, synth.ROE_HH, ny=37, nz=2, delta0=1.93, v=0.9, prec=synth.FP32)
    o = O.Oracle(p)
    sol = sm.Solver(p)
    err = F.check_fp32_steps(sol, o, F.perturbed(o.init_state(), seed=120 + N), synth.cfl_dt(p), 20, pieces=[7, 13])
    print("N=%d: increment rel L2 %.2e" % (N, err))
    sol.close()


@pytest.mark.parametrize("N", range(1, 8))
def test_split_free_stream_preserved_gpu(sm, N):
    for prec, tol in ((synth.FP64, 1e-13), (synth.FP32, 1e-5)):
        p = synth.config_box(N=N, flow="free", v=0.37, precision=prec, riemann=synth.ROE_HH)
        p.delta0, p.volume = 0.011, synth.VOLUME_SPLIT
        sol = sm.Solver(p)
        sol.init_state()
        U0, _ = sol.get_state()
        U0 = U0.clone()
        sol.step(synth.cfl_dt(p), 50)
        U1, _ = sol.get_state()
        sol.close()
        assert (U1 - U0).abs().max().item() < tol, (N, prec)


def test_split_interface_heavy_full_size_sampled(sm):
    """2 x 4 x 256 x 256 elements, N = 5, FP32, Roe/HH: the launch configuration the
    benchmark times for the split form; sampled elements against the oracle."""
    p = synth.config_interface_heavy(seed=1, precision=synth.FP32)
    p.volume, p.riemann = synth.VOLUME_SPLIT, synth.ROE_HH
    E, nn = p.nelem, (p.N + 1) ** 3
    iz_s = [0, 1, 128, 255]
    slabs = sorted({(iz + d) % 256 for iz in iz_s for d in (-1, 0, 1)})
    per_slab = 4 * 256
    Uh = torch.empty((E, 5, nn), dtype=torch.float32, pin_memory=True)
    chunk = 16 * per_slab
    lo = np.array([0.8, -0.3, -0.3, -0.3, 2.3])[None, :, None]
    hi = np.array([1.2, 0.3, 0.3, 0.3, 2.7])[None, :, None]
    for e0 in range(0, E, chunk):
        e1 = min(E, e0 + chunk)
        vals = synth.uniform(17, (e1 - e0) * 5 * nn, offset=e0 * 5 * nn).reshape(e1 - e0, 5, nn)
        Uh[e0:e1] = torch.from_numpy((lo + (hi - lo) * vals).astype(np.float32))
    sol = sm.Solver(p)
    t = 0.0123
    Ut = sol.rhs(Uh.cuda(), t)
    torch.cuda.synchronize()
    U64 = np.zeros((E, 5, nn))
    Es = p.nelem // 2
    for blk in (0, 1):
        for iz in slabs:
            a = blk * Es + iz * per_slab
            U64[a:a + per_slab] = Uh[a:a + per_slab].numpy().astype(np.float64)
    rng = np.random.default_rng(5)
    elems = []
    for blk in (0, 1):
        for iz in iz_s:
            for ix in (0, 2, 3):
                for iy in rng.choice(256, 5, replace=False):
                    elems.append(blk * Es + ix + 4 * (int(iy) + 256 * iz))
    elems = np.array(sorted(set(elems)))
    ref = O.Oracle(p).rhs_elements(U64, t, elems)
    got = Ut[torch.from_numpy(elems).cuda()].cpu().numpy()
    sol.close()
    assert rel_l2(got, ref) < FP32_TOL
    assert rel_max(got, ref) < 1e-4
