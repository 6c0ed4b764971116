"""GPU parity: the CUDA path (through the C-ABI) against the FP64 CPU oracle.

Bars: the interface configuration is bit-exact (n, s and partner table) against the
oracle's brute-force overlap search; FP64 results agree to 1e-12 relative (max-norm over
the array, relative to the array's max magnitude); FP32 results agree to 1e-5 relative L2.
Inputs are seeded (paper_2008_04356_gb300.synth) or computed by the oracle.
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


def rel_operator(Ut, ref, U, p):
    """Error of a residual relative to the size of the terms it is the difference of,
    |U| * (|v| + c) / h: for smooth data the residual is a small difference of such terms."""
    vel, c = synth.wave_speed_bounds(p)
    h = min((p.x1 - p.x0) / p.nel_s[0], (p.x2 - p.x1) / p.nel_m[0], (p.y1 - p.y0) / p.nel_s[1],
            (p.z1 - p.z0) / p.nel_s[2])
    scale = np.abs(U).max() * (max(vel) + abs(p.v) + c) / h
    return np.abs(np.asarray(Ut, np.float64) - ref).max() / scale


def rel_l2(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def to_dev(U, dtype):
    return torch.from_numpy(np.ascontiguousarray(U)).to(dtype).cuda()


# ------------------------------------------------------------------ mapper and matrices
@pytest.mark.parametrize("n_par,l", [(4, 0.25), (256, 1.0 / 256), (48, np.pi / 192), (7, 0.3)])
def test_map_bit_exact_vs_bruteforce(sm, n_par, l):
    count = 25000 if n_par <= 48 else 2000          # the brute force costs O(n_par^2) per call
    deltas = np.concatenate([synth.random_displacements(seed=100 + n_par, count=count, scale=9.0 * n_par * l),
                             np.arange(-3 * n_par, 3 * n_par + 1) * l, [0.0, -0.0, 1e-12, -1e-12]])
    n, s, pairs = sm.sm_map(torch.from_numpy(deltas).cuda(), l, n_par, with_pairs=True)
    torch.cuda.synchronize()
    n, s, pairs = n.cpu().numpy(), s.cpu().numpy(), pairs.cpu().numpy()
    for m, d in enumerate(deltas):
        rc, nb, sb, pb = O.map_bruteforce(d, l, n_par)
        if rc != 0:                      # outside the brute force's exact range: closed form
            nb, sb = O.map_closed(d, l)
            pb = O.map_pairs(nb, n_par)
        assert n[m] == nb, (d, n[m], nb)
        assert s[m].tobytes() == np.float64(sb).tobytes(), (d, s[m], sb)
        if m % 97 == 0 or m >= count:
            assert np.array_equal(pairs[m], pb)


@pytest.mark.parametrize("N", range(1, 8))
def test_mortar_matrices_vs_oracle(sm, N):
    for sigma in (-1.0, -0.731, -0.2, 0.0, 0.4142, 0.97, 1.0):
        g = sm.sm_mortar_matrices(N, sigma).cpu().numpy()
        ref = O.mortar_mats(N, sigma)
        for k in range(4):
            assert np.abs(g[k] - ref[k]).max() < 1e-13, (N, sigma, k)
        if sigma in (-1.0, 1.0):         # conforming instants are exact
            full = 1 if sigma == -1.0 else 0
            assert np.array_equal(g[full], np.eye(N + 1)) and np.array_equal(g[2 + full], np.eye(N + 1))


# ------------------------------------------------------------------ interface operator
def ragged_box(N, riemann, ny=11, nz=3, nx=(2, 3), delta0=0.3337, v=0.37, prec=synth.FP64):
    p = synth.config_box(N=N, v=v, precision=prec, riemann=riemann)
    p.nel_s, p.nel_m = (nx[0], ny, nz), (nx[1], ny, nz)
    p.x2 = 2.3
    p.delta0 = delta0
    return p


@pytest.mark.parametrize("riemann", [synth.RUSANOV, synth.ROE_HH])
@pytest.mark.parametrize("N", [1, 2, 3, 5, 7])
def test_interface_fp64(sm, N, riemann):
    for ny, delta0, t in ((11, 0.3337, 0.21), (4, 0.0, 0.0), (17, -2.71, 0.05), (1, 0.4, 0.0)):
        p = ragged_box(N, riemann, ny=ny, delta0=delta0)
        o = O.Oracle(p)
        U = synth.random_state(p, seed=N * 10 + ny)
        Fs_ref, Fm_ref = o.interface_fluxes(U, t)
        sol = sm.Solver(p)
        Fs, Fm = sol.interface(to_dev(U, torch.float64), t)
        torch.cuda.synchronize()
        assert rel_max(Fs.cpu().numpy(), Fs_ref) < FP64_TOL
        assert rel_max(Fm.cpu().numpy(), Fm_ref) < FP64_TOL
        sol.close()


@pytest.mark.parametrize("riemann", [synth.RUSANOV, synth.ROE_HH])
@pytest.mark.parametrize("N", [1, 2, 3, 5, 7])
def test_interface_fp32(sm, N, riemann):
    """FP32 interface fluxes (warp-owned row pairs in tiles of 4 faces at odd N, staged tile
    of 8 faces at even N) against the oracle: ragged last tiles (11, 17, 40), a single tile
    (4), one face (1), partner offsets that wrap both ways, and the conforming instant."""
    for ny, delta0, t in ((11, 0.3337, 0.21), (4, 0.0, 0.0), (17, -2.71, 0.05), (1, 0.4, 0.0), (40, 5.123, 0.3)):
        p = ragged_box(N, riemann, ny=ny, delta0=delta0, prec=synth.FP32)
        o = O.Oracle(p)
        U = synth.random_state(p, seed=N * 10 + ny).astype(np.float32)
        Fs_ref, Fm_ref = o.interface_fluxes(U.astype(np.float64), t)
        sol = sm.Solver(p)
        Fs, Fm = sol.interface(to_dev(U, torch.float32), t)
        torch.cuda.synchronize()
        assert rel_l2(Fs.cpu().numpy(), Fs_ref) < FP32_TOL, (ny, "static")
        assert rel_l2(Fm.cpu().numpy(), Fm_ref) < FP32_TOL, (ny, "moving")
        sol.close()


# ------------------------------------------------------------------ full right-hand side
@pytest.mark.parametrize("riemann", [synth.RUSANOV, synth.ROE_HH])
@pytest.mark.parametrize("N", range(1, 8))
def test_rhs_fp64_random_state(sm, N, riemann):
    p = ragged_box(N, riemann)
    o = O.Oracle(p)
    U = synth.random_state(p, seed=77 + N)
    t = 0.123
    ref = o.rhs(U, t)
    sol = sm.Solver(p)
    Ut = sol.rhs(to_dev(U, torch.float64), t).cpu().numpy()
    assert rel_max(Ut, ref) < FP64_TOL
    sol.close()


@pytest.mark.parametrize("N", [2, 4, 6])
def test_rhs_fp64_smooth_wave_and_polynomial(sm, N):
    for p in (synth.config_box(N=N), synth.config_poly_x(N=min(N, 3) + 1, v=0.41)):
        p.delta0 = 0.1234
        o = O.Oracle(p)
        U = o.exact_state(0.05)
        ref = o.rhs(U, 0.05)
        sol = sm.Solver(p)
        Ut = sol.rhs(to_dev(U, torch.float64), 0.05).cpu().numpy()
        assert rel_operator(Ut, ref, U, p) < FP64_TOL
        sol.close()


def test_zero_displacement_reproduces_conforming_mesh(sm):
    """At zero displacement the sliding path (identity mortar operators) and the conforming
    coupling of the two blocks give the same residual to rounding.  (The oracle, compiled
    without multiply-add contraction, pins this bit for bit; on the GPU the two code paths
    inline the Riemann solver in different kernels, where the compiler may contract
    multiply-adds differently.)"""
    for prec, dt, tol in ((synth.FP64, torch.float64, 1e-14), (synth.FP32, torch.float32, 1e-6)):
        for riemann in (synth.RUSANOV, synth.ROE_HH):
            p = synth.config_box(N=3, v=0.0, precision=prec, riemann=riemann)
            U = to_dev(synth.random_state(p, seed=5), dt)
            a = sm.Solver(p).rhs(U, 0.2)
            p.interface_conforming = 1
            b = sm.Solver(p).rhs(U, 0.2)
            torch.cuda.synchronize()
            err = rel_max(a.cpu().numpy(), b.cpu().numpy())
            assert err < tol, (prec, riemann, err)


@pytest.mark.parametrize("riemann", [synth.RUSANOV, synth.ROE_HH])
def test_rhs_fp32_vs_oracle(sm, riemann):
    for N in (1, 3, 5, 7):
        p = ragged_box(N, riemann, prec=synth.FP32)
        U = synth.random_state(p, seed=31 + N).astype(np.float32)
        ref = O.Oracle(p).rhs(U.astype(np.float64), 0.3)
        Ut = sm.Solver(p).rhs(to_dev(U, torch.float32), 0.3).cpu().numpy()
        assert rel_l2(Ut, ref) < FP32_TOL


# ------------------------------------------------------------------ time stepping
def test_step_fp64_box_100_steps(sm):
    """The 8x4x2 box, N = 3, moving block at v = 0.5, entropy wave, 100 steps, CFL 0.9."""
    p = synth.config_box(N=3)
    o = O.Oracle(p)
    U0 = o.init_state()
    dt = synth.cfl_dt(p)
    Uo, Go = U0.copy(), np.zeros_like(U0)
    t_ref = o.step(Uo, Go, 0.0, dt, 100)
    sol = sm.Solver(p)
    sol.set_state(U0, 0.0)
    sol.step(dt, 100)
    Ug, tg = sol.get_state()
    assert tg == t_ref
    assert rel_max(Ug.cpu().numpy(), Uo) < FP64_TOL


@pytest.mark.parametrize("riemann", [synth.RUSANOV, synth.ROE_HH])
@pytest.mark.parametrize("N", [1, 4, 7])
def test_step_fp64_ragged(sm, N, riemann):
    p = ragged_box(N, riemann, delta0=0.91)
    o = O.Oracle(p)
    U0 = o.init_state()
    dt = synth.cfl_dt(p)
    Uo, Go = U0.copy(), np.zeros_like(U0)
    t_ref = o.step(Uo, Go, 0.0, dt, 7)
    sol = sm.Solver(p)
    sol.set_state(U0, 0.0)
    sol.step(dt, 3)
    sol.step(dt, 4)                      # graph replays on both buffer parities
    Ug, tg = sol.get_state()
    assert tg == t_ref
    assert rel_max(Ug.cpu().numpy(), Uo) < FP64_TOL


def test_step_fp32_vs_oracle(sm):
    """FP32 steps of the 2 x 4^3 box, N = 5, by increments (see fp32_steps): the smooth
    entropy wave over 100 steps, whose increment the FP32 storage pins only to its emulated
    floor of 1.6e-5 (bar 5e-5), and the same flow with seeded noise over 10 steps at 1e-5."""
    p = synth.config_box(N=5, k=4, precision=synth.FP32)
    o = O.Oracle(p)
    dt = synth.cfl_dt(p)
    sol = sm.Solver(p)
    U0 = o.init_state().astype(np.float32).astype(np.float64)
    err = F.check_fp32_steps(sol, o, U0, dt, 100, tol=5e-5)
    print("smooth 100 steps: increment rel L2 %.2e" % err)
    err = F.check_fp32_steps(sol, o, F.perturbed(o.init_state(), seed=21), dt, 10)
    print("perturbed 10 steps: increment rel L2 %.2e" % err)
    sol.close()


@pytest.mark.parametrize("N", [3, 5, 7])
def test_step_fp32_ragged_tiles(sm, N):
    """FP32 steps through the compact interface traces (the stepping path of the interface
    kernel): 37 faces along the sliding direction (4 full tiles and a ragged one), moving
    block crossing several faces; increments against the oracle (fp32_steps), in two sm_step
    calls so that both buffer parities of the captured step run."""
    p = ragged_box(N, synth.RUSANOV, ny=37, nz=2, delta0=1.93, v=0.9, prec=synth.FP32)
    o = O.Oracle(p)
    sol = sm.Solver(p)
    err = F.check_fp32_steps(sol, o, F.perturbed(o.init_state(), seed=30 + N), synth.cfl_dt(p), 6, pieces=[1, 5])
    print("N=%d: increment rel L2 %.2e" % (N, err))
    sol.close()


def test_step_fp32_interface_ring_wraps(sm):
    """More interface tiles than resident CTAs (2 x 4 x 256 x 32 elements, N = 5: 1,024
    tiles of 8 faces), so every CTA of the persistent FP32 interface kernel cycles its
    three trace buffers; one RK step (first-stage and later-stage element kernels, trace
    writes, interface kernel on the written traces) by increments against the oracle."""
    p = synth.config_interface_heavy(seed=3, precision=synth.FP32, nz=32)
    o = O.Oracle(p)
    sol = sm.Solver(p)
    err = F.check_fp32_steps(sol, o, F.perturbed(o.init_state(), seed=41), synth.cfl_dt(p), 1)
    print("increment rel L2 %.2e" % err)
    sol.close()


def near_uniform_state(E, nn, seed, out):
    """Fills the pinned FP32 tensor out (E, 5, nn) with conservative states drawn uniformly
    around rho = 1, m = 0, rho e = 2.5 (rho in [0.9, 1.1], m in [-0.1, 0.1]^3, rho e in
    [2.25, 2.75]): an input generated without the oracle and the CUDA path alike."""
    lo = np.array([0.9, -0.1, -0.1, -0.1, 2.25])[None, :, None]
    hi = np.array([1.1, 0.1, 0.1, 0.1, 2.75])[None, :, None]
    chunk = 16384
    for e0 in range(0, E, chunk):
        e1 = min(E, e0 + chunk)
        vals = synth.uniform(seed, (e1 - e0) * 5 * nn, offset=e0 * 5 * nn).reshape(e1 - e0, 5, nn)
        out[e0:e1] = torch.from_numpy((lo + (hi - lo) * vals).astype(np.float32))


@pytest.mark.slow
def test_step_fp32_full_size_sampled(sm):
    """The benchmarked stage-mode launches at full size: 2 x 4 x 256 x 256 elements, N = 5,
    FP32, one RK step through sm_step (element kernel with the RK update and trace writes,
    persistent interface kernel on the written traces).  The increment of whole z-slabs is
    compared with the oracle's FP64 stages, which are run on shrinking slab ranges: the five
    stages of a step reach at most five elements along z (through faces, the interface and
    its partner shift), so stage k is evaluated on the slabs within 4 - k of a sampled slab,
    from a state that is exact on the slabs within 5 - k."""
    p = synth.config_interface_heavy(seed=1, precision=synth.FP32)
    E, nn = p.nelem, (p.N + 1) ** 3
    nx, ny, nz = p.nel_s
    per_slab = nx * ny
    Es = E // 2
    Uh = torch.empty((E, 5, nn), dtype=torch.float32, pin_memory=True)
    near_uniform_state(E, nn, 17, Uh)
    dt = synth.cfl_dt(p)
    sol = sm.Solver(p)
    sol.set_state(Uh, 0.0)
    sol.step(dt, 1)
    Ug, _ = sol.get_state()
    torch.cuda.synchronize()
    sol.close()
    A, B, c = O.lsrk_coeffs()
    o = O.Oracle(p)
    for izc in (0, 137):
        def slab_elems(radius):
            out = []
            for blk in (0, 1):
                for dz in range(-radius, radius + 1):
                    a = blk * Es + ((izc + dz) % nz) * per_slab
                    out.append(np.arange(a, a + per_slab))
            return np.concatenate(out)
        # a lazily zeroed full-size FP64 state, exact on the slabs within 5 of izc
        U = np.zeros((E, 5, nn))
        e5 = slab_elems(5)
        U[e5] = Uh[torch.from_numpy(e5)].numpy().astype(np.float64)
        U0c = U[slab_elems(0)].copy()
        G = np.zeros((E, 5, nn))
        for k in range(5):
            ek = slab_elems(4 - k)
            Ut = o.rhs_elements(U, c[k] * dt, ek)
            G[ek] = A[k] * G[ek] + dt * Ut
            U[ek] += B[k] * G[ek]
        e0 = slab_elems(0)
        got = Ug[torch.from_numpy(e0).cuda()].cpu().numpy().astype(np.float64)
        err = F.increment_error(U0c, got, U[e0])
        print("slab %d: increment rel L2 %.2e" % (izc, err))
        assert err < F.INCREMENT_TOL
        assert rel_max(got - U0c, U[e0] - U0c) < 1e-4


def test_init_state_matches_oracle(sm):
    for p in (synth.config_box(N=4), synth.config_interface_heavy(seed=2, precision=synth.FP64, nz=4, ny=8)):
        p.delta0 = 0.07
        ref = O.Oracle(p).init_state()
        sol = sm.Solver(p)
        sol.init_state()
        U, t = sol.get_state()
        assert t == 0.0
        assert rel_max(U.cpu().numpy(), ref) < 1e-14


# ------------------------------------------------------------------ properties
@pytest.mark.parametrize("N", range(1, 8))
def test_free_stream_preserved_gpu(sm, N):
    for prec, tol in ((synth.FP64, 1e-13), (synth.FP32, 1e-5)):
        p = synth.config_box(N=N, flow="free", v=0.37, precision=prec)
        p.delta0 = 0.011
        sol = sm.Solver(p)
        sol.init_state()
        U0, _ = sol.get_state()
        U0 = U0.clone()
        sol.step(synth.cfl_dt(p), 100)
        U1, _ = sol.get_state()
        assert (U1 - U0).abs().max().item() < tol


def test_interface_conservation_gpu(sm):
    for prec, dt, tol in ((synth.FP64, torch.float64, 1e-13), (synth.FP32, torch.float32, 1e-5)):
        for delta0 in (0.05, 0.3337, 1.91, -0.77):
            p = synth.config_box(N=4, precision=prec)
            p.delta0 = delta0
            sol = sm.Solver(p)
            U = to_dev(synth.random_state(p, seed=9), dt)
            Fs, Fm = sol.interface(U, 0.0)
            _, w = O.lgl(4)
            W = torch.from_numpy(np.outer(w, w)).cuda()
            ss = (Fs.double() * W).sum(dim=(0, 1, 3, 4))
            sm_ = (Fm.double() * W).sum(dim=(0, 1, 3, 4))
            scale = Fs.double().abs().sum(dim=(0, 1, 3, 4))
            assert ((ss + sm_).abs() <= tol * scale).all()


def test_diag_totals_and_interface_sums(sm):
    p = synth.config_box(N=3)
    p.delta0 = 0.3
    o = O.Oracle(p)
    U0 = o.init_state()
    sol = sm.Solver(p)
    sol.set_state(U0, 0.0)
    sol.step(synth.cfl_dt(p), 2)
    d = sol.diag()
    U, _ = sol.get_state()
    assert np.allclose(d["totals"], o.totals(U.cpu().numpy()), rtol=1e-13, atol=0)
    ss, sm_ = np.array(d["iface_sum_static"]), np.array(d["iface_sum_moving"])
    assert np.all(np.abs(ss + sm_) < 1e-13 * (1 + np.abs(ss)))
    assert d["status"] == 0


# ------------------------------------------------------------------ full-size workload
def test_interface_heavy_full_size_sampled(sm):
    """2 x 4 x 256 x 256 elements, N = 5, FP32 (the benchmarked launch configuration of the
    element and interface kernels), random state: sampled elements against the oracle."""
    p = synth.config_interface_heavy(seed=1, precision=synth.FP32)
    E, nn = p.nelem, (p.N + 1) ** 3
    # slabs of constant iz feed the sampled elements and all their neighbours
    iz_s = [0, 1, 128, 255]
    slabs = sorted({(iz + d) % 256 for iz in iz_s for d in (-1, 0, 1)})
    per_slab = 4 * 256
    Uh = torch.empty((E, 5, nn), dtype=torch.float32, pin_memory=True)
    chunk = 16 * per_slab
    for e0 in range(0, E, chunk):
        e1 = min(E, e0 + chunk)
        vals = synth.uniform(7, (e1 - e0) * 5 * nn, offset=e0 * 5 * nn).reshape(e1 - e0, 5, nn)
        lo = np.array([0.8, -0.3, -0.3, -0.3, 2.3])[None, :, None]
        hi = np.array([1.2, 0.3, 0.3, 0.3, 2.7])[None, :, None]
        Uh[e0:e1] = torch.from_numpy((lo + (hi - lo) * vals).astype(np.float32))
    sol = sm.Solver(p)
    dU = Uh.cuda()
    t = 0.0123
    Ut = sol.rhs(dU, t)
    torch.cuda.synchronize()
    # oracle on the sampled elements: a lazily zeroed full-size FP64 array, filled on the slabs
    U64 = np.zeros((E, 5, nn))
    Es = p.nelem // 2
    for blk in (0, 1):
        for iz in slabs:
            a = blk * Es + iz * per_slab
            U64[a:a + per_slab] = Uh[a:a + per_slab].numpy().astype(np.float64)
    rng = np.random.default_rng(3)
    elems = []
    for blk in (0, 1):
        for iz in iz_s:
            for ix in (0, 1, 3):
                for iy in rng.choice(256, 6, replace=False):
                    elems.append(blk * Es + ix + 4 * (int(iy) + 256 * iz))
    elems = np.array(sorted(set(elems)))
    ref = O.Oracle(p).rhs_elements(U64, t, elems)
    got = Ut[torch.from_numpy(elems).cuda()].cpu().numpy()
    assert rel_l2(got, ref) < FP32_TOL
    assert rel_max(got, ref) < 1e-4


@pytest.mark.parametrize("prec", [synth.FP32, synth.FP64])
def test_misaligned_device_arrays_are_refused(sm, prec):
    """The kernels move caller arrays in 8- and 16-byte vectors: a state or output that is
    not 16-byte aligned is refused with SM_ERR_ARG before any launch."""
    p = ragged_box(3, synth.RUSANOV, prec=prec)
    dt = torch.float64 if prec == synth.FP64 else torch.float32
    sol = sm.Solver(p)
    n = p.nelem * 5 * (p.N + 1) ** 3
    buf = torch.zeros(n + 4, dtype=dt, device="cuda")
    out = torch.empty(n, dtype=dt, device="cuda")
    L = sm.lib()
    st = torch.cuda.current_stream().cuda_stream
    for off in (1, 2, 3):
        if (off * buf.element_size()) % 16 == 0:
            continue
        rc = L.sm_rhs(sol.h, 0.1, buf[off:].data_ptr(), out.data_ptr(), st)
        assert rc == -1 and b"aligned" in L.sm_last_error()
        rc = L.sm_rhs(sol.h, 0.1, out.data_ptr(), buf[off:].data_ptr(), st)
        assert rc == -1
    torch.cuda.synchronize()
    sol.close()
