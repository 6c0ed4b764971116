"""Thin ctypes binding of libslidemesh (include/slidemesh.h): argument marshalling only.

Every computation runs in the library's CUDA kernels; PyTorch supplies device memory and
the current CUDA stream.  Importing this module does not load the library; the first call
does, and raises if libslidemesh.so is missing (build it with build.build_library()).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import synth

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libslidemesh.so")

SM_OK, SM_PENDING = 0, 1
SM_FP64, SM_FP32 = 0, 1


class SmMeshDesc(C.Structure):
    _fields_ = [("N", C.c_int), ("geom", C.c_int), ("nel_static", C.c_int * 3), ("nel_moving", C.c_int * 3),
                ("x0", C.c_double), ("x1", C.c_double), ("x2", C.c_double), ("y0", C.c_double),
                ("y1", C.c_double), ("z0", C.c_double), ("z1", C.c_double), ("gamma", C.c_double),
                ("riemann", C.c_int), ("precision", C.c_int), ("interface_conforming", C.c_int),
                ("flow", C.c_int), ("fpar", C.c_double * 16), ("modes", C.c_double * 160),
                ("physics", C.c_int), ("mu", C.c_double), ("Pr", C.c_double), ("Rgas", C.c_double),
                ("volume", C.c_int), ("periodic_x", C.c_int), ("cone_angle", C.c_double)]


class SmMotion(C.Structure):
    _fields_ = [("v", C.c_double), ("omega", C.c_double), ("delta0", C.c_double)]


class SmDiag(C.Structure):
    _fields_ = [("n_delta", C.c_longlong), ("s_delta", C.c_double), ("t", C.c_double),
                ("totals", C.c_double * 5), ("iface_sum_static", C.c_double * 5),
                ("iface_sum_moving", C.c_double * 5)]


class SmRequest(C.Structure):
    _fields_ = [("desc", SmMeshDesc), ("motion", SmMotion), ("dt", C.c_double), ("nsteps", C.c_int),
                ("keep_state", C.c_int)]


class SmResult(C.Structure):
    _fields_ = [("status", C.c_int), ("t_submit", C.c_double), ("t_admit", C.c_double), ("t_done", C.c_double),
                ("sim_time", C.c_double), ("dof", C.c_longlong), ("steps", C.c_int), ("totals", C.c_double * 5),
                ("state", C.c_void_p), ("state_bytes", C.c_longlong)]


class SmServerStats(C.Structure):
    _fields_ = [("submitted", C.c_longlong), ("completed", C.c_longlong), ("failed", C.c_longlong),
                ("running", C.c_longlong), ("queued", C.c_longlong), ("batched_steps", C.c_longlong),
                ("dof_updates", C.c_longlong), ("busy_seconds", C.c_double), ("bytes_in_use", C.c_size_t),
                ("peak_bytes", C.c_size_t), ("max_concurrent", C.c_int)]


_vp = C.c_void_p
_SIGS = {
    "sm_init_mesh": (C.c_int, [C.POINTER(SmMeshDesc), C.POINTER(_vp)]),
    "sm_set_motion": (C.c_int, [_vp, C.POINTER(SmMotion)]),
    "sm_state_size": (C.c_longlong, [_vp]),
    "sm_scalar_bytes": (C.c_int, [_vp]),
    "sm_init_state": (C.c_int, [_vp, _vp]),
    "sm_set_state": (C.c_int, [_vp, _vp, C.c_int, C.c_double, _vp]),
    "sm_get_state": (C.c_int, [_vp, _vp, C.c_int, C.POINTER(C.c_double), _vp]),
    "sm_rhs": (C.c_int, [_vp, C.c_double, _vp, _vp, _vp]),
    "sm_interface": (C.c_int, [_vp, C.c_double, _vp, _vp, _vp, _vp]),
    "sm_step": (C.c_int, [_vp, C.c_double, C.c_int, _vp]),
    "sm_stream_jobs": (C.c_int, [_vp, _vp, C.c_longlong, _vp, C.c_longlong, C.c_int, C.c_double, C.c_double, C.c_int,
                                 _vp]),
    "sm_gradients": (C.c_int, [_vp, C.c_double, _vp, _vp, _vp]),
    "sm_step_profiled": (C.c_int, [_vp, C.c_double, C.c_int, _vp, C.POINTER(C.c_double), C.POINTER(C.c_int)]),
    "sm_diag": (C.c_int, [_vp, C.POINTER(SmDiag), _vp]),
    "sm_state_ptr": (_vp, [_vp]),
    "sm_destroy": (None, [_vp]),
    "sm_rhs_static": (C.c_int, [C.POINTER(SmMeshDesc), C.POINTER(SmMotion), C.c_double, _vp, _vp, _vp]),
    "sm_map": (C.c_int, [_vp, C.c_int, C.c_double, C.c_int, _vp, _vp, _vp, _vp]),
    "sm_mortar_matrices": (C.c_int, [C.c_int, C.c_double, _vp, _vp]),
    "sm_fp64_fma_probe": (C.c_int, [C.c_int, C.c_int, C.c_int, _vp, _vp]),
    "sm_batch_create": (C.c_int, [C.POINTER(_vp), C.POINTER(C.c_double), C.c_int, C.POINTER(_vp)]),
    "sm_batch_autotune": (C.c_int, [_vp, _vp]),
    "sm_batch_step": (C.c_int, [_vp, C.c_int, _vp]),
    "sm_batch_shapes": (C.c_int, [_vp, C.c_int, C.POINTER(C.c_int)]),
    "sm_batch_destroy": (None, [_vp]),
    "sm_server_create": (C.c_int, [C.c_size_t, C.c_int, C.POINTER(_vp)]),
    "sm_submit": (C.c_int, [_vp, C.POINTER(SmRequest), C.POINTER(C.c_uint64)]),
    "sm_poll": (C.c_int, [_vp, C.c_uint64, C.POINTER(SmResult)]),
    "sm_server_wait": (C.c_int, [_vp, C.c_double]),
    "sm_server_stats": (C.c_int, [_vp, C.POINTER(SmServerStats)]),
    "sm_server_destroy": (None, [_vp]),
    "sm_status_string": (C.c_char_p, [C.c_int]),
    "sm_last_error": (C.c_char_p, []),
}

_LIB = None


def lib():
    """The loaded library; raises if it has not been built."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libslidemesh.so is missing at %s: run paper_2008_04356_gb300.build.build_library()"
                               % LIB_PATH)
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _LIB = L
    return _LIB


class SlidemeshError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        L = lib()
        msg = "%s failed: %s (%s)" % (where, L.sm_status_string(status).decode(), L.sm_last_error().decode())
        super().__init__(msg)


def check(status, where):
    if status != SM_OK:
        raise SlidemeshError(status, where)


def _stream(stream):
    if stream is None:
        import torch
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(stream.cuda_stream)


def mesh_desc(p: synth.Problem) -> SmMeshDesc:
    d = SmMeshDesc()
    d.N, d.geom = p.N, int(getattr(p, "geom", 0))
    for k in range(3):
        d.nel_static[k], d.nel_moving[k] = int(p.nel_s[k]), int(p.nel_m[k])
    for name in ("x0", "x1", "x2", "y0", "y1", "z0", "z1", "gamma"):
        setattr(d, name, float(getattr(p, name)))
    d.riemann, d.precision = int(p.riemann), int(p.precision)
    d.interface_conforming, d.flow = int(p.interface_conforming), int(p.flow)
    for k, f in enumerate(p.fpar16()):
        d.fpar[k] = f
    for k, m in enumerate(p.modes_array().ravel()):
        d.modes[k] = m
    d.physics, d.mu, d.Pr, d.Rgas = int(p.physics), float(p.mu), float(p.Pr), float(p.Rgas)
    d.volume = int(getattr(p, "volume", 0))
    d.periodic_x = int(getattr(p, "periodic_x", 0))
    d.cone_angle = float(getattr(p, "cone_angle", 0.0))
    return d


def sm_map(d_delta, l: float, n_par: int, with_pairs: bool = True, stream=None):
    """Device interface configuration for a batch of displacements (torch float64 cuda)."""
    import torch
    count = d_delta.numel()
    n = torch.empty(count, dtype=torch.int64, device=d_delta.device)
    s = torch.empty(count, dtype=torch.float64, device=d_delta.device)
    pairs = torch.empty((count, n_par, 2), dtype=torch.int32, device=d_delta.device) if with_pairs else None
    check(lib().sm_map(d_delta.data_ptr(), count, float(l), int(n_par), n.data_ptr(), s.data_ptr(),
                       pairs.data_ptr() if pairs is not None else None, _stream(stream)), "sm_map")
    return n, s, pairs


def sm_rhs_static(problem: synth.Problem, dU, t: float, out=None, stream=None):
    """dU/dt through the entry point that allocates no device memory (the library keeps its
    scratch in a fixed device array); dU and out are the caller's device tensors."""
    import torch
    if out is None:
        out = torch.empty_like(dU)
    desc = mesh_desc(problem)
    mo = SmMotion(float(problem.v), 0.0, float(problem.delta0))
    check(lib().sm_rhs_static(C.byref(desc), C.byref(mo), float(t), dU.data_ptr(), out.data_ptr(),
                              _stream(stream)), "sm_rhs_static")
    return out


def sm_fp64_fma_probe(blocks: int, threads: int, iters: int, out, stream=None):
    """Launches the FP64 FMA throughput probe (16 * iters * blocks * threads flop) on the
    stream; out: a cuda float64 tensor of blocks * threads elements."""
    assert out.is_cuda and out.numel() >= blocks * threads
    check(lib().sm_fp64_fma_probe(int(blocks), int(threads), int(iters), out.data_ptr(), _stream(stream)),
          "sm_fp64_fma_probe")
    return out


def sm_mortar_matrices(N: int, sigma: float, device="cuda", stream=None):
    import torch
    out = torch.empty((4, N + 1, N + 1), dtype=torch.float64, device=device)
    check(lib().sm_mortar_matrices(int(N), float(sigma), out.data_ptr(), _stream(stream)), "sm_mortar_matrices")
    return out  # P_lo, P_hi, B_lo, B_hi


class Solver:
    """One sliding-mesh solve on the current CUDA device (library-owned state)."""

    def __init__(self, problem: synth.Problem):
        self.problem = problem
        self._desc = mesh_desc(problem)
        h = C.c_void_p()
        check(lib().sm_init_mesh(C.byref(self._desc), C.byref(h)), "sm_init_mesh")
        self.h = h
        self.set_motion(problem.v, problem.delta0)
        self.N = problem.N
        self.nn = (problem.N + 1) ** 3
        self.E = problem.nelem
        self.size = int(lib().sm_state_size(self.h))
        self.dtype_np = np.float64 if problem.precision == SM_FP64 else np.float32

    @property
    def torch_dtype(self):
        import torch
        return torch.float64 if self.problem.precision == SM_FP64 else torch.float32

    def shape(self):
        return (self.E, 5, self.nn)

    def close(self):
        if getattr(self, "h", None):
            lib().sm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_motion(self, v: float, delta0: float = 0.0):
        """Plane: block speed v and initial displacement; cylinder and annulus: rotor angular speed v
        and initial angle delta0."""
        if getattr(self.problem, "geom", 0) in (synth.GEOM_CYLINDER, synth.GEOM_ANNULAR, synth.GEOM_CONE):
            mo = SmMotion(0.0, float(v), float(delta0))
        else:
            mo = SmMotion(float(v), 0.0, float(delta0))
        check(lib().sm_set_motion(self.h, C.byref(mo)), "sm_set_motion")

    def init_state(self, stream=None):
        check(lib().sm_init_state(self.h, _stream(stream)), "sm_init_state")

    def set_state(self, U, t: float = 0.0, stream=None):
        """U: torch tensor (cuda or pinned/pageable cpu) or numpy array in solver precision."""
        import torch
        if isinstance(U, np.ndarray):
            U = torch.from_numpy(np.ascontiguousarray(U, dtype=self.dtype_np))
        assert U.dtype == self.torch_dtype and U.is_contiguous() and U.numel() == self.size
        check(lib().sm_set_state(self.h, U.data_ptr(), int(U.is_cuda), float(t), _stream(stream)), "sm_set_state")
        return U

    def get_state(self, out=None, stream=None):
        import torch
        if out is None:
            out = torch.empty(self.shape(), dtype=self.torch_dtype, device="cuda")
        t = C.c_double()
        check(lib().sm_get_state(self.h, out.data_ptr(), int(out.is_cuda), C.byref(t), _stream(stream)),
              "sm_get_state")
        return out, t.value

    def rhs(self, dU, t: float, out=None, stream=None):
        import torch
        assert dU.is_cuda and dU.dtype == self.torch_dtype and dU.is_contiguous() and dU.numel() == self.size
        if out is None:
            out = torch.empty_like(dU)
        check(lib().sm_rhs(self.h, float(t), dU.data_ptr(), out.data_ptr(), _stream(stream)), "sm_rhs")
        return out

    def interface(self, dU, t: float, stream=None):
        import torch
        p = self.problem
        shp = (p.nel_s[2], p.nel_s[1], 5, p.N + 1, p.N + 1)
        Fs = torch.empty(shp, dtype=self.torch_dtype, device=dU.device)
        Fm = torch.empty(shp, dtype=self.torch_dtype, device=dU.device)
        check(lib().sm_interface(self.h, float(t), dU.data_ptr(), Fs.data_ptr(), Fm.data_ptr(), _stream(stream)),
              "sm_interface")
        return Fs, Fm

    def gradients(self, dU, t: float, stream=None):
        """BR1-lifted gradients of the primitive variables, shape (E, 3, 5, np^3)."""
        import torch
        out = torch.empty((self.E, 3, 5, self.nn), dtype=self.torch_dtype, device=dU.device)
        check(lib().sm_gradients(self.h, float(t), dU.data_ptr(), out.data_ptr(), _stream(stream)), "sm_gradients")
        return out

    def step(self, dt: float, nsteps: int, stream=None):
        check(lib().sm_step(self.h, float(dt), int(nsteps), _stream(stream)), "sm_step")

    def stream_jobs(self, inputs, outputs, t0: float, dt: float, nsteps: int, count=None, stream=None):
        """sm_stream_jobs: inputs / outputs are CPU tensors (pinned for overlap) holding count
        states each ([count, *shape]), or one state each, which every job then reuses."""
        for x in (inputs, outputs):
            assert not x.is_cuda and x.dtype == self.torch_dtype and x.is_contiguous()
            assert x.numel() % self.size == 0
        n_in, n_out = inputs.numel() // self.size, outputs.numel() // self.size
        if count is None:
            count = max(n_in, n_out)
        assert n_in in (1, count) and n_out in (1, count)
        state_bytes = self.size * inputs.element_size()
        check(lib().sm_stream_jobs(self.h, inputs.data_ptr(), state_bytes if n_in > 1 else 0, outputs.data_ptr(),
                                   state_bytes if n_out > 1 else 0, int(count), float(t0), float(dt), int(nsteps),
                                   _stream(stream)), "sm_stream_jobs")
        return outputs

    def step_profiled(self, dt: float, nsteps: int, stream=None):
        """Per-kernel device times (ms) and launch counts of nsteps steps: mapper, interface, element."""
        ms = (C.c_double * 3)()
        cnt = (C.c_int * 3)()
        check(lib().sm_step_profiled(self.h, float(dt), int(nsteps), _stream(stream), ms, cnt), "sm_step_profiled")
        return list(ms), list(cnt)

    def diag(self, stream=None) -> dict:
        d = SmDiag()
        st = lib().sm_diag(self.h, C.byref(d), _stream(stream))
        out = {"n_delta": d.n_delta, "s_delta": d.s_delta, "t": d.t, "totals": list(d.totals),
               "iface_sum_static": list(d.iface_sum_static), "iface_sum_moving": list(d.iface_sum_moving),
               "status": st}
        if st not in (SM_OK, -4):
            check(st, "sm_diag")
        return out


class Batch:
    """Several FP32 solvers advanced by shared launches (sm_batch_*)."""

    def __init__(self, solvers, dts):
        self.solvers = list(solvers)
        arr = (C.c_void_p * len(self.solvers))(*[s.h.value for s in self.solvers])
        dt = (C.c_double * len(self.solvers))(*[float(x) for x in dts])
        h = C.c_void_p()
        check(lib().sm_batch_create(arr, dt, len(self.solvers), C.byref(h)), "sm_batch_create")
        self.h = h

    def autotune(self, stream=None):
        check(lib().sm_batch_autotune(self.h, _stream(stream)), "sm_batch_autotune")

    def step(self, nsteps, stream=None):
        check(lib().sm_batch_step(self.h, int(nsteps), _stream(stream)), "sm_batch_step")

    def shapes(self):
        out, g = [], 0
        while True:
            sh = (C.c_int * 4)()
            n = lib().sm_batch_shapes(self.h, g, sh)
            if n < 0:
                break
            out.append({"N": sh[0], "tile_faces": sh[1], "grid_interface": sh[2], "grid_element": sh[3]})
            g += 1
            if g >= n:
                break
        return out

    def close(self):
        if getattr(self, "h", None):
            lib().sm_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous-batching request loop (sm_server_*)."""

    def __init__(self, hbm_budget_bytes: int, max_slots: int):
        h = C.c_void_p()
        check(lib().sm_server_create(C.c_size_t(int(hbm_budget_bytes)), int(max_slots), C.byref(h)),
              "sm_server_create")
        self.h = h

    def submit(self, problem: synth.Problem, dt: float, nsteps: int, keep_state: bool = False) -> int:
        req = SmRequest()
        req.desc = mesh_desc(problem)
        if getattr(problem, "geom", 0) in (synth.GEOM_CYLINDER, synth.GEOM_ANNULAR, synth.GEOM_CONE):
            req.motion = SmMotion(0.0, float(problem.v), float(problem.delta0))
        else:
            req.motion = SmMotion(float(problem.v), 0.0, float(problem.delta0))
        req.dt, req.nsteps, req.keep_state = float(dt), int(nsteps), int(keep_state)
        t = C.c_uint64()
        check(lib().sm_submit(self.h, C.byref(req), C.byref(t)), "sm_submit")
        return t.value

    def poll(self, ticket: int) -> dict:
        r = SmResult()
        st = lib().sm_poll(self.h, C.c_uint64(ticket), C.byref(r))
        out = {"status": st, "t_submit": r.t_submit, "t_admit": r.t_admit, "t_done": r.t_done,
               "sim_time": r.sim_time, "dof": r.dof, "steps": r.steps, "totals": list(r.totals)}
        if r.state and r.state_bytes:
            out["state"] = bytes(C.string_at(r.state, r.state_bytes))
        return out

    def wait(self, timeout_s: float = 600.0):
        check(lib().sm_server_wait(self.h, float(timeout_s)), "sm_server_wait")

    def stats(self) -> dict:
        s = SmServerStats()
        check(lib().sm_server_stats(self.h, C.byref(s)), "sm_server_stats")
        return {k: getattr(s, k) for k, _ in SmServerStats._fields_}

    def close(self):
        if getattr(self, "h", None):
            lib().sm_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
