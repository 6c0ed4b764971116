"""ctypes wrapper of the CPU oracle (test infrastructure only).

Only tests/, __graft_entry__.smoke() and the CPU-baseline leg of bench.py may import this
module.  It loads oracle/liboracle.so (built from dg_oracle.cpp by oracle/build.py) and
reads the problem description from paper_2008_04356_gb300.synth, the shared input module.
"""
from __future__ import annotations

import ctypes as C
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))

from oracle.build import build_oracle  # noqa: E402

_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int)
_llp = C.POINTER(C.c_longlong)


class OrcProblem(C.Structure):
    _fields_ = [("N", C.c_int), ("nel_s", C.c_int * 3), ("nel_m", C.c_int * 3),
                ("x0", C.c_double), ("x1", C.c_double), ("x2", C.c_double),
                ("y0", C.c_double), ("y1", C.c_double), ("z0", C.c_double), ("z1", C.c_double),
                ("v", C.c_double), ("delta0", C.c_double), ("gamma", C.c_double),
                ("riemann", C.c_int), ("interface_conforming", C.c_int), ("flow", C.c_int),
                ("fpar", C.c_double * 16), ("modes", C.c_double * 160),
                ("physics", C.c_int), ("mu", C.c_double), ("Pr", C.c_double), ("Rgas", C.c_double),
                ("geom", C.c_int), ("volume", C.c_int), ("periodic_x", C.c_int), ("cone_angle", C.c_double)]


_LIB = None


def lib():
    global _LIB
    if _LIB is None:
        L = C.CDLL(build_oracle())
        L.orc_lgl.argtypes = [C.c_int, _dp, _dp]
        L.orc_gl.argtypes = [C.c_int, _dp, _dp]
        L.orc_lagrange.argtypes = [C.c_int, _dp, C.c_double, _dp]
        L.orc_dmatrix.argtypes = [C.c_int, _dp, _dp]
        L.orc_mass_exact.argtypes = [C.c_int, _dp]
        L.orc_map_closed.argtypes = [C.c_double, C.c_double, _llp, _dp]
        L.orc_map_pairs.argtypes = [C.c_longlong, C.c_int, _ip]
        L.orc_map_bruteforce.argtypes = [C.c_double, C.c_double, C.c_int, _llp, _dp, _ip]
        L.orc_map_bruteforce.restype = C.c_int
        L.orc_mortar_mats.argtypes = [C.c_int, C.c_double, _dp, _dp, _dp, _dp]
        L.orc_euler_flux.argtypes = [_dp, _dp, C.c_double, C.c_double, _dp]
        L.orc_riemann.argtypes = [C.c_int, _dp, _dp, _dp, C.c_double, C.c_double, _dp]
        L.orc_two_point_flux.argtypes = [C.c_int, _dp, _dp, _dp, C.c_double, C.c_double, _dp]
        L.orc_lsrk_coeffs.argtypes = [_dp, _dp, _dp]
        L.orc_create.argtypes = [C.POINTER(OrcProblem)]
        L.orc_create.restype = C.c_void_p
        L.orc_destroy.argtypes = [C.c_void_p]
        L.orc_nelem.argtypes = [C.c_void_p]
        L.orc_nelem.restype = C.c_longlong
        L.orc_node_coords.argtypes = [C.c_void_p, C.c_double, _dp]
        L.orc_init_state.argtypes = [C.c_void_p, _dp]
        L.orc_exact_state.argtypes = [C.c_void_p, C.c_double, _dp]
        L.orc_rhs.argtypes = [C.c_void_p, _dp, C.c_double, _dp]
        L.orc_rhs_elements.argtypes = [C.c_void_p, _dp, C.c_double, _llp, C.c_int, _dp]
        L.orc_interface_fluxes.argtypes = [C.c_void_p, _dp, C.c_double, _dp, _dp]
        L.orc_step.argtypes = [C.c_void_p, _dp, _dp, _dp, C.c_double, C.c_int]
        L.orc_totals.argtypes = [C.c_void_p, _dp, _dp]
        L.orc_lifting.argtypes = [C.c_void_p, _dp, C.c_double, _dp]
        L.orc_viscous_flux.argtypes = [_dp, _dp, C.c_double, C.c_double, C.c_double, C.c_double, _dp]
        L.orc_face_flux_sums.argtypes = [C.POINTER(OrcProblem), _dp, _dp, _dp, _dp]
        L.orc_l2_error_rho.argtypes = [C.c_void_p, _dp, C.c_double]
        L.orc_l2_error_rho.restype = C.c_double
        L.orc_num_threads.restype = C.c_int
        L.orc_metrics.argtypes = [C.c_void_p, C.c_double, _dp, _dp]
        L.orc_flow_state.argtypes = [C.POINTER(OrcProblem), _dp, C.c_double, C.c_int, _dp]
        _LIB = L
    return _LIB


def _p(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_dp)


def lgl(N):
    x, w = np.zeros(N + 1), np.zeros(N + 1)
    lib().orc_lgl(N, _p(x), _p(w))
    return x, w


def gl(N):
    x, w = np.zeros(N + 1), np.zeros(N + 1)
    lib().orc_gl(N, _p(x), _p(w))
    return x, w


def lagrange(N, nodes, x):
    nodes = np.ascontiguousarray(nodes, dtype=np.float64)
    out = np.zeros(N + 1)
    lib().orc_lagrange(N, _p(nodes), float(x), _p(out))
    return out


def dmatrix(N, nodes):
    nodes = np.ascontiguousarray(nodes, dtype=np.float64)
    D = np.zeros((N + 1, N + 1))
    lib().orc_dmatrix(N, _p(nodes), _p(D))
    return D


def mass_exact(N):
    M = np.zeros((N + 1, N + 1))
    lib().orc_mass_exact(N, _p(M))
    return M


def map_closed(delta, l):
    n, s = C.c_longlong(), C.c_double()
    lib().orc_map_closed(float(delta), float(l), C.byref(n), C.byref(s))
    return n.value, s.value


def map_pairs(n, n_par):
    pairs = np.zeros(2 * n_par, dtype=np.int32)
    lib().orc_map_pairs(int(n), int(n_par), pairs.ctypes.data_as(_ip))
    return pairs.reshape(n_par, 2)


def map_bruteforce(delta, l, n_par):
    n, s = C.c_longlong(), C.c_double()
    pairs = np.zeros(2 * n_par, dtype=np.int32)
    rc = lib().orc_map_bruteforce(float(delta), float(l), int(n_par), C.byref(n), C.byref(s),
                                  pairs.ctypes.data_as(_ip))
    return rc, n.value, s.value, pairs.reshape(n_par, 2)


def mortar_mats(N, sigma):
    mats = [np.zeros((N + 1, N + 1)) for _ in range(4)]
    lib().orc_mortar_mats(N, float(sigma), *[_p(m) for m in mats])
    return mats  # P_lo, P_hi, B_lo, B_hi


def euler_flux(U, n, vgn, gamma=1.4):
    U = np.ascontiguousarray(U, dtype=np.float64)
    n = np.ascontiguousarray(n, dtype=np.float64)
    F = np.zeros(5)
    lib().orc_euler_flux(_p(U), _p(n), float(vgn), float(gamma), _p(F))
    return F


def riemann(kind, UL, UR, n, vgn=0.0, gamma=1.4):
    UL = np.ascontiguousarray(UL, dtype=np.float64)
    UR = np.ascontiguousarray(UR, dtype=np.float64)
    n = np.ascontiguousarray(n, dtype=np.float64)
    F = np.zeros(5)
    lib().orc_riemann(int(kind), _p(UL), _p(UR), _p(n), float(vgn), float(gamma), _p(F))
    return F


def two_point_flux(kind, UL, UR, n, vgn=0.0, gamma=1.4):
    """Split-form volume flux F#(UL, UR) along n: kind 0 Pirozzoli, 1 central."""
    UL = np.ascontiguousarray(UL, dtype=np.float64)
    UR = np.ascontiguousarray(UR, dtype=np.float64)
    n = np.ascontiguousarray(n, dtype=np.float64)
    F = np.zeros(5)
    lib().orc_two_point_flux(int(kind), _p(UL), _p(UR), _p(n), float(vgn), float(gamma), _p(F))
    return F


def viscous_flux(U, grad15, mu, Pr, Rgas, gamma=1.4):
    U = np.ascontiguousarray(U, dtype=np.float64)
    g = np.ascontiguousarray(grad15, dtype=np.float64)
    F = np.zeros(15)
    lib().orc_viscous_flux(_p(U), _p(g), float(mu), float(Pr), float(Rgas), float(gamma), _p(F))
    return F.reshape(3, 5)


def lsrk_coeffs():
    A, B, c = np.zeros(5), np.zeros(5), np.zeros(5)
    lib().orc_lsrk_coeffs(_p(A), _p(B), _p(c))
    return A, B, c


def num_threads() -> int:
    return int(lib().orc_num_threads())


def to_orc_problem(p) -> OrcProblem:
    s = OrcProblem()
    s.N = p.N
    for k in range(3):
        s.nel_s[k] = int(p.nel_s[k])
        s.nel_m[k] = int(p.nel_m[k])
    for name in ("x0", "x1", "x2", "y0", "y1", "z0", "z1", "v", "delta0", "gamma"):
        setattr(s, name, float(getattr(p, name)))
    s.riemann = int(p.riemann)
    s.interface_conforming = int(p.interface_conforming)
    s.flow = int(p.flow)
    for k, f in enumerate(p.fpar16()):
        s.fpar[k] = f
    for k, m in enumerate(p.modes_array().ravel()):
        s.modes[k] = m
    s.physics = int(p.physics)
    s.mu, s.Pr, s.Rgas = float(p.mu), float(p.Pr), float(p.Rgas)
    s.geom = int(getattr(p, "geom", 0))
    s.volume = int(getattr(p, "volume", 0))
    s.periodic_x = int(getattr(p, "periodic_x", 0))
    s.cone_angle = float(getattr(p, "cone_angle", 0.0))
    return s


class Oracle:
    """The FP64 CPU operator for one problem (a synth.Problem)."""

    def __init__(self, problem):
        self.problem = problem
        self._s = to_orc_problem(problem)
        self.h = lib().orc_create(C.byref(self._s))
        if not self.h:
            raise ValueError("oracle rejected the problem description")
        self.N = problem.N
        self.np_ = problem.N + 1
        self.nn = self.np_ ** 3
        self.E = int(lib().orc_nelem(self.h))

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            lib().orc_destroy(h)
            self.h = None

    def shape(self):
        return (self.E, 5, self.nn)

    def zeros(self):
        return np.zeros(self.shape())

    def coords(self, t=0.0):
        X = np.zeros((self.E, 3, self.nn))
        lib().orc_node_coords(self.h, float(t), _p(X))
        return X

    def init_state(self):
        U = self.zeros()
        lib().orc_init_state(self.h, _p(U))
        return U

    def exact_state(self, t):
        U = self.zeros()
        lib().orc_exact_state(self.h, float(t), _p(U))
        return U

    def rhs(self, U, t):
        U = np.ascontiguousarray(U, dtype=np.float64)
        Ut = self.zeros()
        lib().orc_rhs(self.h, _p(U), float(t), _p(Ut))
        return Ut

    def rhs_elements(self, U, t, elems):
        U = np.ascontiguousarray(U, dtype=np.float64)
        el = np.ascontiguousarray(elems, dtype=np.int64)
        Ut = np.zeros((len(el), 5, self.nn))
        lib().orc_rhs_elements(self.h, _p(U), float(t), el.ctypes.data_as(_llp), len(el), _p(Ut))
        return Ut

    def interface_fluxes(self, U, t):
        """Face fluxes of both sides, (nz, ny, 5, np, np) each; with periodic x the two
        interfaces, (2, nz, ny, 5, np, np): x = x1 first, then x = x0 = x2."""
        U = np.ascontiguousarray(U, dtype=np.float64)
        p = self.problem
        shp = (p.nel_s[2], p.nel_s[1], 5, self.np_, self.np_)
        if getattr(p, "periodic_x", 0):
            shp = (2,) + shp
        Fs, Fm = np.zeros(shp), np.zeros(shp)
        lib().orc_interface_fluxes(self.h, _p(U), float(t), _p(Fs), _p(Fm))
        return Fs, Fm

    def step(self, U, G, t, dt, nsteps):
        """Advance U (and the RK register G) in place; returns the new time."""
        assert U.dtype == np.float64 and G.dtype == np.float64
        tt = C.c_double(t)
        lib().orc_step(self.h, _p(U), _p(G), C.byref(tt), float(dt), int(nsteps))
        return tt.value

    def metrics(self, t=0.0):
        """Ja^i_n at the nodes, shape (E, 3 (i), 3 (n), np^3), and J, shape (E, np^3)."""
        Ja = np.zeros((self.E, 3, 3, self.nn))
        J = np.zeros((self.E, self.nn))
        lib().orc_metrics(self.h, float(t), _p(Ja), _p(J))
        return Ja, J

    def lifting(self, U, t):
        """BR1 gradients of the primitive variables, shape (E, 3, 5, np^3)."""
        U = np.ascontiguousarray(U, dtype=np.float64)
        g = np.zeros((self.E, 3, 5, self.nn))
        lib().orc_lifting(self.h, _p(U), float(t), _p(g))
        return g

    def totals(self, U):
        U = np.ascontiguousarray(U, dtype=np.float64)
        out = np.zeros(5)
        lib().orc_totals(self.h, _p(U), _p(out))
        return out

    def face_flux_sums(self, Fs, Fm):
        Fs = np.ascontiguousarray(Fs, dtype=np.float64)
        Fm = np.ascontiguousarray(Fm, dtype=np.float64)
        ss, sm = np.zeros(5), np.zeros(5)
        lib().orc_face_flux_sums(C.byref(self._s), _p(Fs), _p(Fm), _p(ss), _p(sm))
        return ss, sm

    def l2_error_rho(self, U, t):
        U = np.ascontiguousarray(U, dtype=np.float64)
        return float(lib().orc_l2_error_rho(self.h, _p(U), float(t)))
