"""Workload descriptions and seeded synthetic inputs.

This module holds configuration and random-number generation only; none of the method's
arithmetic lives here.  It is the one module both the CUDA path's tests/benchmark and the
CPU oracle read, so that both sides see the same problem and the same random inputs.

Random numbers come from SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014) used as a counter-based generator: the k-th draw of a
stream with seed S is mix(S * 2^32 + k), uniform doubles take the top 53 bits.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
M1 = np.uint64(0xBF58476D1CE4E5B9)
M2 = np.uint64(0x94D049BB133111EB)

FLOW_CONSTANT, FLOW_ENTROPY_WAVE, FLOW_MODES, FLOW_POLY_X, FLOW_SHEAR_X = 0, 1, 2, 3, 4
FLOW_AXIAL_PULSE, FLOW_RIGID_ROTATION = 5, 6
GEOM_PLANE, GEOM_CYLINDER, GEOM_PLANE_CURVILINEAR, GEOM_ANNULAR, GEOM_CONE = 0, 1, 2, 3, 4
EULER, NAVIER_STOKES = 0, 1
RUSANOV, ROE_HH = 0, 1
FP64, FP32 = 0, 1
VOLUME_WEAK, VOLUME_SPLIT = 0, 1       # weak-form DGSEM; split form with Pirozzoli's flux


def splitmix64(counters: np.ndarray) -> np.ndarray:
    """SplitMix64 output for each 64-bit counter value (vectorised, wraps mod 2^64)."""
    with np.errstate(over="ignore"):
        z = counters.astype(np.uint64) * GOLDEN + GOLDEN
        z = (z ^ (z >> np.uint64(30))) * M1
        z = (z ^ (z >> np.uint64(27))) * M2
        return z ^ (z >> np.uint64(31))


def uniform(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """count uniform doubles in [0, 1) from stream `seed`, draws offset..offset+count-1."""
    base = np.uint64((seed & 0xFFFFFFFF) << 32)
    k = np.arange(offset, offset + count, dtype=np.uint64) + base
    return (splitmix64(k) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


@dataclasses.dataclass
class Problem:
    """Two structured hexahedral blocks sharing the plane sliding interface x = x1.

    Static block: x in [x0, x1]; moving block: x in [x1, x2]; both y in [y0, y1],
    z in [z0, z1], periodic in y and z.  The moving block translates along +y with speed v
    (displacement delta0 + v t).  Boundaries x = x0 and x = x2 take the flow's exact (or
    background) state weakly.

    geom GEOM_CYLINDER: the cylindrical sliding interface; x0 < x1 < x2 are radii (block 0,
    the rotor, inside), [y0, y1] the periodic angular sector, v the rotor's angular speed and
    delta0 its initial angle; walls r = x0, x2 are slip walls.  GEOM_PLANE_CURVILINEAR: the
    plane box through the curvilinear operator (general metrics).

    periodic_x = 1 closes the box in x (period x2 - x0): the moving block's face x = x2 meets
    the static block's face x = x0 in a second sliding interface (no Dirichlet faces).
    """
    N: int = 3
    nel_s: tuple = (4, 4, 2)
    nel_m: tuple = (4, 4, 2)
    x0: float = 0.0
    x1: float = 1.0
    x2: float = 2.0
    y0: float = 0.0
    y1: float = 1.0
    z0: float = 0.0
    z1: float = 1.0
    v: float = 0.5
    delta0: float = 0.0
    gamma: float = 1.4
    riemann: int = RUSANOV
    interface_conforming: int = 0
    flow: int = FLOW_ENTROPY_WAVE
    fpar: tuple = (1.0, 0.2, 1.0, 1.0, 1.0, 0.3, 0.0, 0.0, 1.0)
    modes: Optional[np.ndarray] = None          # (5, 8, 4): amp, ky, kz, phase
    precision: int = FP64
    physics: int = EULER
    mu: float = 0.0
    Pr: float = 0.72
    Rgas: float = 1.0
    geom: int = GEOM_PLANE
    volume: int = VOLUME_WEAK
    periodic_x: int = 0          # 1: x periodic, a second sliding interface at x0 = x2
    cone_angle: float = 0.0      # GEOM_CONE: half-angle of the conical interface from the z axis

    @property
    def np_(self) -> int:
        return self.N + 1

    @property
    def nelem(self) -> int:
        ny, nz = self.nel_s[1], self.nel_s[2]
        return (self.nel_s[0] + self.nel_m[0]) * ny * nz

    @property
    def ndof(self) -> int:
        return self.nelem * self.np_ ** 3

    @property
    def n_faces(self) -> int:
        return self.nel_s[1] * self.nel_s[2]

    def fpar16(self) -> List[float]:
        f = list(self.fpar) + [0.0] * 16
        return f[:16]

    def modes_array(self) -> np.ndarray:
        if self.modes is None:
            return np.zeros((5, 8, 4))
        return np.asarray(self.modes, dtype=np.float64).reshape(5, 8, 4)


# ---------------------------------------------------------------------------------------
# The workloads (sizes, flows and motion of the five configurations of the study).
# ---------------------------------------------------------------------------------------

def config_box(N: int = 3, k: Optional[int] = None, flow: str = "wave", v: float = 0.5,
               precision: int = FP64, riemann: int = RUSANOV) -> Problem:
    """[0,2]x[0,1]x[0,1] split at x = 1, moving right block (+y at v).

    k=None gives the 8x4x2 mesh (4x4x2 per block); an integer k gives k^3 per block.
    flow "wave": rho = 1 + 0.2 sin(2 pi (x + y + z)), u = (0.3, 0, 0), p = 1.
    flow "free": rho = 1, u = (0.5, 0.2, 0.1), p = 1.
    """
    nel = (4, 4, 2) if k is None else (k, k, k)
    p = Problem(N=N, nel_s=nel, nel_m=nel, v=v, precision=precision, riemann=riemann)
    if flow == "free":
        p.flow = FLOW_CONSTANT
        p.fpar = (1.0, 0.5, 0.2, 0.1, 1.0)
    elif flow != "wave":
        raise ValueError(flow)
    return p


def fourier_modes(seed: int, n_modes: int = 8, amp: float = 0.05, kmax: int = 4) -> np.ndarray:
    """Per primitive variable, n_modes modes amp * sin(2 pi (ky y + kz z) + phase) with
    integer (ky, kz) in [-kmax, kmax]^2 \\ {0} and phase in [0, 2 pi), drawn from stream seed."""
    u = uniform(seed, 5 * n_modes * 3).reshape(5, n_modes, 3)
    modes = np.zeros((5, 8, 4))
    for var in range(5):
        for m in range(n_modes):
            ky = int(math.floor(u[var, m, 0] * (2 * kmax + 1))) - kmax
            kz = int(math.floor(u[var, m, 1] * (2 * kmax + 1))) - kmax
            if ky == 0 and kz == 0:
                ky = 1
            modes[var, m] = (amp, ky, kz, 2.0 * math.pi * u[var, m, 2])
    return modes


def config_interface_heavy(seed: int = 1, precision: int = FP32, nz: int = 256, ny: int = 256,
                           nx: int = 4, N: int = 5, v: float = 0.37) -> Problem:
    """Interface-heavy single solve: two blocks of nx x ny x nz hexes (4 x 256 x 256) with
    h = 1/ny, N = 5, v = 0.37 (not commensurate with the face size), rho = 1, p = 1 background plus
    8 seeded Fourier modes of amplitude 0.05 per primitive variable."""
    h = 1.0 / ny
    return Problem(N=N, nel_s=(nx, ny, nz), nel_m=(nx, ny, nz), x0=0.0, x1=nx * h, x2=2 * nx * h,
                   y0=0.0, y1=ny * h, z0=0.0, z1=nz * h,
                   v=v, flow=FLOW_MODES, fpar=(1.0, 0.0, 0.0, 0.0, 1.0),
                   modes=fourier_modes(seed), precision=precision)


def config_shear_x(N: int = 3, v: float = 0.5, mu: float = 0.01, w=(0.1, 0.3, -0.2),
                   rho: float = 1.0, p: float = 1.0) -> Problem:
    """Navier-Stokes, rho and p constant, velocity (0, 0, w(x)) with w quadratic in x."""
    return Problem(N=N, nel_s=(3, 4, 2), nel_m=(2, 4, 2), v=v, flow=FLOW_SHEAR_X,
                   fpar=(rho, p) + tuple(w), physics=NAVIER_STOKES, mu=mu)


def config_cylinder(N: int = 3, nel=(3, 8, 2), omega: float = 0.4, phi0: float = 0.0,
                    r=(1.0, 1.25, 1.5), sector: float = math.pi / 4, z=(0.0, 0.5),
                    flow: str = "pulse", mach: float = 0.3, precision: int = FP64,
                    physics: int = EULER, reynolds: float = 1.0e4) -> Problem:
    """Cylindrical sliding interface: rotor r in [r0, r1] inside, stator r in [r1, r2],
    angular sector [0, sector] periodic, z periodic, nel = (radial per block, angular, axial).
    flow "pulse": axial stream Mach `mach` (rho = 1, p = 1) with a pressure pulse of 1e-2
    at the interface; "rotation": rigid rotation with the rotor's angular speed; "free":
    uniform axial stream.  Navier-Stokes: mu = rho |u| L / Re with L the axial length."""
    c = math.sqrt(1.4)
    w = mach * c
    if flow == "pulse":
        fl, fpar = FLOW_AXIAL_PULSE, (1.0, 1.0, w, 1.0e-2, r[1], 0.5 * sector, 0.5 * (z[0] + z[1]), 0.05)
    elif flow == "rotation":
        fl, fpar = FLOW_RIGID_ROTATION, (1.0, 1.0, omega)
    else:
        fl, fpar = FLOW_CONSTANT, (1.0, 0.0, 0.0, w, 1.0)
    mu = 1.0 * w * (z[1] - z[0]) / reynolds if physics == NAVIER_STOKES else 0.0
    return Problem(N=N, nel_s=(nel[0], nel[1], nel[2]), nel_m=(nel[0], nel[1], nel[2]),
                   x0=r[0], x1=r[1], x2=r[2], y0=0.0, y1=sector, z0=z[0], z1=z[1],
                   v=omega, delta0=phi0, flow=fl, fpar=fpar, precision=precision,
                   physics=physics, mu=mu, geom=GEOM_CYLINDER)


def config_annular(N: int = 3, nel=(2, 8, 2), omega: float = 0.4, phi0: float = 0.0,
                   z=(0.0, 0.25, 0.5), sector: float = math.pi / 4, r=(1.0, 1.5),
                   flow: str = "pulse", precision: int = FP64) -> Problem:
    """Plane annular sliding interface normal to the rotation axis: rotor z in [z0, z1]
    below the stator z in [z1, z2], radii [r0, r1], angular sector [0, sector] periodic, slip
    walls at both radii and at both axial ends; nel = (axial per block, angular, radial).
    flow "pulse": fluid at rest (rho = 1, p = 1) with a Gaussian pressure pulse of 1e-2 on
    the interface; "rotation": rigid rotation with the rotor's angular speed (a steady
    solution); "rest": uniform state at rest."""
    if flow == "pulse":
        fl, fpar = FLOW_AXIAL_PULSE, (1.0, 1.0, 0.0, 1.0e-2, 0.5 * (r[0] + r[1]), 0.5 * sector, z[1], 0.08)
    elif flow == "rotation":
        fl, fpar = FLOW_RIGID_ROTATION, (1.0, 1.0, omega)
    else:
        fl, fpar = FLOW_CONSTANT, (1.0, 0.0, 0.0, 0.0, 1.0)
    return Problem(N=N, nel_s=(nel[0], nel[1], nel[2]), nel_m=(nel[0], nel[1], nel[2]),
                   x0=z[0], x1=z[1], x2=z[2], y0=0.0, y1=sector, z0=r[0], z1=r[1],
                   v=omega, delta0=phi0, flow=fl, fpar=fpar, precision=precision, geom=GEOM_ANNULAR)


def cone_radii(p: Problem):
    """Smallest and largest radius of a conical mesh (at the corners of its (s, n) ranges)."""
    sa, ca = math.sin(p.cone_angle), math.cos(p.cone_angle)
    rs = [s * sa + n * ca for s in (p.z0, p.z1) for n in (p.x0, p.x2)]
    return min(rs), max(rs)


def config_cone(N: int = 3, nel=(2, 8, 2), omega: float = 0.4, phi0: float = 0.0, alpha: float = math.pi / 6,
                n=(1.0, 1.25, 1.5), s=(0.0, 0.5), sector: float = math.pi / 4, flow: str = "pulse",
                precision: int = FP64) -> Problem:
    """Conical sliding interface about the z axis with half-angle alpha: a point of
    generator coordinate s and normal offset n lies at radius s sin(alpha) + n cos(alpha),
    height s cos(alpha) - n sin(alpha); rotor n in [n0, n1] inside, stator [n1, n2]; angular
    sector periodic, slip walls at the ends of s and n; nel = (normal per block, angular,
    along the generator).  Flows as for config_annular."""
    p = Problem(N=N, nel_s=(nel[0], nel[1], nel[2]), nel_m=(nel[0], nel[1], nel[2]),
                x0=n[0], x1=n[1], x2=n[2], y0=0.0, y1=sector, z0=s[0], z1=s[1],
                v=omega, delta0=phi0, precision=precision, geom=GEOM_CONE, cone_angle=alpha)
    sa, ca = math.sin(alpha), math.cos(alpha)
    if flow == "pulse":
        sm, nm = 0.5 * (s[0] + s[1]), n[1]
        p.flow = FLOW_AXIAL_PULSE
        p.fpar = (1.0, 1.0, 0.0, 1.0e-2, sm * sa + nm * ca, 0.5 * sector, sm * ca - nm * sa, 0.08)
    elif flow == "rotation":
        p.flow, p.fpar = FLOW_RIGID_ROTATION, (1.0, 1.0, omega)
    else:
        p.flow, p.fpar = FLOW_CONSTANT, (1.0, 0.0, 0.0, 0.0, 1.0)
    return p


def config_poly_x(N: int = 3, v: float = 0.5, coeffs=(1.0, 0.1, -0.05, 0.02),
                  vel=(0.3, 0.2, -0.1), p: float = 1.0) -> Problem:
    """State polynomial in x (degree <= 3) with constant velocity and pressure."""
    return Problem(N=N, nel_s=(3, 4, 2), nel_m=(2, 4, 2), v=v, flow=FLOW_POLY_X,
                   fpar=tuple(coeffs) + tuple(vel) + (p,))


# ---------------------------------------------------------------------------------------
# Time step (fixed once per run, from bounds of the initial flow)
# ---------------------------------------------------------------------------------------

def wave_speed_bounds(p: Problem):
    """Upper bounds of |v_d| (d = x, y, z) and of the sound speed over the initial flow."""
    g = p.gamma
    f = list(p.fpar)
    if p.flow == FLOW_CONSTANT:
        rho_min, pmax, vel = f[0], f[4], [abs(f[1]), abs(f[2]), abs(f[3])]
    elif p.flow == FLOW_ENTROPY_WAVE:
        rho_min, pmax, vel = f[0] - abs(f[1]), f[8], [abs(f[5]), abs(f[6]), abs(f[7])]
    elif p.flow == FLOW_MODES:
        a = np.abs(p.modes_array()[:, :, 0]).sum(axis=1)
        rho_min, pmax = f[0] - a[0], f[4] + a[4]
        vel = [abs(f[1]) + a[1], abs(f[2]) + a[2], abs(f[3]) + a[3]]
    elif p.flow == FLOW_AXIAL_PULSE:
        rho_min, pmax, vel = f[0], f[1] + abs(f[3]), [0.0, 0.0, abs(f[2])]
    elif p.flow == FLOW_RIGID_ROTATION:
        rmax = (max(abs(p.z0), abs(p.z1)) if p.geom == GEOM_ANNULAR else
                (cone_radii(p)[1] if p.geom == GEOM_CONE else max(abs(p.x0), abs(p.x2))))
        w = abs(f[2]) * rmax
        rho_min, pmax, vel = f[0], f[1] + 0.5 * f[0] * w * w, [w, w, 0.0]
    elif p.flow == FLOW_POLY_X:
        c = f[:4]
        rho_min = min(c[0] + x * (c[1] + x * (c[2] + x * c[3])) for x in np.linspace(p.x0 - 1, p.x2, 401))
        pmax, vel = f[7], [abs(f[4]), abs(f[5]), abs(f[6])]
    else:
        xs = np.linspace(p.x0, p.x2, 401)
        rho_min, pmax = f[0], f[1]
        vel = [0.0, 0.0, float(np.abs(f[2] + xs * (f[3] + xs * f[4])).max())]
    return vel, math.sqrt(g * pmax / rho_min)


def cfl_dt(p: Problem, cfl: float = 0.9) -> float:
    """dt = CFL / ((2N+1) * sum_d (|v_d - v^g_d| + c) / h_d), the largest over both blocks
    (grid velocity 0 in the static block, v along y in the moving one)."""
    vel, c = wave_speed_bounds(p)
    if p.geom == GEOM_CONE:
        # angular (arc length at the smallest radius), generator and normal sizes; the rotor's
        # grid speed is at most omega rho_max
        rmin, rmax = cone_radii(p)
        ha = rmin * (p.y1 - p.y0) / p.nel_s[1]
        hs = (p.z1 - p.z0) / p.nel_s[2]
        vmax = math.sqrt(vel[0] ** 2 + vel[1] ** 2 + vel[2] ** 2)
        rate = 0.0
        for hn, vg in (((p.x1 - p.x0) / p.nel_s[0], abs(p.v) * rmax), ((p.x2 - p.x1) / p.nel_m[0], 0.0)):
            rate = max(rate, (vmax + c) / hn + (vmax + vg + c) / ha + (vmax + c) / hs)
        return cfl / ((2 * p.N + 1) * rate)
    if p.geom == GEOM_ANNULAR:
        # angular (arc length at the inner radius), radial and axial sizes; the rotor's grid
        # speed is at most omega r1
        ha = p.z0 * (p.y1 - p.y0) / p.nel_s[1]
        hr = (p.z1 - p.z0) / p.nel_s[2]
        vmax = math.sqrt(vel[0] ** 2 + vel[1] ** 2 + vel[2] ** 2)
        rate = 0.0
        for hz, vg in (((p.x1 - p.x0) / p.nel_s[0], abs(p.v) * p.z1), ((p.x2 - p.x1) / p.nel_m[0], 0.0)):
            rate = max(rate, (vmax + c) / hz + (vmax + vg + c) / ha + (vmax + c) / hr)
        return cfl / ((2 * p.N + 1) * rate)
    if p.geom == GEOM_CYLINDER:
        # radial, angular (arc length at the inner radius) and axial sizes; the rotor's grid
        # speed is omega r
        ha = p.x0 * (p.y1 - p.y0) / p.nel_s[1]
        hz = (p.z1 - p.z0) / p.nel_s[2]
        vmax = math.sqrt(vel[0] ** 2 + vel[1] ** 2 + vel[2] ** 2)
        rate, hmin = 0.0, min(ha, hz)
        for hr, vg in (((p.x1 - p.x0) / p.nel_s[0], abs(p.v) * p.x1), ((p.x2 - p.x1) / p.nel_m[0], 0.0)):
            rate = max(rate, (vmax + c) / hr + (vmax + vg + c) / ha + (vmax + c) / hz)
            hmin = min(hmin, hr)
        dt = cfl / ((2 * p.N + 1) * rate)
        if p.physics == NAVIER_STOKES and p.mu > 0.0:
            nu = p.mu / p.fpar[0] * max(4.0 / 3.0, p.gamma / p.Pr)
            dt = min(dt, 0.5 * hmin * hmin / ((2 * p.N + 1) ** 2 * nu))
        return dt
    hy = (p.y1 - p.y0) / p.nel_s[1]
    hz = (p.z1 - p.z0) / p.nel_s[2]
    rate, hmin = 0.0, min(hy, hz)
    for hx, vg in (((p.x1 - p.x0) / p.nel_s[0], 0.0), ((p.x2 - p.x1) / p.nel_m[0], p.v)):
        r = (vel[0] + c) / hx + (vel[1] + abs(vg) + c) / hy + (vel[2] + c) / hz
        rate = max(rate, r)
        hmin = min(hmin, hx)
    dt = cfl / ((2 * p.N + 1) * rate)
    if p.physics == NAVIER_STOKES and p.mu > 0.0:
        # diffusive limit: dt <= 0.5 h^2 / ((2N+1)^2 nu_max), nu_max = mu/rho * max(4/3, gamma/Pr)
        rho_min = p.fpar[0] if p.flow in (FLOW_CONSTANT, FLOW_SHEAR_X, FLOW_MODES) else 0.5
        nu = p.mu / rho_min * max(4.0 / 3.0, p.gamma / p.Pr)
        dt = min(dt, 0.5 * hmin * hmin / ((2 * p.N + 1) ** 2 * nu))
    return dt


# ---------------------------------------------------------------------------------------
# Random inputs for parity tests
# ---------------------------------------------------------------------------------------

def random_state(p: Problem, seed: int) -> np.ndarray:
    """Conservative state drawn uniformly from a box that keeps density and pressure
    positive: rho in [0.8, 1.2], momenta in [-0.3, 0.3], total energy in [2.3, 2.7].
    Shape (E, 5, np^3), float64."""
    nn = p.np_ ** 3
    u = uniform(seed, p.nelem * 5 * nn).reshape(p.nelem, 5, nn)
    lo = np.array([0.8, -0.3, -0.3, -0.3, 2.3])[None, :, None]
    hi = np.array([1.2, 0.3, 0.3, 0.3, 2.7])[None, :, None]
    return lo + (hi - lo) * u


def random_displacements(seed: int, count: int, scale: float) -> np.ndarray:
    """Displacements uniform in [-scale, scale]."""
    return (2.0 * uniform(seed, count) - 1.0) * scale
