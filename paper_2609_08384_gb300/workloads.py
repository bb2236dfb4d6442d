"""Seeded synthetic workloads: grids, crystal stand-ins and input envelopes.

This module is shared by the CUDA path, the FP64 oracle's tests and the
benchmark.  It holds NO arithmetic of the split-step method itself (no
propagator, no nonlinear step, no FFT): only the problem statement -- grid
sizes and spacings, per-field coefficients, and the initial envelopes.

Input envelopes follow the paper's focused-beam entrance field (Sec. 2.1,
Eq. gaussianbeamc) multiplied by the Gaussian pulse factor of the OPG example
(Sec. 6, the pulsed form with exp[-(tau/tau0)^2]).  Peak intensity I is
converted to the focal amplitude through the power expression of Sec. 6,
P = 1/2 c eps0 n |A|^2 integrated over the beam, i.e. |A0|^2 = 2 I / (c eps0 n).

Crystal constants are synthetic, MgO:PPLN-like stand-ins (the paper's crystal
database is not part of the method): n_p=2.15, n_s=2.14, n_i=2.08 for the
1064/1450/3997 nm OPG triplet of Sec. 6, n_F=2.156, n_SH=2.234 for 1064 nm SHG,
d_eff = 14 pm/V.  Every random draw uses numpy ``default_rng(20260902 + index)``.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence

import numpy as np

C0 = 299792458.0
EPS0 = 8.8541878128e-12
HBAR = 1.054571817e-34

SEED_BASE = 20260902

FS = 1e-15
UM = 1e-6
MM = 1e-3
NM = 1e-9


@dataclasses.dataclass
class FieldParams:
    """Per-field linear coefficients, SI units (Eqs. dispOp, diffOp).

    lambda_: vacuum wavelength [m]; n: refractive index; delta: group-velocity
    mismatch 1/v_s - 1/v_lambda [s/m]; k2: GVD [s^2/m]; k3: TOD [s^3/m];
    rho: walk-off angle [rad]; alpha: linear loss [1/m].
    """

    lambda_: float
    n: float
    delta: float = 0.0
    k2: float = 0.0
    k3: float = 0.0
    rho: float = 0.0
    alpha: float = 0.0

    def as_tuple(self):
        return (self.lambda_, self.n, self.delta, self.k2, self.k3, self.rho, self.alpha)


@dataclasses.dataclass
class Grid:
    nx: int
    ny: int
    nt: int
    dx: float
    dy: float
    dt: float

    @property
    def npoints(self) -> int:
        return self.nx * self.ny * self.nt

    def axes(self):
        """Cell-centred axes x_j = (j - N/2) dx, same for y and tau."""
        x = (np.arange(self.nx) - self.nx // 2) * self.dx
        y = (np.arange(self.ny) - self.ny // 2) * self.dy
        t = (np.arange(self.nt) - self.nt // 2) * self.dt
        return x, y, t


@dataclasses.dataclass
class Problem:
    """One simulation: grid, fields (p,s,i) or (SH,F), coupling and z-grid."""

    name: str
    grid: Grid
    fields: List[FieldParams]
    d_eff: float
    dk: float
    length: float
    nz: int
    dk_profile: Optional[np.ndarray] = None

    @property
    def nfields(self) -> int:
        return len(self.fields)

    @property
    def dz(self) -> float:
        return self.length / self.nz


def peak_amplitude(intensity_w_m2: float, n: float) -> float:
    """|A0| from peak intensity, |A0|^2 = 2 I / (c eps0 n) (Sec. 6 power formula)."""
    return math.sqrt(2.0 * intensity_w_m2 / (C0 * EPS0 * n))


def focused_pulse(grid: Grid, fp: FieldParams, a0: float, w0: float, tau0: Optional[float],
                  length: float, focus: Optional[float] = None, delay: float = 0.0) -> np.ndarray:
    """Focused Gaussian beam at the crystal entrance (Eq. gaussianbeamc) times a
    Gaussian pulse exp[-((tau - delay)/tau0)^2] (Sec. 6).  ``focus`` defaults
    to the crystal centre L/2 (Sec. 2.1).  Returns complex128 [nt, ny, nx]."""
    if focus is None:
        focus = 0.5 * length
    k = 2.0 * math.pi * fp.n / fp.lambda_
    z_r = 0.5 * w0 * w0 * k
    xi = focus / z_r  # = L/(2 z_R) for f = L/2
    x, y, t = grid.axes()
    r2 = x[None, None, :] ** 2 + y[None, :, None] ** 2
    q = 1.0 - 1j * xi
    a = (a0 / q) * np.exp(-r2 / (w0 * w0 * q))
    if tau0 is not None:
        a = a * np.exp(-(((t - delay) / tau0) ** 2))[:, None, None]
    return np.ascontiguousarray(np.broadcast_to(a, (grid.nt, grid.ny, grid.nx))).astype(np.complex128)


def complex_noise(grid: Grid, rms: float, rng: np.random.Generator) -> np.ndarray:
    """i.i.d. circular complex Gaussian noise with E|xi|^2 = rms^2."""
    shape = (grid.nt, grid.ny, grid.nx)
    s = rms / math.sqrt(2.0)
    return (rng.standard_normal(shape) * s + 1j * rng.standard_normal(shape) * s).astype(np.complex128)


# ---------------------------------------------------------------------------
# Synthetic crystal stand-ins
# ---------------------------------------------------------------------------
D_EFF = 14e-12  # m/V
LAM_P, LAM_S, LAM_I = 1064 * NM, 1450 * NM, 3997 * NM
N_P, N_S, N_I = 2.15, 2.14, 2.08
LAM_F = 1064 * NM
LAM_SH = 532 * NM
N_F, N_SH = 2.156, 2.234

GVM = 100 * FS / MM          # 100 fs/mm -> s/m
GVD_P, GVD_S, GVD_I = 200 * FS**2 / MM, 100 * FS**2 / MM, 50 * FS**2 / MM


def shg_fields() -> List[FieldParams]:
    """Degenerate SHG, field order (SH, F); co-moving frame at the F group velocity."""
    return [FieldParams(LAM_SH, N_SH), FieldParams(LAM_F, N_F)]


def problem_shg_small() -> Problem:
    """SHG 32x32x64, 100 steps over 1 mm, Delta k = 0 (oracle-size case)."""
    g = Grid(32, 32, 64, 12.5 * UM, 12.5 * UM, 50 * FS)
    return Problem("shg_32x32x64", g, shg_fields(), D_EFF, 0.0, 1 * MM, 100)


def inputs_shg_small(p: Problem, seed_index: int = 0) -> List[np.ndarray]:
    a0 = peak_amplitude(1e13, N_F)  # 1 GW/cm^2
    f = focused_pulse(p.grid, p.fields[1], a0, 50 * UM, 200 * FS, p.length)
    return [np.zeros_like(f), f]


def problem_sfg() -> Problem:
    """SFG 128x128x256, 500 steps over 5 mm, field order (p, s, i)."""
    g = Grid(128, 128, 256, 3.75 * UM, 3.75 * UM, 4000 * FS / 256)
    fields = [FieldParams(LAM_P, N_P, delta=+GVM, k2=GVD_P),
              FieldParams(LAM_S, N_S, delta=0.0, k2=GVD_S),
              FieldParams(LAM_I, N_I, delta=-GVM, k2=GVD_I, rho=2e-3)]
    return Problem("sfg_128x128x256", g, fields, D_EFF, 20.0, 5 * MM, 500)


def inputs_sfg(p: Problem, seed_index: int = 1) -> List[np.ndarray]:
    s = focused_pulse(p.grid, p.fields[1], peak_amplitude(1e13, N_S), 40 * UM, 150 * FS, p.length)
    i = focused_pulse(p.grid, p.fields[2], peak_amplitude(1e13, N_I), 60 * UM, 250 * FS, p.length,
                      delay=30 * FS)
    return [np.zeros_like(s), s, i]


def problem_opg() -> Problem:
    """OPG 256x256x512, 1000 steps over 10 mm, field order (p, s, i)."""
    g = Grid(256, 256, 512, 3.125 * UM, 3.125 * UM, 16000 * FS / 512)
    fields = [FieldParams(LAM_P, N_P, delta=+GVM, k2=GVD_P, rho=2e-3),
              FieldParams(LAM_S, N_S, delta=0.0, k2=GVD_S, rho=0.0),
              FieldParams(LAM_I, N_I, delta=-GVM, k2=GVD_I, rho=1e-3)]
    return Problem("opg_256x256x512", g, fields, D_EFF, 0.0, 10 * MM, 1000)


def inputs_opg(p: Problem, seed_index: int = 2) -> List[np.ndarray]:
    rng = np.random.default_rng(SEED_BASE + seed_index)
    a0 = peak_amplitude(1e13, N_P)
    pump = focused_pulse(p.grid, p.fields[0], a0, 100 * UM, 1000 * FS, p.length)
    s = complex_noise(p.grid, 1e-6 * a0, rng)
    i = complex_noise(p.grid, 1e-6 * a0, rng)
    return [pump, s, i]


def problem_batch_member(nx: int, nt: int, dk: float, length: float, nz: int) -> Problem:
    g = Grid(nx, nx, nt, 12.5 * UM, 12.5 * UM, 50 * FS)
    return Problem(f"shg_{nx}x{nx}x{nt}", g, shg_fields(), D_EFF, dk, length, nz)


def problems_batched(count: int = 64, seed_index: int = 3) -> List[Problem]:
    """64 independent SHG runs: grid from {64^2x128, 96^2x192, 128^2x256},
    dk ~ U[-200, 200] 1/m, L ~ U[0.5, 5] mm, nz ~ U{200..800}."""
    rng = np.random.default_rng(SEED_BASE + seed_index)
    sizes = [(64, 128), (96, 192), (128, 256)]
    out = []
    for _ in range(count):
        nx, nt = sizes[int(rng.integers(0, 3))]
        dk = float(rng.uniform(-200.0, 200.0))
        length = float(rng.uniform(0.5, 5.0)) * MM
        nz = int(rng.integers(200, 801))
        out.append(problem_batch_member(nx, nt, dk, length, nz))
    return out


def problems_batched_small(count: int = 256, seed_index: int = 5) -> List[Problem]:
    """Many small SHG runs (32x32x64, window 400 um x 3.2 ps): dk ~ U[-200, 200]
    1/m, L ~ U[0.5, 5] mm, nz ~ U{200..800}."""
    rng = np.random.default_rng(SEED_BASE + seed_index)
    out = []
    for _ in range(count):
        dk = float(rng.uniform(-200.0, 200.0))
        length = float(rng.uniform(0.5, 5.0)) * MM
        nz = int(rng.integers(200, 801))
        out.append(problem_batch_member(32, 64, dk, length, nz))
    return out


def inputs_shg(p: Problem) -> List[np.ndarray]:
    a0 = peak_amplitude(1e13, N_F)
    f = focused_pulse(p.grid, p.fields[1], a0, 50 * UM, 200 * FS, p.length)
    return [np.zeros_like(f), f]


def problem_cw_shg() -> Problem:
    """cw focused SHG (nt = 1) at the Boyd-Kleinman optimum: 1024x1024 with
    dx = 0.5 um, F waist 20 um at the crystal centre (b = k_F w0^2 = 5.1 mm),
    L = 2.84 b, dk b / 2 = -0.57 (the Gouy-compensating sign for the SH
    equation's e^{-i dk z}), 1000 steps."""
    g = Grid(1024, 1024, 1, 0.5 * UM, 0.5 * UM, 1.0 * FS)
    w0 = 20 * UM
    b = 2 * math.pi * N_F / LAM_F * w0 * w0
    length = 2.84 * b
    p = Problem("cw_shg_1024x1024", g, shg_fields(), D_EFF, -2 * 0.57 / b, length, 1000)
    p.w0 = w0  # type: ignore[attr-defined]
    return p


def inputs_cw_shg(p: Problem) -> List[np.ndarray]:
    f = focused_pulse(p.grid, p.fields[1], peak_amplitude(1e13, N_F), p.w0, None, p.length)  # type: ignore[attr-defined]
    return [np.zeros_like(f), f]


def problem_adjoint() -> Problem:
    """SHG 128x128x256, 400 steps over 2 mm with a piecewise Delta k profile."""
    g = Grid(128, 128, 256, 12.5 * UM, 12.5 * UM, 50 * FS)
    rng = np.random.default_rng(SEED_BASE + 4)
    phi = rng.normal(0.0, 0.1, size=256)
    dk = 0.0 + rng.normal(0.0, 0.1, size=400) * (1.0 / MM)
    p = Problem("shg_adjoint_128x128x256", g, shg_fields(), D_EFF, 0.0, 2 * MM, 400, dk_profile=dk)
    p.spectral_phase = phi  # type: ignore[attr-defined]
    return p


def to_c64(arrs: Sequence[np.ndarray]) -> List[np.ndarray]:
    return [np.ascontiguousarray(a, dtype=np.complex64) for a in arrs]
