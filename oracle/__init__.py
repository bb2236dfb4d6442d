"""FP64 CPU oracle (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg load this package.  The CUDA library never imports it, and it imports
nothing from the CUDA library.  The arithmetic lives in ``brahms_oracle.c``
(plain C99 complex double, own recursive FFT); this module compiles it with
gcc and marshals numpy arrays.

Parity status of each function (what pins it, see tests/test_oracle_*.py):
  fft1d / fft3        naive O(N^2) DFT, numpy.fft, Parseval, impulse<->constant
  linear_step         Gaussian-beam waist w(z) with focus at L/2 (diffraction
                      sign), Gaussian-pulse broadening (GVD), exact integer
                      shifts (walk-off and group-velocity mismatch), loss
                      decay, composition and unitarity
  nonlinear_step      plane-wave tanh^2 SHG, undepleted sinc SHG/SFG/DFG,
                      undepleted-pump parametric gain (cosh/sinh)
  propagate           energy and Manley-Rowe invariants, second-order
                      self-convergence in dz
  energy              analytic Gaussian-beam/pulse energy
  heat_load           Gaussian beam/pulse absorbed power, the linear step's
                      own loss rate
  thermal_solve       discrete eigenmodes, second-order convergence to a
                      continuum solution, the discrete heat-flux balance
  adjoint_gradient    dot-product identities (linear step; RK4 against an
                      independent tangent-linear RK4), stage-phase
                      sensitivities and full gradients against central
                      finite differences of objective(), with and without
                      a transverse mismatch map
  adjoint_gradient    (also under a map that changes along z: uniform
                      segments give the step-profile gradient, one segment
                      the static-map gradient, central differences of
                      objective() with three segments)
  propagate_map_z     piecewise-constant mismatch per column against the
                      undepleted closed form sum_s e^{-i Phi(z_s)} (1 -
                      e^{-i dk_s l_s}) / (i dk_s); uniform segments equal the
                      per-step profile, one segment equals propagate_map
  spectral_phase      a linear phase Omega m dt is an exact circular shift
                      by m samples (both signs, 1e-13); a quadratic phase on a
                      Gaussian gives the chirped-Gaussian closed form (1e-9)
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "brahms_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain IEEE FP64; no fast-math)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-fcx-fortran-rules",
               "-fno-fast-math", _SRC, "-o", tmp, "-lm", "-lpthread"]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB)
    return _LIB


class _Field(ctypes.Structure):
    _fields_ = [("lambda_", ctypes.c_double), ("n", ctypes.c_double), ("delta", ctypes.c_double),
                ("k2", ctypes.c_double), ("k3", ctypes.c_double), ("rho", ctypes.c_double),
                ("alpha", ctypes.c_double)]


class _Problem(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nt", ctypes.c_int), ("nf", ctypes.c_int),
                ("dx", ctypes.c_double), ("dy", ctypes.c_double), ("dt", ctypes.c_double),
                ("d_eff", ctypes.c_double), ("f", _Field * 3)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.POINTER
            dp = P(ctypes.c_double)
            vp = ctypes.c_void_p
            lib.orc_set_threads.argtypes = [ctypes.c_int]
            lib.orc_get_threads.restype = ctypes.c_int
            lib.orc_dft_naive.argtypes = [vp, vp, ctypes.c_int, ctypes.c_int]
            lib.orc_fft1d.argtypes = [vp, ctypes.c_int, ctypes.c_int]
            lib.orc_fft3.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int]
            lib.orc_angular_freq.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double]
            lib.orc_angular_freq.restype = ctypes.c_double
            lib.orc_linear_step.argtypes = [P(_Problem), vp, ctypes.c_double]
            lib.orc_kappa.argtypes = [P(_Problem), ctypes.c_int]
            lib.orc_kappa.restype = ctypes.c_double
            lib.orc_nonlinear_step.argtypes = [P(_Problem), vp, ctypes.c_double, ctypes.c_double,
                                               ctypes.c_double]
            lib.orc_rk4_point.argtypes = [ctypes.c_int, dp, ctypes.c_double, ctypes.c_double,
                                          ctypes.c_double, vp]
            lib.orc_propagate.argtypes = [P(_Problem), vp, ctypes.c_int, ctypes.c_double, dp, dp]
            lib.orc_propagate.restype = ctypes.c_int
            lib.orc_energy.argtypes = [P(_Problem), vp, dp, dp]
            lib.orc_propagate_map.argtypes = [P(_Problem), vp, ctypes.c_int, ctypes.c_double, dp, dp,
                                              ctypes.c_double, dp]
            lib.orc_propagate_map.restype = ctypes.c_int
            lib.orc_propagate_map_z.argtypes = [P(_Problem), vp, ctypes.c_int, ctypes.c_double, dp, dp, ctypes.c_int,
                                                dp, dp]
            lib.orc_propagate_map_z.restype = ctypes.c_int
            lib.orc_power_trace.argtypes = [P(_Problem), vp, dp]
            lib.orc_spectrum.argtypes = [P(_Problem), vp, dp]
            lib.orc_heat_load.argtypes = [P(_Problem), vp, ctypes.c_double, dp]
            lib.orc_rk4_jvp_point.argtypes = [ctypes.c_int, dp, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                              vp, vp, vp, vp]
            lib.orc_rk4_vjp_point.argtypes = [ctypes.c_int, dp, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                              vp, vp, vp, dp]
            lib.orc_linear_step_adjoint.argtypes = [P(_Problem), vp, ctypes.c_double]
            lib.orc_spectral_phase.argtypes = [P(_Problem), vp, dp, ctypes.c_int]
            lib.orc_nonlinear_step_adjoint.argtypes = [P(_Problem), vp, vp, ctypes.c_double, ctypes.c_double,
                                                       ctypes.c_double, dp]
            lib.orc_adjoint_gradient.argtypes = [P(_Problem), vp, ctypes.c_int, ctypes.c_double, dp, dp,
                                                 ctypes.c_int, dp, dp, dp, dp]
            lib.orc_adjoint_gradient.restype = ctypes.c_double
            lib.orc_objective.argtypes = [P(_Problem), vp, ctypes.c_int, ctypes.c_double, dp, dp, ctypes.c_int, dp,
                                          dp]
            lib.orc_objective.restype = ctypes.c_double
            lib.orc_adjoint_gradient_z.argtypes = [P(_Problem), vp, ctypes.c_int, ctypes.c_double, dp, dp,
                                                   ctypes.c_int, dp, dp, dp, ctypes.c_int, dp, dp]
            lib.orc_adjoint_gradient_z.restype = ctypes.c_double
            lib.orc_objective_z.argtypes = [P(_Problem), vp, ctypes.c_int, ctypes.c_double, dp, dp, ctypes.c_int, dp,
                                            ctypes.c_int, dp, dp]
            lib.orc_objective_z.restype = ctypes.c_double
            _lib = lib
    return _lib


def set_threads(n: int) -> None:
    _load().orc_set_threads(int(n))


def get_threads() -> int:
    return int(_load().orc_get_threads())


def _c128(a: np.ndarray) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.complex128)


def dft_naive(x: np.ndarray, sign: int = -1) -> np.ndarray:
    x = _c128(x)
    out = np.empty_like(x)
    _load().orc_dft_naive(x.ctypes.data, out.ctypes.data, x.size, sign)
    return out


def fft1d(x: np.ndarray, sign: int = -1) -> np.ndarray:
    y = _c128(x).copy()
    _load().orc_fft1d(y.ctypes.data, y.size, sign)
    return y


def fft3(a: np.ndarray, sign: int = -1) -> np.ndarray:
    """Unnormalised 3D DFT of an [nt, ny, nx] array (sign -1 forward)."""
    y = _c128(a).copy()
    nt, ny, nx = y.shape
    _load().orc_fft3(y.ctypes.data, nx, ny, nt, sign)
    return y


def angular_freq(m: int, n: int, d: float) -> float:
    return float(_load().orc_angular_freq(m, n, d))


def make_problem(grid, fields, d_eff: float) -> _Problem:
    p = _Problem()
    p.nx, p.ny, p.nt = grid.nx, grid.ny, grid.nt
    p.nf = len(fields)
    p.dx, p.dy, p.dt = grid.dx, grid.dy, grid.dt
    p.d_eff = d_eff
    for i, f in enumerate(fields):
        p.f[i] = _Field(*f.as_tuple())
    return p


def _stack(fields: Sequence[np.ndarray]) -> np.ndarray:
    return np.ascontiguousarray(np.stack([_c128(f) for f in fields]))


def kappa(prob: _Problem, f: int) -> float:
    return float(_load().orc_kappa(ctypes.byref(prob), f))


def linear_step(prob: _Problem, fields: Sequence[np.ndarray], dz: float) -> np.ndarray:
    a = _stack(fields)
    _load().orc_linear_step(ctypes.byref(prob), a.ctypes.data, dz)
    return a


def nonlinear_step(prob: _Problem, fields: Sequence[np.ndarray], phi_a: float, dk: float,
                   h: float) -> np.ndarray:
    a = _stack(fields)
    _load().orc_nonlinear_step(ctypes.byref(prob), a.ctypes.data, phi_a, dk, h)
    return a


def propagate(prob: _Problem, fields: Sequence[np.ndarray], nz: int, dz: float, dk,
              phi0: float = 0.0, check: bool = True):
    """Run nz split steps.  ``dk`` is a scalar or an array of nz per-step values.
    Returns (fields[nf, nt, ny, nx] complex128, phi_end)."""
    a = _stack(fields)
    dks = np.ascontiguousarray(np.broadcast_to(np.asarray(dk, dtype=np.float64), (nz,)))
    phi = ctypes.c_double(phi0)
    rc = _load().orc_propagate(ctypes.byref(prob), a.ctypes.data, int(nz), float(dz),
                               dks.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), ctypes.byref(phi))
    if check and rc != 0:
        raise FloatingPointError("oracle: non-finite fields (dz too large)")
    return a, phi.value


def energy(prob: _Problem, fields: Sequence[np.ndarray]):
    a = _stack(fields)
    e = np.zeros(prob.nf)
    ph = np.zeros(prob.nf)
    dp = ctypes.POINTER(ctypes.c_double)
    _load().orc_energy(ctypes.byref(prob), a.ctypes.data, e.ctypes.data_as(dp), ph.ctypes.data_as(dp))
    return e, ph


def propagate_map(prob: _Problem, fields: Sequence[np.ndarray], nz: int, dz: float, dk, dk_map: np.ndarray,
                  phi0: float = 0.0, z0: float = 0.0, check: bool = True):
    """propagate() with a transverse mismatch map dk_map[ny, nx] [1/m] added to
    every step's dk; z0 is the distance from the start of the crystal."""
    a = _stack(fields)
    dks = np.ascontiguousarray(np.broadcast_to(np.asarray(dk, dtype=np.float64), (nz,)))
    m = np.ascontiguousarray(dk_map, dtype=np.float64).reshape(prob.ny, prob.nx)
    phi = ctypes.c_double(phi0)
    dp = ctypes.POINTER(ctypes.c_double)
    rc = _load().orc_propagate_map(ctypes.byref(prob), a.ctypes.data, int(nz), float(dz), dks.ctypes.data_as(dp),
                                   ctypes.byref(phi), float(z0), m.ctypes.data_as(dp))
    if check and rc != 0:
        raise FloatingPointError("oracle: non-finite fields (dz too large)")
    return a, phi.value


def propagate_map_z(prob: _Problem, fields: Sequence[np.ndarray], nz: int, dz: float, dk, z_edges,
                    maps: np.ndarray, phi0: float = 0.0, check: bool = True):
    """propagate() from z = 0 under a mismatch map that changes along z:
    maps[s, ny, nx] [1/m] on the segments separated by the increasing
    distances z_edges (len(maps) - 1 of them); step j takes the segment of
    its midpoint, and the coupling phase is the integral of the mismatch
    (orc_propagate_map_z)."""
    a = _stack(fields)
    dks = np.ascontiguousarray(np.broadcast_to(np.asarray(dk, dtype=np.float64), (nz,)))
    m = np.ascontiguousarray(maps, dtype=np.float64).reshape(-1, prob.ny, prob.nx)
    e = np.ascontiguousarray(np.asarray(z_edges, dtype=np.float64).reshape(-1))
    if len(e) != len(m) - 1 or np.any(np.diff(e) <= 0):
        raise ValueError("need len(maps) - 1 increasing z_edges")
    e = e if len(e) else np.zeros(1)
    phi = ctypes.c_double(phi0)
    dp = ctypes.POINTER(ctypes.c_double)
    rc = _load().orc_propagate_map_z(ctypes.byref(prob), a.ctypes.data, int(nz), float(dz), dks.ctypes.data_as(dp),
                                     ctypes.byref(phi), int(len(m)), e.ctypes.data_as(dp), m.ctypes.data_as(dp))
    if rc == 1:
        raise MemoryError("oracle: map phase buffers")
    if check and rc != 0:
        raise FloatingPointError("oracle: non-finite fields (dz too large)")
    return a, phi.value


def power_trace(prob: _Problem, fields: Sequence[np.ndarray]) -> np.ndarray:
    """[nf, nt] temporal power [W] (orc_power_trace)."""
    a = _stack(fields)
    out = np.zeros((prob.nf, prob.nt))
    _load().orc_power_trace(ctypes.byref(prob), a.ctypes.data, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    return out


def spectrum(prob: _Problem, fields: Sequence[np.ndarray]) -> np.ndarray:
    """[nf, nt] energy per Omega bin [J], FFT order (orc_spectrum)."""
    a = _stack(fields)
    out = np.zeros((prob.nf, prob.nt))
    _load().orc_spectrum(ctypes.byref(prob), a.ctypes.data, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    return out


def heat_load(prob: _Problem, fields: Sequence[np.ndarray], rep_rate: float = 0.0) -> np.ndarray:
    """[ny, nx] absorbed power density Q [W/m^3] (orc_heat_load)."""
    a = _stack(fields)
    out = np.zeros((prob.ny, prob.nx))
    _load().orc_heat_load(ctypes.byref(prob), a.ctypes.data, float(rep_rate),
                          out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    return out


def thermal_matrix(nx: int, ny: int, dx: float, dy: float):
    """The 5-point operator -(d_xx + d_yy) on the fields' (x, y) grid as a
    sparse matrix (row index y * nx + x), with T = 0 half a cell outside the
    window: the missing neighbour of an edge point is its mirror image -T, so
    the edge's diagonal entry gains one more 1/d^2.  An axis of length 1 has
    no derivative along it (Sec. 4.1, heat equation; the boundary reading is the
    crystal's side faces held at the mount temperature)."""
    import scipy.sparse as sp

    def second_difference(n, d):
        if n == 1:
            return sp.csr_matrix((1, 1))
        main = np.full(n, 2.0)
        main[0] += 1.0
        main[-1] += 1.0
        off = np.full(n - 1, -1.0)
        return sp.diags([off, main, off], [-1, 0, 1], format="csr") / (d * d)

    return (sp.kron(sp.identity(ny), second_difference(nx, dx))
            + sp.kron(second_difference(ny, dy), sp.identity(nx))).tocsc()


def thermal_solve(q: np.ndarray, dx: float, dy: float, kappa_th: float) -> np.ndarray:
    """Steady-state temperature rise T [ny, nx] [K] of -kappa_th lap T = q:
    the stencil matrix of thermal_matrix() solved by a sparse direct solver."""
    import scipy.sparse.linalg as spla
    ny, nx = q.shape
    a = thermal_matrix(nx, ny, dx, dy) * kappa_th
    return spla.spsolve(a, np.ascontiguousarray(q, dtype=np.float64).ravel()).reshape(ny, nx)


def problem_from(p) -> _Problem:
    """Oracle problem struct from a workloads.Problem."""
    return make_problem(p.grid, p.fields, p.d_eff)


# --------------------------------------------------------------- adjoint
def _dptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _kap(prob):
    return np.array([kappa(prob, f) for f in range(prob.nf)] + [0.0] * (3 - prob.nf))


def rk4_jvp_point(prob, phi_a, dk, h, x, dx):
    """Tangent of one RK4 step at one point: returns (y, dy)."""
    x = _c128(x)
    dx = _c128(dx)
    y = np.zeros(3, complex)
    dy = np.zeros(3, complex)
    k = _kap(prob)
    _load().orc_rk4_jvp_point(prob.nf, _dptr(k), phi_a, dk, h, x.ctypes.data, dx.ctypes.data, y.ctypes.data,
                              dy.ctypes.data)
    return y[:prob.nf], dy[:prob.nf]


def rk4_vjp_point(prob, phi_a, dk, h, x, gy):
    """Adjoint of one RK4 step at one point: returns (gx, sens[3])."""
    x = _c128(x)
    gy = _c128(gy)
    gx = np.zeros(3, complex)
    sens = np.zeros(3)
    k = _kap(prob)
    _load().orc_rk4_vjp_point(prob.nf, _dptr(k), phi_a, dk, h, x.ctypes.data, gy.ctypes.data, gx.ctypes.data,
                              _dptr(sens))
    return gx[:prob.nf], sens


def linear_step_adjoint(prob, fields, dz):
    a = _stack(fields)
    _load().orc_linear_step_adjoint(ctypes.byref(prob), a.ctypes.data, dz)
    return a


def spectral_phase(prob, field, phi, sign=+1):
    a = _c128(field).copy()
    ph = np.ascontiguousarray(phi, dtype=np.float64)
    _load().orc_spectral_phase(ctypes.byref(prob), a.ctypes.data, _dptr(ph), int(sign))
    return a


def _map(prob, dk_map):
    return None if dk_map is None else np.ascontiguousarray(dk_map, dtype=np.float64).reshape(prob.ny, prob.nx)


def _zmaps(prob, z_edges, maps):
    m = np.ascontiguousarray(maps, dtype=np.float64).reshape(-1, prob.ny, prob.nx)
    e = np.ascontiguousarray(np.asarray(z_edges, dtype=np.float64).reshape(-1))
    if len(e) != len(m) - 1 or np.any(np.diff(e) <= 0):
        raise ValueError("need len(maps) - 1 increasing z_edges")
    return m, (e if len(e) else np.zeros(1))


def objective(prob, fields, nz, dz, dk, weights, phi=None, phi_field=1, dk_map=None, z_edges=None, maps=None):
    """J of adjoint_gradient alone (for finite differences); maps (with
    z_edges) is a map that changes along z, as in propagate_map_z."""
    a = _stack(fields)
    dks = np.ascontiguousarray(np.broadcast_to(np.asarray(dk, dtype=np.float64), (nz,)))
    w = np.ascontiguousarray(weights, dtype=np.float64)
    ph = None if phi is None else np.ascontiguousarray(phi, dtype=np.float64)
    if maps is not None:
        mz, e = _zmaps(prob, z_edges, maps)
        return float(_load().orc_objective_z(ctypes.byref(prob), a.ctypes.data, int(nz), float(dz), _dptr(dks),
                                             _dptr(ph), int(phi_field), _dptr(w), int(len(mz)), _dptr(e), _dptr(mz)))
    m = _map(prob, dk_map)
    return float(_load().orc_objective(ctypes.byref(prob), a.ctypes.data, int(nz), float(dz), _dptr(dks),
                                       _dptr(ph), int(phi_field), _dptr(w), _dptr(m)))


def adjoint_gradient(prob, fields, nz, dz, dk, weights, phi=None, phi_field=1, dk_map=None, z_edges=None, maps=None):
    """J = sum_f w_f sum |A_f(L)|^2 and its gradient with respect to the
    spectral phase phi (centred order, applied to field phi_field) and the
    per-step mismatch, optionally under a transverse mismatch map dk_map
    [ny, nx] or a map that changes along z (maps [nseg, ny, nx] with
    z_edges, as in propagate_map_z).  Returns (J, grad_phi or None, grad_dk)."""
    a = _stack(fields)
    dks = np.ascontiguousarray(np.broadcast_to(np.asarray(dk, dtype=np.float64), (nz,)))
    w = np.ascontiguousarray(weights, dtype=np.float64)
    ph = None if phi is None else np.ascontiguousarray(phi, dtype=np.float64)
    gphi = None if phi is None else np.zeros(prob.nt)
    gdk = np.zeros(nz)
    if maps is not None:
        mz, e = _zmaps(prob, z_edges, maps)
        J = _load().orc_adjoint_gradient_z(ctypes.byref(prob), a.ctypes.data, int(nz), float(dz), _dptr(dks),
                                           _dptr(ph), int(phi_field), _dptr(w), _dptr(gphi), _dptr(gdk),
                                           int(len(mz)), _dptr(e), _dptr(mz))
        return float(J), gphi, gdk
    m = _map(prob, dk_map)
    J = _load().orc_adjoint_gradient(ctypes.byref(prob), a.ctypes.data, int(nz), float(dz), _dptr(dks),
                                     _dptr(ph), int(phi_field), _dptr(w), _dptr(gphi), _dptr(gdk), _dptr(m))
    return float(J), gphi, gdk
