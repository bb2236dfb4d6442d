"""Python binding of the GB300 split-step chi(2) solver (C ABI in include/brahms.h).

Argument marshalling only: every step of the split-step path runs in the CUDA
library ``_build/libbrahms.so``.  PyTorch provides device memory (the
workspace), CUDA streams and pinned host buffers.  If the library has not
been built, importing the binding works but every call raises -- there is no
CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libbrahms.so")

BRAHMS_OK = 0
BRAHMS_E_ARG = 1
BRAHMS_E_SIZE = 2
BRAHMS_E_CUDA = 3
BRAHMS_E_OOM = 4
BRAHMS_E_NONFINITE = 5
BRAHMS_E_TIMEOUT = 6
BRAHMS_E_STATE = 7
BRAHMS_C64 = 0
BRAHMS_C128 = 1

KIND_NAMES = ("xpass_nl", "ypass_fwd", "tpass_prop", "ypass_inv", "other")
BRAHMS_OPT_TMA_TAU = 1
BRAHMS_OPT_FIELD_STREAMS = 2
BRAHMS_OPT_TMA_WAIT_US = 3

# Every entry point declared in include/brahms.h, with its ctypes signature.
_c = ctypes
_vp = _c.c_void_p
_dp = _c.POINTER(_c.c_double)
_llp = _c.POINTER(_c.c_longlong)


class FieldParams(ctypes.Structure):
    _fields_ = [("lambda_", _c.c_double), ("n", _c.c_double), ("delta", _c.c_double), ("k2", _c.c_double),
                ("k3", _c.c_double), ("rho", _c.c_double), ("alpha", _c.c_double)]


SIGNATURES = {
    "brahms_workspace_size": (_c.c_int, [_c.c_int, _c.c_int, _c.c_int, _c.c_int, _c.POINTER(_c.c_size_t)]),
    "brahms_init_grid": (_c.c_int, [_c.POINTER(_vp), _c.c_int, _c.c_int, _c.c_int, _c.c_double, _c.c_double,
                                    _c.c_double, _c.c_int, _c.POINTER(FieldParams), _c.c_double, _c.c_double,
                                    _vp, _c.c_size_t, _vp]),
    "brahms_set_fields": (_c.c_int, [_vp, _c.POINTER(_vp), _c.c_int, _c.c_int]),
    "brahms_set_dk_profile": (_c.c_int, [_vp, _dp, _c.c_int]),
    "brahms_propagate": (_c.c_int, [_vp, _c.c_int, _c.c_double]),
    "brahms_get_fields": (_c.c_int, [_vp, _c.POINTER(_vp), _c.c_int, _c.c_int]),
    "brahms_energy": (_c.c_int, [_vp, _dp, _dp]),
    "brahms_sync": (_c.c_int, [_vp]),
    "brahms_transform": (_c.c_int, [_vp, _c.c_int]),
    "brahms_get_z": (_c.c_int, [_vp, _dp, _dp]),
    "brahms_diagnostics": (_c.c_int, [_vp, _dp, _dp]),
    "brahms_set_dk_map": (_c.c_int, [_vp, _dp]),
    "brahms_set_dk_map_z": (_c.c_int, [_vp, _c.c_int, _dp, _dp]),
    "brahms_heat_accumulate": (_c.c_int, [_vp, _c.c_double, _c.c_double]),
    "brahms_heat_accumulate_segment": (_c.c_int, [_vp, _c.c_int, _c.c_double, _c.c_double]),
    "brahms_heat_set": (_c.c_int, [_vp, _dp]),
    "brahms_thermal_map": (_c.c_int, [_vp, _c.c_double, _c.c_double, _dp]),
    "brahms_timing": (_c.c_int, [_vp, _c.c_int, _dp, _llp, _c.c_int]),
    "brahms_launch_count": (_c.c_longlong, [_vp]),
    "brahms_set_option": (_c.c_int, [_vp, _c.c_int, _c.c_int]),
    "brahms_get_option": (_c.c_int, [_vp, _c.c_int]),
    "brahms_energy_static": (_c.c_int, [_c.POINTER(_vp), _c.c_int, _c.c_int, _c.c_int, _c.c_int, _c.c_double,
                                        _c.c_double, _c.c_double, _c.POINTER(FieldParams), _vp, _vp]),
    "brahms_adjoint_forward": (_c.c_int, [_vp, _c.POINTER(_vp), _c.c_int, _c.c_int, _dp, _c.c_int, _dp, _c.c_int,
                                          _c.c_double, _dp, _c.c_int, _dp]),
    "brahms_adjoint_backward": (_c.c_int, [_vp, _c.c_double, _dp, _dp]),
    "brahms_shg_efficiency_weights": (_c.c_int, [_vp, _dp]),
    "brahms_batch_create": (_c.c_int, [_c.POINTER(_vp), _vp]),
    "brahms_batch_add": (_c.c_int, [_vp, _c.c_int, _c.c_int, _c.c_int, _c.c_double, _c.c_double, _c.c_double,
                                    _c.POINTER(FieldParams), _c.c_double, _c.c_double, _c.c_int, _c.c_double,
                                    _c.POINTER(_c.c_int)]),
    "brahms_batch_set_fields": (_c.c_int, [_vp, _c.c_int, _c.POINTER(_vp), _c.c_int, _c.c_int]),
    "brahms_batch_set_granularity": (_c.c_int, [_vp, _c.c_int, _c.c_int, _c.c_int, _c.c_int]),
    "brahms_batch_tune": (_c.c_int, [_vp, _c.c_int, _dp]),
    "brahms_batch_get_schedule": (_c.c_int, [_vp, _c.c_int, _c.POINTER(_c.c_int), _c.POINTER(_c.c_int),
                                             _c.POINTER(_c.c_int), _c.POINTER(_c.c_int)]),
    "brahms_batch_run": (_c.c_int, [_vp]),
    "brahms_batch_sync": (_c.c_int, [_vp]),
    "brahms_batch_set_timeout": (_c.c_int, [_vp, _c.c_double]),
    "brahms_batch_set_mode": (_c.c_int, [_vp, _c.c_int]),
    "brahms_batch_get_mode": (_c.c_int, [_vp]),
    "brahms_batch_get_fields": (_c.c_int, [_vp, _c.c_int, _c.POINTER(_vp), _c.c_int, _c.c_int]),
    "brahms_batch_info": (_c.c_int, [_vp, _c.POINTER(_c.c_int), _c.POINTER(_c.c_int), _c.POINTER(_c.c_int),
                                     _llp]),
    "brahms_batch_free": (None, [_vp]),
    "brahms_batch_last_error": (_c.c_char_p, [_vp]),
    "brahms_fp32_fma_rate": (_c.c_int, [_vp, _dp]),
    "brahms_dsmem_exchange_rate": (_c.c_int, [_c.c_int, _c.c_int, _vp, _dp]),
    "brahms_fail_next_allocations": (_c.c_int, [_c.c_int]),
    "brahms_pending_allocation_failures": (_c.c_int, []),
    "brahms_free": (None, [_vp]),
    "brahms_last_error": (_c.c_char_p, [_vp]),
    "brahms_status_string": (_c.c_char_p, [_c.c_int]),
}

_lib = None
_lock = threading.Lock()


class BrahmsError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{status_string(status) if _lib else status}: {msg}")
        self.status = status


def library_path() -> str:
    return LIB_PATH


def load(path: Optional[str] = None):
    """Load the CUDA library (raises if it is missing: no fallback)."""
    global _lib
    with _lock:
        if _lib is None:
            p = path or LIB_PATH
            if not os.path.exists(p):
                raise RuntimeError(f"CUDA library not built: {p} (run __graft_entry__.build())")
            lib = ctypes.CDLL(p)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def status_string(s: int) -> str:
    return load().brahms_status_string(int(s)).decode()


def _check(ctx, s: int):
    if s != BRAHMS_OK:
        msg = load().brahms_last_error(ctx).decode() if ctx else ""
        raise BrahmsError(s, msg)


def _ptr_array(ptrs: Sequence[int]):
    arr = (_vp * len(ptrs))(*[_vp(int(p)) for p in ptrs])
    return arr


def field_params(fp) -> FieldParams:
    """FieldParams from a workloads.FieldParams (or any object with as_tuple())."""
    return FieldParams(*fp.as_tuple())


def workspace_size(nx: int, ny: int, nt: int, nfields: int) -> int:
    b = ctypes.c_size_t()
    _check(None, load().brahms_workspace_size(nx, ny, nt, nfields, ctypes.byref(b)))
    return int(b.value)


class Solver:
    """One simulation context: a torch-owned device workspace plus the C
    context.  Methods map one-to-one onto the C entry points."""

    def __init__(self, grid, fields, d_eff: float, dk: float, stream=None, device=None):
        import torch

        lib = load()
        self.nf = len(fields)
        self.nseg = 1  # z-segments of the mismatch map and heat load
        self.grid = grid
        self.shape = (grid.nt, grid.ny, grid.nx)
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        nbytes = workspace_size(grid.nx, grid.ny, grid.nt, self.nf)
        self.workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
        base = self.workspace.data_ptr()
        aligned = (base + 255) & ~255
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        fp = (FieldParams * 3)(*[field_params(f) for f in fields])
        ctx = _vp()
        s = lib.brahms_init_grid(ctypes.byref(ctx), grid.nx, grid.ny, grid.nt, grid.dx, grid.dy, grid.dt,
                                 self.nf, fp, float(d_eff), float(dk), _vp(aligned), nbytes,
                                 _vp(self.stream.cuda_stream))
        _check(None, s)
        self.ctx = ctx

    # -- lifecycle
    def close(self):
        if getattr(self, "ctx", None):
            load().brahms_free(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- entry points
    def set_fields(self, fields, on_device: Optional[bool] = None):
        """fields: sequence of torch tensors (cuda or cpu) or numpy arrays,
        complex64 or complex128, shape (nt, ny, nx), C-contiguous."""
        ptrs, dtype, dev = self._marshal(fields, on_device)
        _check(self.ctx, load().brahms_set_fields(self.ctx, _ptr_array(ptrs), dtype, int(dev)))

    def get_fields(self, out=None, dtype=np.complex64, on_device: bool = False):
        """Returns a list of arrays (numpy on host, torch on device) unless out is given."""
        import torch

        if out is None:
            if on_device:
                tdt = torch.complex64 if np.dtype(dtype) == np.complex64 else torch.complex128
                out = [torch.empty(self.shape, dtype=tdt, device=self.device) for _ in range(self.nf)]
            else:
                out = [np.empty(self.shape, dtype=dtype) for _ in range(self.nf)]
        ptrs, dt, dev = self._marshal(out, on_device, writable=True)
        _check(self.ctx, load().brahms_get_fields(self.ctx, _ptr_array(ptrs), dt, int(dev)))
        return out

    def set_dk_profile(self, dk):
        arr = np.ascontiguousarray(dk, dtype=np.float64)
        _check(self.ctx, load().brahms_set_dk_profile(self.ctx, arr.ctypes.data_as(_dp), int(arr.size)))

    def propagate(self, nz: int, dz: float):
        _check(self.ctx, load().brahms_propagate(self.ctx, int(nz), float(dz)))

    def energy(self):
        e = np.zeros(self.nf)
        ph = np.zeros(self.nf)
        _check(self.ctx, load().brahms_energy(self.ctx, e.ctypes.data_as(_dp), ph.ctypes.data_as(_dp)))
        return e, ph

    def set_dk_map(self, dk_map):
        """Transverse mismatch map [ny, nx] in 1/m added to every step's dk from
        the current z on (the phase is its integral); None removes it."""
        if dk_map is None:
            _check(self.ctx, load().brahms_set_dk_map(self.ctx, None))
        else:
            m = np.ascontiguousarray(dk_map, dtype=np.float64).reshape(self.grid.ny, self.grid.nx)
            _check(self.ctx, load().brahms_set_dk_map(self.ctx, m.ctypes.data_as(_dp)))
        self.nseg = 1

    def set_dk_map_z(self, z_edges, maps=None):
        """Mismatch maps that change along z: maps [nseg, ny, nx] in 1/m on the
        segments separated by the nseg - 1 distances z_edges [m] (step j takes
        the segment of its midpoint); maps None: zero maps (segments of the
        thermal model alone, nseg = len(z_edges) + 1)."""
        e = np.ascontiguousarray(np.asarray(z_edges, dtype=np.float64).reshape(-1))
        nseg = len(e) + 1
        m = None
        if maps is not None:
            m = np.ascontiguousarray(maps, dtype=np.float64).reshape(nseg, self.grid.ny, self.grid.nx)
        _check(self.ctx, load().brahms_set_dk_map_z(self.ctx, nseg, e.ctypes.data_as(_dp) if len(e) else None,
                                                    None if m is None else m.ctypes.data_as(_dp)))
        self.nseg = nseg

    def diagnostics(self):
        """(power [nf, nt] in W, spectrum [nf, nt] in J per Omega bin, FFT order)."""
        p = np.zeros((self.nf, self.grid.nt))
        sp = np.zeros((self.nf, self.grid.nt))
        _check(self.ctx, load().brahms_diagnostics(self.ctx, p.ctypes.data_as(_dp), sp.ctypes.data_as(_dp)))
        return p, sp

    def heat_accumulate(self, rep_rate: float = 0.0, weight: float = 1.0, segment=None):
        """Add weight * Q(x, y) of the current fields to a z-segment's heat load
        [W/m^3] (Q = sum_f alpha_f I_f, time-averaged at rep_rate [Hz] when
        nt > 1); segment None: the segment that holds the current z."""
        if segment is None:
            _check(self.ctx, load().brahms_heat_accumulate(self.ctx, float(rep_rate), float(weight)))
        else:
            _check(self.ctx, load().brahms_heat_accumulate_segment(self.ctx, int(segment), float(rep_rate),
                                                                   float(weight)))

    def heat_set(self, q):
        """Replace the heat loads with q [nseg, ny, nx] (or [ny, nx] for one
        segment) in W/m^3; None zeroes them."""
        if q is None:
            _check(self.ctx, load().brahms_heat_set(self.ctx, None))
            return
        a = np.ascontiguousarray(q, dtype=np.float64).reshape(self.nseg, self.grid.ny, self.grid.nx)
        _check(self.ctx, load().brahms_heat_set(self.ctx, a.ctypes.data_as(_dp)))

    def thermal_map(self, kappa_th: float, dkdT: float, want_temperature: bool = True):
        """Solve -kappa_th lap_perp T_s = Q_s per z-segment (T = 0 half a cell
        outside the window) and install dk_map_s = M_s + dkdT * T_s; returns T
        [ny, nx] in K for one segment, [nseg, ny, nx] for several (or None)."""
        t = np.zeros((self.nseg, self.grid.ny, self.grid.nx)) if want_temperature else None
        _check(self.ctx, load().brahms_thermal_map(self.ctx, float(kappa_th), float(dkdT),
                                                   None if t is None else t.ctypes.data_as(_dp)))
        return t if t is None or self.nseg > 1 else t[0]

    def sync(self):
        _check(self.ctx, load().brahms_sync(self.ctx))

    def transform(self, direction: int):
        _check(self.ctx, load().brahms_transform(self.ctx, int(direction)))

    def get_z(self):
        z = ctypes.c_double()
        phi = ctypes.c_double()
        _check(self.ctx, load().brahms_get_z(self.ctx, ctypes.byref(z), ctypes.byref(phi)))
        return z.value, phi.value

    def timing(self, enable: bool, every: int = 1):
        """Start (enable) or stop per-kernel CUDA-event timing; every > 1 times
        every every-th launch of each kind.  Returns (ms, timed launches) per
        kind accumulated so far."""
        ms = np.zeros(5)
        n = np.zeros(5, dtype=np.int64)
        flag = (max(1, int(every)) if enable else 0)
        _check(self.ctx, load().brahms_timing(self.ctx, flag, ms.ctypes.data_as(_dp),
                                              n.ctypes.data_as(_llp), 5))
        return ms, n

    def launch_count(self) -> int:
        return int(load().brahms_launch_count(self.ctx))

    def set_option(self, option: int, value: int):
        _check(self.ctx, load().brahms_set_option(self.ctx, int(option), int(value)))

    def get_option(self, option: int) -> int:
        return int(load().brahms_get_option(self.ctx, int(option)))

    def adjoint_forward(self, fields, dk, nz, dz, weights, phi=None, phi_field=1, checkpoint_interval=0):
        """J = sum_f w_f sum |A_f(L)|^2 after the phase phi (centred order) and
        nz steps with the mismatch profile dk; keeps checkpoints."""
        ptrs, dtype, dev = self._marshal(fields, None)
        dks = np.ascontiguousarray(np.broadcast_to(np.asarray(dk, dtype=np.float64), (int(nz),)))
        w = np.ascontiguousarray(weights, dtype=np.float64)
        ph = None if phi is None else np.ascontiguousarray(phi, dtype=np.float64)
        J = ctypes.c_double()
        # recorded first: after a failed forward the C library answers a
        # backward with BRAHMS_E_STATE
        self._adj = (int(nz), ph is not None)
        _check(self.ctx, load().brahms_adjoint_forward(
            self.ctx, _ptr_array(ptrs), dtype, int(dev), None if ph is None else ph.ctypes.data_as(_dp),
            int(phi_field), dks.ctypes.data_as(_dp), int(nz), float(dz), w.ctypes.data_as(_dp),
            int(checkpoint_interval), ctypes.byref(J)))
        return J.value

    def shg_efficiency_weights(self, fields=None):
        """Weights (w_SH, w_F) that make adjoint_forward's J the SHG efficiency
        of the input; ``fields`` (if given) are set first as the input."""
        if fields is not None:
            self.set_fields(fields)
        w = np.zeros(2)
        _check(self.ctx, load().brahms_shg_efficiency_weights(self.ctx, w.ctypes.data_as(_dp)))
        return w

    def adjoint_backward(self, gscale=1.0):
        """(gscale dJ/dphi or None, gscale dJ/d dk) for the last adjoint_forward."""
        nz, has_phi = getattr(self, "_adj", (1, False))
        gphi = np.zeros(self.grid.nt)
        gdk = np.zeros(nz)
        _check(self.ctx, load().brahms_adjoint_backward(self.ctx, float(gscale), gphi.ctypes.data_as(_dp),
                                                        gdk.ctypes.data_as(_dp)))
        return (gphi if has_phi else None), gdk

    # -- helpers
    def _marshal(self, arrs, on_device, writable=False):
        import torch

        if len(arrs) != self.nf:
            raise ValueError(f"expected {self.nf} fields")
        ptrs = []
        kinds = set()
        dev = None
        for a in arrs:
            if isinstance(a, torch.Tensor):
                if tuple(a.shape) != self.shape or not a.is_contiguous():
                    raise ValueError("field tensors must be contiguous with shape (nt, ny, nx)")
                kinds.add(a.dtype)
                d = a.is_cuda
                ptrs.append(a.data_ptr())
            else:
                if not isinstance(a, np.ndarray) or a.shape != self.shape or not a.flags["C_CONTIGUOUS"]:
                    raise ValueError("field arrays must be C-contiguous numpy arrays of shape (nt, ny, nx)")
                if writable and not a.flags["WRITEABLE"]:
                    raise ValueError("output array is read-only")
                kinds.add(torch.complex64 if a.dtype == np.complex64 else
                          torch.complex128 if a.dtype == np.complex128 else a.dtype)
                d = False
                ptrs.append(a.ctypes.data)
            if dev is None:
                dev = d
            elif dev != d:
                raise ValueError("all fields must be on the same side (host or device)")
        if on_device is not None and bool(on_device) != bool(dev):
            raise ValueError("on_device does not match the buffers")
        if len(kinds) != 1:
            raise ValueError("all fields must share one dtype")
        k = kinds.pop()
        if k == torch.complex64:
            dt = BRAHMS_C64
        elif k == torch.complex128:
            dt = BRAHMS_C128
        else:
            raise ValueError("fields must be complex64 or complex128")
        return ptrs, dt, dev


class Batch:
    """A batch of two-field SHG instances advanced by one persistent launch
    (brahms_batch_* entry points)."""

    def __init__(self, stream=None):
        import torch

        lib = load()
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        h = _vp()
        _check(None, lib.brahms_batch_create(ctypes.byref(h), _vp(self.stream.cuda_stream)))
        self.h = h
        self.shapes = []

    def _chk(self, s):
        if s != BRAHMS_OK:
            raise BrahmsError(s, load().brahms_batch_last_error(self.h).decode())

    def add(self, grid, fields, d_eff, dk, nz, dz) -> int:
        fp = (FieldParams * 2)(*[field_params(f) for f in fields])
        idx = ctypes.c_int()
        self._chk(load().brahms_batch_add(self.h, grid.nx, grid.ny, grid.nt, grid.dx, grid.dy, grid.dt, fp,
                                          float(d_eff), float(dk), int(nz), float(dz), ctypes.byref(idx)))
        self.shapes.append((grid.nt, grid.ny, grid.nx))
        return idx.value

    def set_fields(self, index, fields):
        """fields: two contiguous complex64 torch tensors (cuda) or numpy arrays."""
        import torch

        ptrs, dev = [], None
        for a in fields:
            if isinstance(a, torch.Tensor):
                assert a.dtype == torch.complex64 and a.is_contiguous()
                ptrs.append(a.data_ptr())
                dev = a.is_cuda
            else:
                a = np.ascontiguousarray(a, dtype=np.complex64)
                ptrs.append(a.ctypes.data)
                dev = False
        self._chk(load().brahms_batch_set_fields(self.h, int(index), _ptr_array(ptrs), BRAHMS_C64, int(bool(dev))))

    def set_granularity(self, shape, gx, gy, gt):
        self._chk(load().brahms_batch_set_granularity(self.h, shape, gx, gy, gt))

    def tune(self, tune_steps=16) -> float:
        ms = ctypes.c_double()
        self._chk(load().brahms_batch_tune(self.h, int(tune_steps), ctypes.byref(ms)))
        return ms.value

    def schedule(self, shape):
        v = [ctypes.c_int() for _ in range(4)]
        self._chk(load().brahms_batch_get_schedule(self.h, shape, *[ctypes.byref(x) for x in v]))
        return tuple(x.value for x in v)

    def run(self):
        self._chk(load().brahms_batch_run(self.h))

    def sync(self):
        self._chk(load().brahms_batch_sync(self.h))

    def set_mode(self, mode: int):
        """0 automatic (the tuner picks), 1 grouped, 2 persistent."""
        self._chk(load().brahms_batch_set_mode(self.h, int(mode)))

    def mode(self) -> int:
        return int(load().brahms_batch_get_mode(self.h))

    def set_timeout(self, seconds: float):
        """Limit of each bounded wait of the persistent kernel (default 5 s)."""
        self._chk(load().brahms_batch_set_timeout(self.h, float(seconds)))

    def get_fields(self, index, on_device=False):
        import torch

        shape = self.shapes[index]
        if on_device:
            out = [torch.empty(shape, dtype=torch.complex64, device="cuda") for _ in range(2)]
            ptrs = [t.data_ptr() for t in out]
        else:
            out = [np.empty(shape, dtype=np.complex64) for _ in range(2)]
            ptrs = [a.ctypes.data for a in out]
        self._chk(load().brahms_batch_get_fields(self.h, int(index), _ptr_array(ptrs), BRAHMS_C64,
                                                 int(bool(on_device))))
        return out

    def info(self):
        n, g, t = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        l = ctypes.c_longlong()
        self._chk(load().brahms_batch_info(self.h, ctypes.byref(n), ctypes.byref(g), ctypes.byref(t),
                                           ctypes.byref(l)))
        return {"instances": n.value, "grid": g.value, "threads": t.value, "launches": l.value}

    def close(self):
        if getattr(self, "h", None):
            load().brahms_batch_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def fp32_fma_rate(stream=None) -> float:
    """Measured FP32 FMA rate of the current GPU in TFLOP/s."""
    import torch

    st = stream if stream is not None else torch.cuda.current_stream()
    v = ctypes.c_double()
    _check(None, load().brahms_fp32_fma_rate(_vp(st.cuda_stream), ctypes.byref(v)))
    return v.value


def dsmem_exchange_rate(cluster_ctas: int, smem_bytes: int, stream=None) -> float:
    """Measured all-to-all exchange rate (TB/s) of distributed shared memory
    in clusters of cluster_ctas CTAs with smem_bytes each."""
    import torch

    st = stream if stream is not None else torch.cuda.current_stream()
    v = ctypes.c_double()
    _check(None, load().brahms_dsmem_exchange_rate(int(cluster_ctas), int(smem_bytes), _vp(st.cuda_stream),
                                                   ctypes.byref(v)))
    return v.value


def fail_next_allocations(count: int) -> None:
    """Fault injection for tests: the library's next ``count`` allocations
    report failure (BRAHMS_E_OOM); 0 clears it."""
    _check(None, load().brahms_fail_next_allocations(int(count)))


def pending_allocation_failures() -> int:
    return int(load().brahms_pending_allocation_failures())


def shg_efficiency_function():
    """torch.autograd.Function: eta(phi, dk) for a Solver of SHG fields.

    forward(phi, dk, solver, fields, nz, dz, weights, interval) runs the
    checkpointed forward through brahms_adjoint_forward and returns eta as a
    float64 tensor; backward calls brahms_adjoint_backward with the incoming
    gradient as gscale and returns gradients for phi and dk (CPU float64)."""
    import torch

    class _Eta(torch.autograd.Function):
        @staticmethod
        def forward(ctx, phi, dk, solver, fields, nz, dz, weights, interval):
            J = solver.adjoint_forward(fields, dk.detach().cpu().numpy(), nz, dz, weights,
                                       phi=phi.detach().cpu().numpy(), phi_field=1,
                                       checkpoint_interval=interval)
            ctx.solver = solver
            return torch.tensor(J, dtype=torch.float64)

        @staticmethod
        def backward(ctx, g):
            gphi, gdk = ctx.solver.adjoint_backward(float(g))
            return (torch.from_numpy(gphi), torch.from_numpy(gdk), None, None, None, None, None, None)

    return _Eta
