"""Thermal model on the GPU against the FP64 oracle (Sec. 4.1: heat equation on
the fields' grid, temperature-dependent phase mismatch).

Tolerances: the heat load squares FP32 fields (FP32 partial sums of four
squares, FP64 accumulation), 1e-6 of its maximum; the solve is FP64 on both
sides (sine-transform diagonalisation against a sparse direct solve),
1e-11 of the maximum temperature."""
import math

import numpy as np
import pytest

import oracle
from paper_2609_08384_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

HEAT_TOL = 1e-6
SOLVE_TOL = 1e-11


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2609_08384_gb300 import build
    build.build()


def _br():
    import paper_2609_08384_gb300 as br
    return br


def _c64(a):
    return np.ascontiguousarray(a, dtype=np.complex64)


def _dev(arrs):
    return [torch.from_numpy(_c64(a)).cuda() for a in arrs]


def _fields(nf):
    lam = [wl.LAM_P, wl.LAM_S, wl.LAM_I] if nf == 3 else [wl.LAM_SH, wl.LAM_F]
    n = [wl.N_P, wl.N_S, wl.N_I] if nf == 3 else [wl.N_SH, wl.N_F]
    alpha = [25.0, 0.0, 40.0] if nf == 3 else [30.0, 12.0]
    return [wl.FieldParams(lam[f], n[f], alpha=alpha[f]) for f in range(nf)]


def _random_fields(g, nf, rng, amp=3e7):
    shape = (g.nt, g.ny, g.nx)
    return [_c64(amp * (rng.standard_normal(shape) + 1j * rng.standard_normal(shape))) for _ in range(nf)]


@pytest.mark.parametrize("shape,nf", [((64, 48, 128), 2), ((32, 32, 96), 3), ((128, 96, 1), 2),
                                      ((2, 2, 2), 3), ((6, 1, 24), 2), ((1024, 2, 8), 3)])
def test_heat_load_parity(shape, nf):
    br = _br()
    nx, ny, nt = shape
    g = wl.Grid(nx, ny, nt, 2e-6, 3e-6, 10e-15)
    fields = _fields(nf)
    rng = np.random.default_rng(11 + nx + ny + nt)
    a1, a2 = _random_fields(g, nf, rng), _random_fields(g, nf, rng, amp=1e7)
    rep = 50e6
    s = br.Solver(g, fields, wl.D_EFF, 0.0)
    s.set_fields(_dev(a1))
    s.heat_accumulate(rep, 1.0)
    s.set_fields(_dev(a2))
    s.heat_accumulate(rep, 0.5)
    # the load is read back through the FP64 solve and the stencil: Q = kappa A T
    t_gpu = s.thermal_map(1.0, 0.0)
    s.close()
    q_gpu = (oracle.thermal_matrix(nx, ny, g.dx, g.dy) @ t_gpu.ravel()).reshape(ny, nx)
    prob = oracle.make_problem(g, fields, wl.D_EFF)
    q = oracle.heat_load(prob, a1, rep) + 0.5 * oracle.heat_load(prob, a2, rep)
    err = np.abs(q_gpu - q).max() / np.abs(q).max()
    assert err < HEAT_TOL, err


@pytest.mark.parametrize("nx,ny", [(64, 48), (96, 192), (2, 2), (768, 1), (12, 6), (4096, 2), (2, 4096),
                                   (256, 256), (384, 24)])
def test_thermal_solve_parity(nx, ny):
    br = _br()
    g = wl.Grid(nx, ny, 1, 2.5e-6, 4e-6, 1e-15)
    rng = np.random.default_rng(nx * 7 + ny)
    q = rng.standard_normal((ny, nx)) * 1e9 + 5e8
    s = br.Solver(g, _fields(2), wl.D_EFF, 0.0)
    s.heat_set(q)
    t = s.thermal_map(4.6, 0.0)
    s.close()
    want = oracle.thermal_solve(q, g.dx, g.dy, 4.6)
    err = np.abs(t - want).max() / np.abs(want).max()
    assert err < SOLVE_TOL, err


@pytest.mark.parametrize("n", [4096, 768])
def test_thermal_solve_full_size_eigenmodes(n):
    """n x n: the discrete eigenmodes sin(pi k (j + 1/2) / n) solve to Q / (kappa mu) for
    the lowest, a middle and the highest mode (any size; the oracle's direct solve is too
    slow here)."""
    br = _br()
    g = wl.Grid(n, n, 1, 1.5e-6, 1.5e-6, 1e-15)
    kap = 5.0
    s = br.Solver(g, _fields(2), wl.D_EFF, 0.0)
    j = np.arange(n)
    for kx, ky in ((1, 1), (n // 3, 17), (n, n)):
        qx = np.sin(math.pi * kx * (j + 0.5) / n)
        qy = np.sin(math.pi * ky * (j + 0.5) / n)
        q = np.outer(qy, qx)
        mu = 4 * (math.sin(math.pi * kx / (2 * n)) ** 2 + math.sin(math.pi * ky / (2 * n)) ** 2) / g.dx**2
        s.heat_set(q)
        t = s.thermal_map(kap, 0.0)
        want = q / (kap * mu)
        err = np.abs(t - want).max() / np.abs(want).max()
        # rounding in the low sine coefficients is amplified by mu / mu_min relative
        # to a high mode (the problem's conditioning); a wrong eigenvalue is an O(1) error
        mu_min = 8 * math.sin(math.pi / (2 * n)) ** 2 / g.dx**2
        assert err < max(SOLVE_TOL, 1e-15 * mu / mu_min), (kx, ky, err)
    s.close()


def test_thermal_map_drives_the_mismatch_map():
    """cw SHG with absorption: heat load sampled at z = 0, L/2, L (trapezoid
    weights), the thermal map from it, then a propagation under that map --
    the same chain through the oracle (heat_load, thermal_solve, propagate_map)."""
    br = _br()
    n_f, n_sh, lam, w0 = wl.N_F, wl.N_SH, wl.LAM_F, 25e-6
    fields = [wl.FieldParams(lam / 2, n_sh, alpha=40.0), wl.FieldParams(lam, n_f, alpha=15.0)]
    g = wl.Grid(128, 96, 1, 2.5e-6, 3e-6, 1e-15)
    x, y, _ = g.axes()
    r2 = x[None, :] ** 2 + y[:, None] ** 2
    a_f = (3e7 * np.exp(-r2 / w0**2))[None].astype(np.complex128)
    a_sh = np.zeros_like(a_f)
    L, nz, dk = 4e-3, 80, 150.0
    dz = L / nz
    prob = oracle.make_problem(g, fields, wl.D_EFF)
    kap = 4.6
    # oracle chain
    f0 = [a_sh, a_f]
    fh, _ = oracle.propagate(prob, f0, nz // 2, dz, dk)
    fl, _ = oracle.propagate(prob, list(fh), nz // 2, dz, dk, phi0=dk * L / 2)
    q = (0.25 * oracle.heat_load(prob, f0) + 0.5 * oracle.heat_load(prob, list(fh))
         + 0.25 * oracle.heat_load(prob, list(fl)))
    t_orc = oracle.thermal_solve(q, g.dx, g.dy, kap)
    dkdT = 3.0 / (t_orc.max() * L)  # about 3 rad of thermal dephasing on axis
    want, _ = oracle.propagate_map(prob, f0, nz, dz, dk, dkdT * t_orc)
    # GPU chain
    s = br.Solver(g, fields, wl.D_EFF, dk)
    s.set_fields(_dev(f0))
    s.heat_accumulate(0.0, 0.25)
    s.propagate(nz // 2, dz)
    s.heat_accumulate(0.0, 0.5)
    s.propagate(nz // 2, dz)
    s.heat_accumulate(0.0, 0.25)
    t_gpu = s.thermal_map(kap, dkdT)
    s.set_fields(_dev(f0))
    s.propagate(nz, dz)
    got = [np.asarray(x) for x in s.get_fields()]
    s.close()
    assert np.abs(t_gpu - t_orc).max() / t_orc.max() < 1e-5
    for f in range(2):
        err = np.linalg.norm(got[f] - want[f]) / np.linalg.norm(want[f])
        assert err < 1e-4, (f, err)
    # the map matters: without it the SH differs by far more than the tolerance
    plain, _ = oracle.propagate(prob, f0, nz, dz, dk)
    assert np.linalg.norm(plain[0] - want[0]) / np.linalg.norm(want[0]) > 1e-2


def test_z_resolved_thermal_map_drives_the_mismatch_map():
    """Two z-segments with their own heat loads (strong cw SHG whose load grows
    along z as the absorbing SH builds up): each segment's load sampled at
    its ends and middle (trapezoid), one temperature per segment, and the
    propagation under the z-resolved map -- the same chain through the oracle
    (heat_load, thermal_solve per segment, propagate_map_z)."""
    br = _br()
    n_f, n_sh, lam, w0 = wl.N_F, wl.N_SH, wl.LAM_F, 25e-6
    fields = [wl.FieldParams(lam / 2, n_sh, alpha=60.0), wl.FieldParams(lam, n_f, alpha=5.0)]
    g = wl.Grid(96, 64, 1, 2.5e-6, 3e-6, 1e-15)
    x, y, _ = g.axes()
    r2 = x[None, :] ** 2 + y[:, None] ** 2
    a_f = (2e7 * np.exp(-r2 / w0**2))[None].astype(np.complex128)
    a_sh = np.zeros_like(a_f)
    L, nz, dk = 4e-3, 80, 0.0
    dz = L / nz
    q4 = nz // 4
    prob = oracle.make_problem(g, fields, wl.D_EFF)
    kap = 4.6
    # oracle chain: fields at z = 0, L/4, L/2, 3L/4, L without a map
    f = [[a_sh, a_f]]
    ph = 0.0
    for _ in range(4):
        nxt, ph = oracle.propagate(prob, list(f[-1]), q4, dz, dk, phi0=ph)
        f.append(list(nxt))
    q = [oracle.heat_load(prob, a) for a in f]
    q_seg = [0.25 * q[0] + 0.5 * q[1] + 0.25 * q[2], 0.25 * q[2] + 0.5 * q[3] + 0.25 * q[4]]
    t_orc = np.stack([oracle.thermal_solve(qs, g.dx, g.dy, kap) for qs in q_seg])
    assert t_orc[1].max() > 1.5 * t_orc[0].max()  # the load grows along z
    dkdT = 6.0 / (t_orc.max() * L)
    want, _ = oracle.propagate_map_z(prob, f[0], nz, dz, dk, [L / 2], dkdT * t_orc)
    # GPU chain
    s = br.Solver(g, fields, wl.D_EFF, dk)
    s.set_dk_map_z([L / 2])
    s.set_fields(_dev(f[0]))
    s.heat_accumulate(0.0, 0.25, segment=0)
    s.propagate(q4, dz)
    s.heat_accumulate(0.0, 0.5)                 # z = L/4: the segment that holds z
    s.propagate(q4, dz)
    s.heat_accumulate(0.0, 0.25, segment=0)
    s.heat_accumulate(0.0, 0.25, segment=1)
    s.propagate(q4, dz)
    s.heat_accumulate(0.0, 0.5)                 # z = 3L/4
    s.propagate(q4, dz)
    s.heat_accumulate(0.0, 0.25, segment=1)
    t_gpu = s.thermal_map(kap, dkdT)
    assert t_gpu.shape == (2, g.ny, g.nx)
    s.set_fields(_dev(f[0]))
    s.propagate(nz, dz)
    got = [np.asarray(a) for a in s.get_fields()]
    s.close()
    assert np.abs(t_gpu - t_orc).max() / t_orc.max() < 1e-5
    for k in range(2):
        err = np.linalg.norm(got[k] - want[k]) / np.linalg.norm(want[k])
        assert err < 1e-4, (k, err)
    # the z-averaged map (one segment under the mean load) gives another result
    avg, _ = oracle.propagate_map(prob, f[0], nz, dz, dk, dkdT * oracle.thermal_solve(0.5 * (q_seg[0] + q_seg[1]),
                                                                                       g.dx, g.dy, kap))
    assert np.linalg.norm(avg[0] - want[0]) / np.linalg.norm(want[0]) > 3e-3


def test_z_segment_status_codes():
    br = _br()
    g = wl.Grid(16, 8, 4, 2e-6, 2e-6, 10e-15)
    s = br.Solver(g, _fields(2), wl.D_EFF, 0.0)
    for edges in ([0.0], [2e-3, 1e-3], [float("nan")], [-1e-3]):
        with pytest.raises(br.BrahmsError) as ei:
            s.set_dk_map_z(edges)
        assert ei.value.status == br.BRAHMS_E_ARG
    s.set_dk_map_z([1e-3, 2e-3])
    z = np.zeros((4, 8, 16), np.complex64)
    s.set_fields(_dev([z, z]))
    with pytest.raises(br.BrahmsError) as ei:
        s.heat_accumulate(0.0, 1.0, segment=3)
    assert ei.value.status == br.BRAHMS_E_ARG
    s.heat_accumulate(0.0, 1.0, segment=0)
    with pytest.raises(br.BrahmsError) as ei:
        s.thermal_map(1.0, 1.0)  # segments 1 and 2 have no load
    assert ei.value.status == br.BRAHMS_E_STATE
    s.heat_set(np.ones((3, 8, 16)))
    t = s.thermal_map(1.0, 1.0)
    assert t.shape == (3, 8, 16) and (t > 0).all()
    # the adjoint takes up to 16 z-segments
    s.adjoint_forward(_dev([z, z]), np.zeros(2), 2, 1e-5, np.array([1.0, 0.0]))
    s.set_dk_map_z(1e-4 * np.arange(1, 17))
    with pytest.raises(br.BrahmsError) as ei:
        s.adjoint_forward(_dev([z, z]), np.zeros(2), 2, 1e-5, np.array([1.0, 0.0]))
    assert ei.value.status == br.BRAHMS_E_STATE
    s.set_dk_map(None)  # back to one segment
    s.adjoint_forward(_dev([z, z]), np.zeros(2), 2, 1e-5, np.array([1.0, 0.0]))
    s.close()


def test_thermal_map_adds_to_a_static_map():
    """A fan-out grating map M set by set_dk_map stays under the thermal map:
    the propagation runs with M + dkdT T, as the oracle's under the same sum."""
    br = _br()
    fields = [wl.FieldParams(wl.LAM_SH, wl.N_SH, alpha=30.0), wl.FieldParams(wl.LAM_F, wl.N_F, alpha=12.0)]
    g = wl.Grid(64, 48, 1, 3e-6, 3e-6, 1e-15)
    x, y, _ = g.axes()
    r2 = x[None, :] ** 2 + y[:, None] ** 2
    a_f = (3e7 * np.exp(-r2 / (25e-6) ** 2))[None].astype(np.complex128)
    f0 = [np.zeros_like(a_f), a_f]
    m = np.tile(4e6 * x, (g.ny, 1))
    rng = np.random.default_rng(5)
    q = 1e12 * np.exp(-r2 / (30e-6) ** 2) + 1e10 * rng.random((g.ny, g.nx))
    kap, nz, dz, dk = 4.6, 40, 50e-6, 100.0
    t_orc = oracle.thermal_solve(q, g.dx, g.dy, kap)
    dkdT = 2.0 / (t_orc.max() * nz * dz)
    prob = oracle.make_problem(g, fields, wl.D_EFF)
    want, _ = oracle.propagate_map(prob, f0, nz, dz, dk, m + dkdT * t_orc)
    s = br.Solver(g, fields, wl.D_EFF, dk)
    s.set_dk_map(m)
    s.heat_set(q)
    s.thermal_map(kap, dkdT)
    s.set_fields(_dev(f0))
    s.propagate(nz, dz)
    got = [np.asarray(a) for a in s.get_fields()]
    s.close()
    for f in range(2):
        err = np.linalg.norm(got[f] - want[f]) / np.linalg.norm(want[f])
        assert err < 1e-4, (f, err)
    # without the static map the result is clearly different
    alt, _ = oracle.propagate_map(prob, f0, nz, dz, dk, dkdT * t_orc)
    assert np.linalg.norm(alt[0] - want[0]) / np.linalg.norm(want[0]) > 1e-2


def test_thermal_status_codes():
    br = _br()
    g = wl.Grid(16, 8, 4, 2e-6, 2e-6, 10e-15)
    s = br.Solver(g, _fields(2), wl.D_EFF, 0.0)
    with pytest.raises(br.BrahmsError) as ei:
        s.heat_accumulate(1.0, 1.0)
    assert ei.value.status == br.BRAHMS_E_STATE  # no fields
    with pytest.raises(br.BrahmsError) as ei:
        s.thermal_map(1.0, 0.0)
    assert ei.value.status == br.BRAHMS_E_STATE  # no load
    z = np.zeros((4, 8, 16), np.complex64)
    s.set_fields(_dev([z, z]))
    with pytest.raises(br.BrahmsError) as ei:
        s.heat_accumulate(-1.0, 1.0)
    assert ei.value.status == br.BRAHMS_E_ARG
    q = np.ones((8, 16))
    q[3, 5] = np.nan
    with pytest.raises(br.BrahmsError) as ei:
        s.heat_set(q)
    assert ei.value.status == br.BRAHMS_E_ARG
    s.heat_set(None)
    for bad in (0.0, -2.0, float("inf")):
        with pytest.raises(br.BrahmsError) as ei:
            s.thermal_map(bad, 0.0)
        assert ei.value.status == br.BRAHMS_E_ARG
    t = s.thermal_map(1.0, 1.0)  # zero load: zero temperature, zero map
    assert not t.any()
    # an overflowing load: finite fields, a weight that takes the FP64 load past 1e308
    big = np.full((4, 8, 16), 1e10, np.complex64)
    s.set_fields(_dev([big, big]))
    s.heat_set(None)
    s.heat_accumulate(1.0, 1e308)
    with pytest.raises(br.BrahmsError) as ei:
        s.thermal_map(1.0, 1.0)
    assert ei.value.status == br.BRAHMS_E_NONFINITE
    # the context stays usable: a finite load solves again
    s.heat_set(np.ones((8, 16)))
    assert np.isfinite(s.thermal_map(1.0, 1.0)).all()
    s.close()
