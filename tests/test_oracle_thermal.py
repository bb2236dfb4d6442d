"""Oracle pins for the thermal model (Sec. 4.1: the steady-state heat equation
lap T = -Q / kappa on the fields' grid; heat load from the absorbed power).

The solve is pinned by what the discrete and continuum problems fix:
- the discrete eigenmodes sin(pi k (j + 1/2) / n) of the 3-point second
  difference with T = 0 half a cell outside the window, eigenvalue
  4 sin^2(pi k / (2n)) / d^2 (derived from the stencil, not from the code);
- second-order convergence to a continuum solution with T = 0 on the faces
  x = x_{-1/2}, x_{n-1/2} (and in y);
- the discrete heat-flux balance: the total load equals the flux through the
  side faces, kappa * 2 T_edge / d per edge cell (the stencil telescopes).
The heat load is pinned by the absorbed power of a Gaussian beam or pulse and
by the loss rate of the oracle's own linear step (alpha as the intensity
absorption coefficient)."""
import math

import numpy as np
import pytest

import oracle
from paper_2609_08384_gb300 import workloads as wl

C0, EPS0 = wl.C0, wl.EPS0


def _mode(n, k):
    j = np.arange(n)
    return np.sin(math.pi * k * (j + 0.5) / n)


@pytest.mark.parametrize("nx,ny", [(12, 8), (16, 1), (6, 9)])
def test_discrete_eigenmodes(nx, ny):
    dx, dy, kap = 3e-6, 5e-6, 4.6
    for kx, ky in ((1, 1), (2, 3), (nx, 1), (nx - 1, ny)):
        ky = min(ky, ny)
        qx = _mode(nx, kx)
        qy = _mode(ny, ky) if ny > 1 else np.ones(1)
        q = np.outer(qy, qx)
        mu = 4 * math.sin(math.pi * kx / (2 * nx)) ** 2 / dx**2
        if ny > 1:
            mu += 4 * math.sin(math.pi * ky / (2 * ny)) ** 2 / dy**2
        t = oracle.thermal_solve(q, dx, dy, kap)
        np.testing.assert_allclose(t, q / (kap * mu), rtol=0, atol=1e-12 * np.abs(q / (kap * mu)).max())


def _continuum_error(n, ny_is_one=False):
    """T = 16 T0 u(1-u) v(1-v) on the window [x_{-1/2}, x_{n-1/2}] (width n dx),
    -kappa lap T = 32 kappa T0 (v(1-v)/Lx^2 + u(1-u)/Ly^2)."""
    lx, ly, kap, t0 = 1e-3, 0.6e-3, 5.0, 2.0
    dx, dy = lx / n, ly / n
    u = (np.arange(n) + 0.5) / n  # distance from the face x_{-1/2}, in units of lx
    if ny_is_one:
        t_ex = 4 * t0 * u * (1 - u)
        q = np.full(n, 8 * kap * t0 / lx**2)[None, :]
        return np.abs(oracle.thermal_solve(q, dx, dy, kap)[0] - t_ex).max()
    v = u.copy()
    uu, vv = np.meshgrid(u, v)
    t_ex = 16 * t0 * uu * (1 - uu) * vv * (1 - vv)
    q = 32 * kap * t0 * (vv * (1 - vv) / lx**2 + uu * (1 - uu) / ly**2)
    return np.abs(oracle.thermal_solve(q, dx, dy, kap) - t_ex).max()


@pytest.mark.parametrize("one_d", [False, True])
def test_second_order_convergence_to_continuum(one_d):
    errs = [_continuum_error(n, one_d) for n in (16, 32, 64, 128)]
    slopes = [math.log2(errs[i] / errs[i + 1]) for i in range(3)]
    assert all(1.9 < s < 2.1 for s in slopes), slopes
    assert errs[-1] < 2e-4  # of T0 = 2 K


@pytest.mark.parametrize("nx,ny", [(24, 16), (32, 1)])
def test_heat_flux_balance(nx, ny):
    rng = np.random.default_rng(7)
    dx, dy, kap = 2e-6, 3e-6, 3.3
    q = rng.random((ny, nx)) * 1e9
    t = oracle.thermal_solve(q, dx, dy, kap)
    total = q.sum() * dx * dy
    flux = kap * dy * (2 * (t[:, 0] + t[:, -1]) / dx).sum()
    if ny > 1:
        flux += kap * dx * (2 * (t[0, :] + t[-1, :]) / dy).sum()
    assert flux == pytest.approx(total, rel=1e-11)
    assert (t > 0).all()  # a positive source heats every point (maximum principle)


def _fields():
    return [wl.FieldParams(wl.LAM_SH, wl.N_SH, alpha=30.0), wl.FieldParams(wl.LAM_F, wl.N_F, alpha=12.0)]


def test_heat_load_gaussian_beam_cw():
    g = wl.Grid(96, 96, 1, 2.5e-6, 3e-6, 1e-15)
    x, y, _ = g.axes()
    r2 = x[None, :] ** 2 + y[:, None] ** 2
    fields = _fields()
    a0, w0 = [2e6, 5e6], [22e-6, 30e-6]
    arrs = [(a0[f] * np.exp(-r2 / w0[f] ** 2))[None].astype(np.complex128) for f in range(2)]
    q = oracle.heat_load(oracle.make_problem(g, fields, wl.D_EFF), arrs, rep_rate=123.0)  # ignored for nt = 1
    want = sum(fields[f].alpha * 0.5 * C0 * EPS0 * fields[f].n * a0[f] ** 2 * math.pi * w0[f] ** 2 / 2
               for f in range(2))
    assert q.sum() * g.dx * g.dy == pytest.approx(want, rel=1e-12)
    # on axis: sum_f alpha_f I_f
    want0 = sum(fields[f].alpha * 0.5 * C0 * EPS0 * fields[f].n * a0[f] ** 2 for f in range(2))
    assert q[48, 48] == pytest.approx(want0, rel=1e-14)


def test_heat_load_pulse_train_and_linear_step_loss():
    g = wl.Grid(48, 48, 64, 5e-6, 5e-6, 15e-15)
    x, y, t = g.axes()
    fields = _fields()
    prob = oracle.make_problem(g, fields, wl.D_EFF)
    a0, w0, tau0 = [3e7, 1e7], [28e-6, 24e-6], [90e-15, 120e-15]
    arrs = []
    for f in range(2):
        r2 = x[None, None, :] ** 2 + y[None, :, None] ** 2
        arrs.append((a0[f] * np.exp(-r2 / w0[f] ** 2 - t[:, None, None] ** 2 / tau0[f] ** 2)).astype(np.complex128))
    rep = 80e6
    q = oracle.heat_load(prob, arrs, rep_rate=rep)
    e_pulse = [0.5 * C0 * EPS0 * fields[f].n * a0[f] ** 2 * math.pi * w0[f] ** 2 / 2 * tau0[f] * math.sqrt(math.pi / 2)
               for f in range(2)]
    absorbed = q.sum() * g.dx * g.dy
    assert absorbed == pytest.approx(rep * sum(fields[f].alpha * e_pulse[f] for f in range(2)), rel=1e-12)
    # the same number from the linear step's loss: E_f(dz) = E_f(0) exp(-alpha_f dz)
    dz = 1e-4
    e0, _ = oracle.energy(prob, arrs)
    e1, _ = oracle.energy(prob, list(oracle.linear_step(prob, arrs, dz)))
    rate = sum(-math.log(e1[f] / e0[f]) / dz * e0[f] for f in range(2))
    assert absorbed == pytest.approx(rep * rate, rel=1e-10)
