"""Pins for the oracle's linear step (Eqs. dispOp, diffOp) against closed-form
solutions of the linear PDEs, written here independently of the oracle."""
import math

import numpy as np
import pytest

import oracle
from paper_2609_08384_gb300.workloads import FieldParams, Grid, focused_pulse

FS, UM, MM = 1e-15, 1e-6, 1e-3


def _problem(grid, fields):
    return oracle.make_problem(grid, fields, 0.0)


def _moment2(a, axis_vals, axis):
    """Second moment of |a|^2 along one axis (centred on zero)."""
    p = np.abs(a) ** 2
    other = tuple(i for i in range(3) if i != axis)
    marg = p.sum(axis=other)
    return float(np.sum(marg * axis_vals**2) / np.sum(marg))


def _first_moment(a, axis_vals, axis):
    p = np.abs(a) ** 2
    other = tuple(i for i in range(3) if i != axis)
    marg = p.sum(axis=other)
    return float(np.sum(marg * axis_vals) / np.sum(marg))


def test_focused_beam_reaches_waist_at_centre():
    """Eq. gaussianbeamc input with f = L/2 must follow the textbook waist
    w(z) = w0 sqrt(1 + ((z - f)/z_R)^2) and focus at z = L/2 (pins the sign
    of the diffraction term)."""
    lam, n, w0, L = 1064e-9, 2.156, 30 * UM, 20 * MM
    k = 2 * math.pi * n / lam
    z_r = 0.5 * w0 * w0 * k
    grid = Grid(128, 128, 2, 3.75 * UM, 3.75 * UM, 10 * FS)
    fp = FieldParams(lam, n)
    a = focused_pulse(grid, fp, 1.0, w0, None, L)
    prob = _problem(grid, [fp])
    x, _, _ = grid.axes()
    nz = 8
    dz = L / nz
    cur = a
    for j in range(nz + 1):
        z = j * dz
        w_expect = w0 * math.sqrt(1 + ((z - L / 2) / z_r) ** 2)
        w_got = 2 * math.sqrt(_moment2(cur, x, 2))
        assert abs(w_got / w_expect - 1) < 1e-8, (z, w_got, w_expect)
        if j < nz:
            cur = oracle.linear_step(prob, [cur], dz)[0]
    # minimum at the centre, larger at both faces
    assert 2 * math.sqrt(_moment2(a, x, 2)) > 1.5 * w0


def test_chirped_pulse_gvd_closed_form():
    """dA/dz = -i (k2/2) d2A/dtau2 maps exp(-a tau^2) to exp(-a' tau^2) with
    a' = a / (1 - 2 i k2 a z).  A chirped input (complex a) pins the sign of
    the GVD term, not only its magnitude."""
    k2 = 200 * FS**2 / MM
    tau0 = 20 * FS
    grid = Grid(1, 1, 512, 1.0, 1.0, 2 * FS)
    _, _, t = grid.axes()
    for chirp in (0.0, 1.5, -1.5):
        a = (1 + 1j * chirp) / tau0**2
        A = np.exp(-a * t**2).astype(complex)[:, None, None]
        fp = FieldParams(1064e-9, 2.15, k2=k2)
        prob = _problem(grid, [fp])
        z = 2 * MM
        out = oracle.linear_step(prob, [A], z)[0]
        a_z = a / (1 - 2j * k2 * a * z)
        m2_expect = 1.0 / (4 * a_z.real)
        m2 = _moment2(out, t, 0)
        assert abs(m2 / m2_expect - 1) < 1e-9, (chirp, m2, m2_expect)
        # the full complex envelope, up to its constant prefactor
        ref = np.exp(-a_z * t**2)
        c = np.vdot(ref, out[:, 0, 0]) / np.vdot(ref, ref)
        assert np.abs(out[:, 0, 0] - c * ref).max() < 1e-9 * np.abs(out).max()
        # norm conservation fixes |c|^2 = sqrt(Re a'/Re a) (|A|^2 integrals)
        assert abs(abs(c) ** 2 - math.sqrt(a_z.real / a.real)) < 1e-9


def test_tod_centroid_shift():
    """With k3 only, d/dz A = (k3/6) d3A/dtau3 (unitary reading of the TOD term):
    the centroid of |A|^2 moves as k3 z <Omega^2>/2 = k3 z / (2 tau0^2) for
    exp(-tau^2/tau0^2), and the norm is conserved."""
    k3 = 1000 * FS**3 / MM
    tau0 = 20 * FS
    grid = Grid(1, 1, 1024, 1.0, 1.0, 1 * FS)
    _, _, t = grid.axes()
    A = np.exp(-(t / tau0) ** 2).astype(complex)[:, None, None]
    fp = FieldParams(1064e-9, 2.15, k3=k3)
    prob = _problem(grid, [fp])
    z = 3 * MM
    out = oracle.linear_step(prob, [A], z)[0]
    c = _first_moment(out, t, 0)
    assert abs(c / (k3 * z / (2 * tau0**2)) - 1) < 1e-9
    assert abs(np.sum(np.abs(out) ** 2) / np.sum(np.abs(A) ** 2) - 1) < 1e-13


@pytest.mark.parametrize("m", [3, -5])
def test_walkoff_integer_shift(m):
    """dA/dz = -tan(rho) dA/dx:  A(x, L) = A(x - tan(rho) L, 0).  With
    tan(rho) L = m dx the result is an exact circular shift by m samples,
    even when split into steps of non-integer shift."""
    grid = Grid(16, 8, 4, 2 * UM, 2 * UM, 10 * FS)
    rng = np.random.default_rng(11)
    A = rng.standard_normal((4, 8, 16)) + 1j * rng.standard_normal((4, 8, 16))
    L = 1 * MM
    rho = math.atan(m * grid.dx / L)
    # a vanishing wavelength makes k = 2 pi n / lambda huge and diffraction negligible
    fp = FieldParams(1e-30, 1.0, rho=rho)
    prob = _problem(grid, [fp])
    nz = 7
    cur = A
    for _ in range(nz):
        cur = oracle.linear_step(prob, [cur], L / nz)[0]
    assert np.abs(cur - np.roll(A, m, axis=2)).max() < 1e-13 * np.abs(A).max() * 10


@pytest.mark.parametrize("m", [4, -3])
def test_gvm_integer_shift(m):
    """dA/dz = -delta dA/dtau: A(tau, L) = A(tau - delta L, 0)."""
    grid = Grid(4, 2, 32, 2 * UM, 2 * UM, 10 * FS)
    rng = np.random.default_rng(12)
    A = rng.standard_normal((32, 2, 4)) + 1j * rng.standard_normal((32, 2, 4))
    L = 2 * MM
    fp = FieldParams(1e-30, 1.0, delta=m * grid.dt / L)
    prob = _problem(grid, [fp])
    cur = A
    for _ in range(5):
        cur = oracle.linear_step(prob, [cur], L / 5)[0]
    assert np.abs(cur - np.roll(A, m, axis=0)).max() < 1e-13 * np.abs(A).max() * 10


def test_loss_decay_composition_unitarity():
    grid = Grid(8, 8, 16, 3 * UM, 3 * UM, 20 * FS)
    rng = np.random.default_rng(13)
    A = rng.standard_normal((16, 8, 8)) + 1j * rng.standard_normal((16, 8, 8))
    fp = FieldParams(1450e-9, 2.14, delta=1e-10, k2=1e-25, k3=3e-40, rho=2e-3)
    prob = _problem(grid, [fp])
    # composition: 6 steps of dz equal one step of 6 dz
    six = A
    for _ in range(6):
        six = oracle.linear_step(prob, [six], 0.1 * MM)[0]
    one = oracle.linear_step(prob, [A], 0.6 * MM)[0]
    assert np.abs(six - one).max() < 1e-13 * np.abs(A).max() * 10
    # unitary without loss
    assert abs(np.sum(np.abs(one) ** 2) / np.sum(np.abs(A) ** 2) - 1) < 1e-14
    # loss alpha: |A|^2 decays as exp(-alpha z)
    fp2 = FieldParams(1450e-9, 2.14, delta=1e-10, k2=1e-25, alpha=50.0)
    out = oracle.linear_step(_problem(grid, [fp2]), [A], 2 * MM)[0]
    assert abs(np.sum(np.abs(out) ** 2) / np.sum(np.abs(A) ** 2) - math.exp(-50.0 * 2 * MM)) < 1e-14
