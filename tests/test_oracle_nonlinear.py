"""Pins for the oracle's nonlinear coupling (Eqs. CEp/CEs/CEi and the 2-field
SHG reading), through its full split-step propagation, against closed-form
plane-wave solutions derived here from the coupled equations."""
import math

import numpy as np
import pytest

import oracle
from paper_2609_08384_gb300.workloads import (C0, FieldParams, Grid, HBAR, N_F, N_SH, D_EFF,
                                              LAM_F, LAM_SH)

UM, MM, FS = 1e-6, 1e-3, 1e-15


def _uniform(grid, val):
    return np.full((grid.nt, grid.ny, grid.nx), val, dtype=complex)


# A 2x2x2 grid with uniform fields is a plane-wave, cw problem: only the DC
# bin is populated and the linear multiplier there is exactly 1.
PW = Grid(2, 2, 2, 1 * UM, 1 * UM, 10 * FS)


def _shg_fields():
    return [FieldParams(LAM_SH, N_SH, delta=1e-10, k2=1e-25, rho=1e-3),
            FieldParams(LAM_F, N_F, delta=0.0, k2=2e-25)]


def test_shg_tanh2_plane_wave():
    """Delta k = 0, uniform F input a:  eta = tanh^2(Gamma L) with
    Gamma = kappa_F |a| sqrt(n_F/n_SH), and A_SH = i sqrt(n_F/n_SH) a tanh,
    A_F = a sech (derived from the 2-field equations with the 1/2 factor)."""
    fields = _shg_fields()
    prob = oracle.make_problem(PW, fields, D_EFF)
    kF = 2 * math.pi * D_EFF / (N_F * LAM_F)
    a = 5.9e7 * np.exp(0.3j)
    gamma = kF * abs(a) * math.sqrt(N_F / N_SH)
    L = 2.2 / gamma
    out, _ = oracle.propagate(prob, [_uniform(PW, 0), _uniform(PW, a)], 400, L / 400, 0.0)
    sh, f = out[0, 0, 0, 0], out[1, 0, 0, 0]
    th = math.tanh(gamma * L)
    # phases: A_F keeps arg(a); A_SH = i * a^2/|a| * ... -> arg(i a^2 / |a|)
    expect_sh = 1j * math.sqrt(N_F / N_SH) * th * a * a / abs(a)
    expect_f = a / math.cosh(gamma * L)
    assert abs(sh - expect_sh) / abs(a) < 1e-9
    assert abs(f - expect_f) / abs(a) < 1e-9
    eta = N_SH * abs(sh) ** 2 / (N_F * abs(a) ** 2)
    assert abs(eta - th**2) < 1e-9


@pytest.mark.parametrize("dk", [0.0, 900.0, -2500.0])
def test_shg_undepleted_sinc(dk):
    """Weak F input a, mismatch dk:  A_SH(L) = i (kappa_SH/2) a^2 L
    exp(-i dk L/2) sinc(dk L/2).  Pins the sign and the place of the mismatch
    phase, the RK4 stage z-values and the 1/2 degeneracy factor."""
    fields = _shg_fields()
    prob = oracle.make_problem(PW, fields, D_EFF)
    kSH = 2 * math.pi * D_EFF / (N_SH * LAM_SH)
    a = 1.0 + 0.5j
    L = 3 * MM
    nz = 300
    out, phi = oracle.propagate(prob, [_uniform(PW, 0), _uniform(PW, a)], nz, L / nz, dk)
    x = dk * L / 2
    sinc = 1.0 if x == 0 else math.sin(x) / x
    expect = 1j * (kSH / 2) * a * a * L * np.exp(-1j * dk * L / 2) * sinc
    assert abs(out[0, 0, 0, 0] - expect) / abs(kSH * a * a * L) < 1e-9
    assert abs(phi - dk * L) < 1e-12 * max(1.0, abs(dk * L))


def _opg_fields():
    lp, ls = 1064e-9, 1450e-9
    li = 1.0 / (1.0 / lp - 1.0 / ls)  # omega_p = omega_s + omega_i exactly
    return [FieldParams(lp, 2.15, delta=1e-10, k2=2e-25, rho=2e-3),
            FieldParams(ls, 2.14, k2=1e-25),
            FieldParams(li, 2.08, delta=-1e-10, k2=5e-26, rho=1e-3)]


@pytest.mark.parametrize("dk", [0.0, 700.0, -1800.0])
def test_three_wave_undepleted_sinc(dk):
    """Weak generated field from two strong constant ones:
      SFG  A_p(L) = i kappa_p A_s A_i L exp(-i dk L/2) sinc(dk L/2)
      DFG  A_s(L) = i kappa_s A_p A_i^* L exp(+i dk L/2) sinc(dk L/2)
      DFG  A_i(L) = i kappa_i A_p A_s^* L exp(+i dk L/2) sinc(dk L/2)
    (each from integrating one of Eqs. CEp/CEs/CEi with the others fixed)."""
    fields = _opg_fields()
    prob = oracle.make_problem(PW, fields, D_EFF)
    kap = [2 * math.pi * D_EFF / (f.n * f.lambda_) for f in fields]
    L = 2 * MM
    nz = 200
    x = dk * L / 2
    sinc = 1.0 if x == 0 else math.sin(x) / x
    big1, big2 = 1.0 + 0.2j, 0.7 - 0.4j
    for gen in range(3):
        vals = [big1, big2]
        init = []
        it = iter(vals)
        for f in range(3):
            init.append(0j if f == gen else next(it))
        out, _ = oracle.propagate(prob, [_uniform(PW, v) for v in init], nz, L / nz, dk)
        A = init
        if gen == 0:
            expect = 1j * kap[0] * A[1] * A[2] * L * np.exp(-1j * dk * L / 2) * sinc
        elif gen == 1:
            expect = 1j * kap[1] * A[0] * np.conj(A[2]) * L * np.exp(1j * dk * L / 2) * sinc
        else:
            expect = 1j * kap[2] * A[0] * np.conj(A[1]) * L * np.exp(1j * dk * L / 2) * sinc
        assert abs(out[gen, 0, 0, 0] - expect) / (kap[gen] * L) < 1e-9, gen


def test_parametric_gain_cosh_sinh():
    """Undepleted pump a, dk = 0, seed A_s0:  A_s = A_s0 cosh(g z),
    A_i = i sqrt(kappa_i/kappa_s) (a/|a|) A_s0^* sinh(g z), g = |a| sqrt(kappa_s kappa_i)."""
    fields = _opg_fields()
    prob = oracle.make_problem(PW, fields, D_EFF)
    kap = [2 * math.pi * D_EFF / (f.n * f.lambda_) for f in fields]
    a = 5.9e7 * np.exp(0.7j)
    g = abs(a) * math.sqrt(kap[1] * kap[2])
    L = 3.0 / g
    s0 = 1e-3 * abs(a) * np.exp(-0.4j)  # weak seed: pump depletion ~1e-6 * e^6 stays below tolerance
    out, _ = oracle.propagate(prob, [_uniform(PW, a), _uniform(PW, s0), _uniform(PW, 0)], 600, L / 600, 0.0)
    es = s0 * math.cosh(g * L)
    ei = 1j * math.sqrt(kap[2] / kap[1]) * (a / abs(a)) * np.conj(s0) * math.sinh(g * L)
    assert abs(out[1, 0, 0, 0] - es) / abs(es) < 2e-4
    assert abs(out[2, 0, 0, 0] - ei) / abs(ei) < 2e-4
    # with a 1e-6 seed the undepleted solution is exact to ~1e-10
    s0 = 1e-6 * abs(a)
    out, _ = oracle.propagate(prob, [_uniform(PW, a), _uniform(PW, s0), _uniform(PW, 0)], 600, L / 600, 0.0)
    assert abs(out[1, 0, 0, 0] - s0 * math.cosh(g * L)) / abs(s0 * math.cosh(g * L)) < 1e-8


def _random_smooth(grid, rng, amp):
    """Band-limited random complex field (no content near the grid's Nyquist)."""
    spec = rng.standard_normal((grid.nt, grid.ny, grid.nx)) + 1j * rng.standard_normal((grid.nt, grid.ny, grid.nx))
    kt = np.fft.fftfreq(grid.nt)[:, None, None]
    ky = np.fft.fftfreq(grid.ny)[None, :, None]
    kx = np.fft.fftfreq(grid.nx)[None, None, :]
    spec *= np.exp(-(kt**2 + ky**2 + kx**2) / (2 * 0.08**2))
    f = np.fft.ifftn(spec)
    return amp * f / np.abs(f).max()


def test_energy_and_manley_rowe_invariants():
    """alpha = 0: total energy sum n |A|^2 and the Manley-Rowe photon-flux
    combinations are constants of the coupled equations (all linear terms
    are unitary and commute with the sums)."""
    grid = Grid(16, 12, 24, 4 * UM, 4 * UM, 25 * FS)
    fields = _opg_fields()
    prob = oracle.make_problem(grid, fields, D_EFF)
    rng = np.random.default_rng(3)
    init = [_random_smooth(grid, rng, 3e7) for _ in range(3)]
    out, _ = oracle.propagate(prob, init, 60, 5 * UM, 350.0)

    def flux(arrs):
        return [f.n * np.sum(np.abs(a) ** 2) * f.lambda_ / (2 * math.pi * C0) for f, a in zip(fields, arrs)]

    def energy(arrs):
        return sum(f.n * np.sum(np.abs(a) ** 2) for f, a in zip(fields, arrs))

    e0, e1 = energy(init), energy(out)
    assert abs(e1 / e0 - 1) < 1e-10
    f0, f1 = flux(init), flux(out)
    assert abs((f1[0] + f1[1]) / (f0[0] + f0[1]) - 1) < 1e-10
    assert abs((f1[1] - f1[2]) - (f0[1] - f0[2])) / (f0[1] + f0[2]) < 1e-10
    # and something did happen
    assert abs(f1[0] / f0[0] - 1) > 1e-3


def test_shg_energy_invariant_3d():
    grid = Grid(12, 16, 8, 4 * UM, 4 * UM, 25 * FS)
    fields = _shg_fields()
    prob = oracle.make_problem(grid, fields, D_EFF)
    rng = np.random.default_rng(4)
    init = [_random_smooth(grid, rng, 1e7), _random_smooth(grid, rng, 4e7)]
    out, _ = oracle.propagate(prob, init, 50, 5 * UM, -120.0)
    e0 = sum(f.n * np.sum(np.abs(a) ** 2) for f, a in zip(fields, init))
    e1 = sum(f.n * np.sum(np.abs(a) ** 2) for f, a in zip(fields, out))
    assert abs(e1 / e0 - 1) < 1e-10
    assert np.sum(np.abs(out[0]) ** 2) > 1.1 * np.sum(np.abs(init[0]) ** 2)


def test_split_step_second_order_convergence():
    """Strang splitting (Eq. expon) is second order globally: the error
    against a dz/8 reference falls ~4x per halving of dz."""
    grid = Grid(16, 16, 16, 3 * UM, 3 * UM, 20 * FS)
    fields = _opg_fields()
    prob = oracle.make_problem(grid, fields, D_EFF)
    rng = np.random.default_rng(9)
    init = [_random_smooth(grid, rng, 8e7) for _ in range(3)]
    L = 0.4 * MM
    ref, _ = oracle.propagate(prob, init, 512, L / 512, 2000.0)
    errs = []
    for nz in (8, 16, 32):
        out, _ = oracle.propagate(prob, init, nz, L / nz, 2000.0)
        errs.append(np.sqrt(np.sum(np.abs(out - ref) ** 2)))
    s1 = math.log2(errs[0] / errs[1])
    s2 = math.log2(errs[1] / errs[2])
    assert 1.8 < s1 < 2.2 and 1.8 < s2 < 2.2, (errs, s1, s2)


def test_energy_of_gaussian_matches_closed_form():
    """E = 1/2 c eps0 n  integral |A|^2 (Sec. 6) for A0 exp(-r^2/w^2 - t^2/t0^2)
    is 1/2 c eps0 n A0^2 (pi w^2/2) t0 sqrt(pi/2); photons = E / (hbar omega)."""
    grid = Grid(64, 64, 64, 4 * UM, 4 * UM, 12 * FS)
    w, t0, a0 = 30 * UM, 80 * FS, 3e7
    x, y, t = grid.axes()
    A = a0 * np.exp(-(x[None, None, :] ** 2 + y[None, :, None] ** 2) / w**2 - (t[:, None, None] / t0) ** 2)
    fp = FieldParams(1064e-9, 2.15)
    prob = oracle.make_problem(grid, [fp], D_EFF)
    e, ph = oracle.energy(prob, [A.astype(complex)])
    eps0 = 8.8541878128e-12
    expect = 0.5 * C0 * eps0 * 2.15 * a0**2 * (math.pi * w * w / 2) * t0 * math.sqrt(math.pi / 2)
    assert abs(e[0] / expect - 1) < 1e-12
    assert abs(ph[0] / (expect / (HBAR * 2 * math.pi * C0 / 1064e-9)) - 1) < 1e-12


def test_nonfinite_is_reported():
    fields = _shg_fields()
    prob = oracle.make_problem(PW, fields, D_EFF)
    with pytest.raises(FloatingPointError):
        # absurd step: |Delta A| >> |A| blows up (Sec. 3.2)
        oracle.propagate(prob, [_uniform(PW, 0), _uniform(PW, 1e12)], 40, 1.0, 0.0)


# ------------------------------------------------- transverse mismatch map
def _no_walkoff_shg():
    return [FieldParams(LAM_SH, N_SH, k2=1e-25), FieldParams(LAM_F, N_F, k2=2e-25)]


def test_map_columns_follow_undepleted_sinc():
    """Delta k(x) = dk + m(x) (a fan-out grating): with a uniform weak F and a
    1 m grid spacing (diffraction and walk-off are negligible), every column
    follows its own plane-wave sinc law with its own mismatch."""
    g = Grid(8, 2, 2, 1.0, 1.0, 10 * FS)
    prob = oracle.make_problem(g, _no_walkoff_shg(), D_EFF)
    kSH = 2 * math.pi * D_EFF / (N_SH * LAM_SH)
    a = 1.0 + 0.5j
    L, nz, dk = 3 * MM, 300, 150.0
    m = np.tile(np.linspace(-2000.0, 2000.0, 8), (2, 1))
    out, _ = oracle.propagate_map(prob, [_uniform(g, 0), _uniform(g, a)], nz, L / nz, dk, m)
    for x in range(8):
        d = dk + m[0, x]
        s = math.sin(d * L / 2) / (d * L / 2) if d != 0 else 1.0
        expect = 1j * (kSH / 2) * a * a * L * np.exp(-1j * d * L / 2) * s
        assert abs(out[0, 1, 1, x] - expect) / abs(kSH * a * a * L) < 1e-9


def test_uniform_map_equals_scalar_mismatch():
    """A map that is the same everywhere is the same as adding it to dk."""
    g = Grid(8, 6, 12, 5 * UM, 5 * UM, 30 * FS)
    fields = [FieldParams(1064e-9, 2.15, delta=1e-10, k2=2e-25, rho=2e-3),
              FieldParams(1450e-9, 2.14, k2=1e-25),
              FieldParams(1.0 / (1.0 / 1064e-9 - 1.0 / 1450e-9), 2.08, delta=-1e-10, rho=1e-3)]
    prob = oracle.make_problem(g, fields, D_EFF)
    rng = np.random.default_rng(17)
    init = [3e8 * (rng.standard_normal((12, 6, 8)) + 1j * rng.standard_normal((12, 6, 8))) for _ in range(3)]
    prof = rng.normal(0.0, 300.0, 10)
    ref, phr = oracle.propagate(prob, init, 10, 7 * UM, prof + 450.0)
    got, phg = oracle.propagate_map(prob, init, 10, 7 * UM, prof, np.full((6, 8), 450.0))
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-12
    assert phg == pytest.approx(phr - 450.0 * 10 * 7 * UM, rel=1e-12)


def test_map_split_calls_equal_one_call():
    """z0 carries the distance from the crystal start across calls."""
    g = Grid(8, 4, 8, 5 * UM, 5 * UM, 30 * FS)
    prob = oracle.make_problem(g, _no_walkoff_shg(), D_EFF)
    rng = np.random.default_rng(3)
    init = [1e8 * (rng.standard_normal((8, 4, 8)) + 1j * rng.standard_normal((8, 4, 8))) for _ in range(2)]
    m = rng.normal(0.0, 500.0, (4, 8))
    one, _ = oracle.propagate_map(prob, init, 12, 6 * UM, 80.0, m)
    a, ph = oracle.propagate_map(prob, init, 5, 6 * UM, 80.0, m)
    two, _ = oracle.propagate_map(prob, list(a), 7, 6 * UM, 80.0, m, phi0=ph, z0=5 * 6 * UM)
    assert np.linalg.norm(two - one) / np.linalg.norm(one) < 1e-13


# ------------------------------------------- mismatch map changing along z
def _piecewise_sinc(a, kSH, dks, lengths):
    """Undepleted SHG under a mismatch that is dks[s] over lengths[s]:
    A_SH(L) = i (kSH / 2) a^2 int_0^L e^{-i Phi(z)} dz with Phi the integral
    of the mismatch, summed segment by segment in closed form."""
    acc, phi = 0.0j, 0.0
    for d, ell in zip(dks, lengths):
        seg = ell if d == 0 else (1 - np.exp(-1j * d * ell)) / (1j * d)
        acc += np.exp(-1j * phi) * seg
        phi += d * ell
    return 1j * (kSH / 2) * a * a * acc


def test_map_z_columns_follow_piecewise_closed_form():
    """A fan-out map that changes at two distances: every column follows the
    undepleted plane-wave law of its own piecewise-constant mismatch, with
    the phase continuous at the changes (a phase that restarted, or jumped to
    the new map times z, misses the closed form by O(1))."""
    g = Grid(8, 2, 2, 1.0, 1.0, 10 * FS)
    prob = oracle.make_problem(g, _no_walkoff_shg(), D_EFF)
    kSH = 2 * math.pi * D_EFF / (N_SH * LAM_SH)
    a = 1.0 + 0.5j
    L, nz, dk = 3 * MM, 300, 150.0
    edges = [1.0 * MM, 2.2 * MM]                     # step boundaries 100 and 220
    ramps = [np.linspace(-2000.0, 2000.0, 8), np.linspace(1500.0, -900.0, 8), np.linspace(-300.0, 2500.0, 8)]
    maps = np.stack([np.tile(r, (2, 1)) for r in ramps])
    out, _ = oracle.propagate_map_z(prob, [_uniform(g, 0), _uniform(g, a)], nz, L / nz, dk, edges, maps)
    lengths = [edges[0], edges[1] - edges[0], L - edges[1]]
    for x in range(8):
        expect = _piecewise_sinc(a, kSH, [dk + r[x] for r in ramps], lengths)
        assert abs(out[0, 1, 1, x] - expect) / abs(kSH * a * a * L) < 1e-9, x
    # the phase (dk + map in effect at z) * z, which jumps at each change: far off
    bounds = [0.0, edges[0], edges[1], L]
    for x in range(8):
        jump = sum((np.exp(-1j * d * z0) - np.exp(-1j * d * z1)) / (1j * d)
                   for d, z0, z1 in zip([dk + r[x] for r in ramps], bounds[:-1], bounds[1:]))
        assert abs(out[0, 1, 1, x] - 1j * (kSH / 2) * a * a * jump) / abs(kSH * a * a * L) > 1e-2, x


def test_map_z_uniform_segments_equal_step_profile():
    """Maps uniform in (x, y) on each segment are a per-step mismatch profile:
    step j gets dk_j plus its segment's value (segment of the midpoint)."""
    g = Grid(8, 6, 12, 5 * UM, 5 * UM, 30 * FS)
    fields = [FieldParams(1064e-9, 2.15, delta=1e-10, k2=2e-25, rho=2e-3),
              FieldParams(1450e-9, 2.14, k2=1e-25),
              FieldParams(1.0 / (1.0 / 1064e-9 - 1.0 / 1450e-9), 2.08, delta=-1e-10, rho=1e-3)]
    prob = oracle.make_problem(g, fields, D_EFF)
    rng = np.random.default_rng(23)
    init = [3e8 * (rng.standard_normal((12, 6, 8)) + 1j * rng.standard_normal((12, 6, 8))) for _ in range(3)]
    nz, dz = 14, 7 * UM
    prof = rng.normal(0.0, 300.0, nz)
    edges = [3.2 * dz, 9.6 * dz]                     # midpoints 3.5 dz and 9.5 dz fall on either side
    vals = [450.0, -800.0, 1200.0]
    maps = np.stack([np.full((6, 8), v) for v in vals])
    seg = np.searchsorted(edges, (np.arange(nz) + 0.5) * dz, side="right")
    assert list(np.bincount(seg)) == [3, 7, 4]
    ref, phr = oracle.propagate(prob, init, nz, dz, prof + np.take(vals, seg))
    got, phg = oracle.propagate_map_z(prob, init, nz, dz, prof, edges, maps)
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-12
    assert phg == pytest.approx(phr - float(np.sum(np.take(vals, seg))) * dz, rel=1e-12)


def test_map_z_one_segment_equals_static_map():
    """One segment, or several segments holding the same map, is the static
    map of propagate_map (per-point indexing of the accumulated phase)."""
    g = Grid(8, 4, 8, 5 * UM, 5 * UM, 30 * FS)
    prob = oracle.make_problem(g, _no_walkoff_shg(), D_EFF)
    rng = np.random.default_rng(29)
    init = [1e8 * (rng.standard_normal((8, 4, 8)) + 1j * rng.standard_normal((8, 4, 8))) for _ in range(2)]
    m = rng.normal(0.0, 500.0, (4, 8))
    ref, _ = oracle.propagate_map(prob, init, 12, 6 * UM, 80.0, m)
    one, _ = oracle.propagate_map_z(prob, init, 12, 6 * UM, 80.0, [], m[None])
    three, _ = oracle.propagate_map_z(prob, init, 12, 6 * UM, 80.0, [20 * UM, 41 * UM], np.stack([m, m, m]))
    assert np.linalg.norm(one - ref) / np.linalg.norm(ref) < 1e-13
    assert np.linalg.norm(three - ref) / np.linalg.norm(ref) < 1e-13
