"""Pins for the oracle's discrete adjoint: dot-product identities and
central finite differences of the forward objective."""
import math

import numpy as np
import pytest

import oracle
from paper_2609_08384_gb300 import workloads as wl

UM, MM, FS = 1e-6, 1e-3, 1e-15


def _fields3():
    lp, ls = 1064e-9, 1450e-9
    li = 1.0 / (1.0 / lp - 1.0 / ls)
    return [wl.FieldParams(lp, 2.15, delta=1e-10, k2=2e-25, rho=2e-3, alpha=20.0),
            wl.FieldParams(ls, 2.14, k2=1e-25, k3=3e-40),
            wl.FieldParams(li, 2.08, delta=-1e-10, k2=5e-26, rho=1e-3)]


def _rdot(a, b):
    return float(np.real(np.vdot(a, b)))


def test_linear_adjoint_dot_product():
    g = wl.Grid(12, 8, 16, 3 * UM, 3 * UM, 20 * FS)
    prob = oracle.make_problem(g, _fields3(), wl.D_EFF)
    rng = np.random.default_rng(1)
    shp = (3, 16, 8, 12)
    v = rng.standard_normal(shp) + 1j * rng.standard_normal(shp)
    w = rng.standard_normal(shp) + 1j * rng.standard_normal(shp)
    Lv = oracle.linear_step(prob, list(v), 0.3 * MM)
    Lhw = oracle.linear_step_adjoint(prob, list(w), 0.3 * MM)
    lhs, rhs = np.vdot(Lv, w), np.vdot(v, Lhw)
    assert abs(lhs - rhs) / abs(lhs) < 1e-12


@pytest.mark.parametrize("nf", [2, 3])
def test_rk4_adjoint_dot_product_and_stage_sensitivities(nf):
    fields = _fields3() if nf == 3 else wl.shg_fields()
    prob = oracle.make_problem(wl.Grid(2, 2, 2, UM, UM, FS), fields, wl.D_EFF)
    rng = np.random.default_rng(nf)
    h, phi_a, dk = 40 * UM, 0.7, 900.0
    for _ in range(5):
        x = (rng.standard_normal(nf) + 1j * rng.standard_normal(nf)) * 3e7
        dx = rng.standard_normal(nf) + 1j * rng.standard_normal(nf)
        gy = rng.standard_normal(nf) + 1j * rng.standard_normal(nf)
        _, dy = oracle.rk4_jvp_point(prob, phi_a, dk, h, x, dx)
        gx, sens = oracle.rk4_vjp_point(prob, phi_a, dk, h, x, gy)
        lhs, rhs = _rdot(dy, gy), _rdot(dx, gx)
        assert abs(lhs - rhs) <= 1e-12 * (abs(lhs) + abs(rhs)), (lhs, rhs)
        # J(y) = Re <gy, y>: shifting phi_a moves every stage phase, dk moves
        # the middle and end stages by h/2 and h
        def J(pa, d):
            y, _ = oracle.rk4_jvp_point(prob, pa, d, h, x, np.zeros(nf))
            return _rdot(gy, y)
        e = 1e-5
        dJ_dphi = (J(phi_a + e, dk) - J(phi_a - e, dk)) / (2 * e)
        assert abs(dJ_dphi - sens.sum()) <= 1e-7 * max(abs(dJ_dphi), 1e-30) + 1e-12 * np.abs(x).max()
        ed = 1.0
        dJ_ddk = (J(phi_a, dk + ed) - J(phi_a, dk - ed)) / (2 * ed)
        assert abs(dJ_ddk - (0.5 * h * sens[1] + h * sens[2])) <= 1e-6 * abs(dJ_ddk) + 1e-15


def _small_shg():
    g = wl.Grid(16, 16, 32, 10 * UM, 10 * UM, 40 * FS)
    f = wl.shg_fields()
    a0 = wl.peak_amplitude(5e13, wl.N_F)
    F = wl.focused_pulse(g, f[1], a0, 35 * UM, 200 * FS, 1 * MM)
    return g, f, [np.zeros_like(F), F]


def test_full_gradient_matches_central_differences():
    """eta = E_SH(L)/E_F(0) on 16x16x32, 40 steps: gradient with respect to
    every spectral-phase entry (32) and every per-step mismatch (40) against
    central differences with h = 1e-3 and 1e-4 (phase) and 1e-3 mm^-1
    (mismatch)."""
    g, f, ins = _small_shg()
    prob = oracle.make_problem(g, f, wl.D_EFF)
    rng = np.random.default_rng(wl.SEED_BASE + 40)
    nz, dz = 40, 25 * UM
    phi = rng.normal(0, 0.1, g.nt)
    dk = 0.0 + rng.normal(0, 0.1, nz) / MM
    wF = np.sum(np.abs(ins[1]) ** 2)
    w = np.array([f[0].n / (f[1].n * wF), 0.0])
    J, gphi, gdk = oracle.adjoint_gradient(prob, ins, nz, dz, dk, w, phi=phi, phi_field=1)
    assert 0.01 < J < 0.9  # real conversion, not a trivial point
    def fd_phi_at(h):
        out = np.zeros(g.nt)
        for p in range(g.nt):
            e = np.zeros(g.nt)
            e[p] = h
            out[p] = (oracle.objective(prob, ins, nz, dz, dk, w, phi + e) -
                      oracle.objective(prob, ins, nz, dz, dk, w, phi - e)) / (2 * h)
        return out

    fd_phi = fd_phi_at(1e-3)
    fd_phi_fine = fd_phi_at(1e-4)
    hk = 1e-3 / MM
    fd_dk = np.zeros(nz)
    for j in range(nz):
        e = np.zeros(nz)
        e[j] = hk
        fd_dk[j] = (oracle.objective(prob, ins, nz, dz, dk + e, w, phi) -
                    oracle.objective(prob, ins, nz, dz, dk - e, w, phi)) / (2 * hk)
    # central differences carry an O(h^2) error: ~2e-6 at h = 1e-3 on this
    # strongly converting case, falling ~100x at h = 1e-4
    e_coarse = np.linalg.norm(gphi - fd_phi) / np.linalg.norm(fd_phi)
    e_fine = np.linalg.norm(gphi - fd_phi_fine) / np.linalg.norm(fd_phi_fine)
    assert e_coarse < 1e-5 and e_fine < 1e-6 and e_fine < 0.1 * e_coarse, (e_coarse, e_fine)
    assert np.linalg.norm(gdk - fd_dk) / np.linalg.norm(fd_dk) < 1e-6


def test_three_field_gradient_dk_matches_differences():
    g = wl.Grid(8, 8, 16, 6 * UM, 6 * UM, 30 * FS)
    f = _fields3()
    prob = oracle.make_problem(g, f, wl.D_EFF)
    rng = np.random.default_rng(44)
    x, y, t = g.axes()
    env = np.exp(-(x[None, None] ** 2 + y[None, :, None] ** 2) / (15 * UM) ** 2 - (t[:, None, None] / (120 * FS)) ** 2)
    ins = [8e7 * env + 0j, 2e7 * env * np.exp(0.3j), 1e6 * (rng.standard_normal(env.shape) + 0j)]
    nz, dz = 12, 30 * UM
    dk = rng.normal(300.0, 200.0, nz)
    w = np.array([0.0, 1.0, 0.5])
    phi = rng.normal(0, 0.2, g.nt)
    J, gphi, gdk = oracle.adjoint_gradient(prob, ins, nz, dz, dk, w, phi=phi, phi_field=0)
    hk = 1.0
    for j in (0, 5, 11):
        e = np.zeros(nz)
        e[j] = hk
        fd = (oracle.objective(prob, ins, nz, dz, dk + e, w, phi, 0) -
              oracle.objective(prob, ins, nz, dz, dk - e, w, phi, 0)) / (2 * hk)
        assert abs(gdk[j] - fd) <= 1e-6 * abs(fd) + 1e-9 * abs(J), (j, gdk[j], fd)
    for p in (0, 7, 15):
        e = np.zeros(g.nt)
        e[p] = 1e-3
        fd = (oracle.objective(prob, ins, nz, dz, dk, w, phi + e, 0) -
              oracle.objective(prob, ins, nz, dz, dk, w, phi - e, 0)) / 2e-3
        assert abs(gphi[p] - fd) <= 1e-6 * abs(fd) + 1e-9 * abs(J), (p, gphi[p], fd)


@pytest.mark.parametrize("three", [False, True])
def test_gradient_under_mismatch_map_matches_differences(three):
    """A transverse mismatch map (fan-out ramp plus a bump) changes every
    point's stage phases; the adjoint under the map matches central
    differences of the map objective for the per-step mismatch and the
    spectral phase, and differs clearly from the map-free gradient."""
    rng = np.random.default_rng(47 + three)
    if three:
        g = wl.Grid(8, 8, 16, 6 * UM, 6 * UM, 30 * FS)
        f = _fields3()
        x, y, t = g.axes()
        env = np.exp(-(x[None, None] ** 2 + y[None, :, None] ** 2) / (15 * UM) ** 2 - (t[:, None, None] / (120 * FS)) ** 2)
        ins = [8e7 * env + 0j, 2e7 * env * np.exp(0.3j), 1e6 * (rng.standard_normal(env.shape) + 0j)]
        nz, dz, w, pf = 12, 30 * UM, np.array([0.0, 1.0, 0.5]), 0
        dk = rng.normal(300.0, 200.0, nz)
    else:
        g, f, ins = _small_shg()
        x, y, _ = g.axes()
        nz, dz, pf = 16, 40 * UM, 1
        wF = np.sum(np.abs(ins[1]) ** 2)
        w = np.array([f[0].n / (f[1].n * wF), 0.0])
        dk = rng.normal(0, 0.1, nz) / MM
    prob = oracle.make_problem(g, f, wl.D_EFF)
    m = 4e6 * x[None, :] + 3e3 * np.exp(-(x[None, :] ** 2 + y[:, None] ** 2) / (12 * UM) ** 2) + 0 * y[:, None]
    phi = rng.normal(0, 0.2, g.nt)
    J, gphi, gdk = oracle.adjoint_gradient(prob, ins, nz, dz, dk, w, phi=phi, phi_field=pf, dk_map=m)
    assert J == pytest.approx(oracle.objective(prob, ins, nz, dz, dk, w, phi, pf, dk_map=m), rel=1e-14)
    hk = 1.0
    for j in (0, nz // 2, nz - 1):
        e = np.zeros(nz)
        e[j] = hk
        fd = (oracle.objective(prob, ins, nz, dz, dk + e, w, phi, pf, dk_map=m) -
              oracle.objective(prob, ins, nz, dz, dk - e, w, phi, pf, dk_map=m)) / (2 * hk)
        assert abs(gdk[j] - fd) <= 1e-6 * abs(fd) + 1e-9 * abs(J), (j, gdk[j], fd)
    for p in (0, g.nt // 2 - 1, g.nt - 1):
        e = np.zeros(g.nt)
        e[p] = 1e-3
        fd = (oracle.objective(prob, ins, nz, dz, dk, w, phi + e, pf, dk_map=m) -
              oracle.objective(prob, ins, nz, dz, dk, w, phi - e, pf, dk_map=m)) / 2e-3
        assert abs(gphi[p] - fd) <= 1e-6 * abs(fd) + 1e-9 * abs(J), (p, gphi[p], fd)
    _, gphi0, gdk0 = oracle.adjoint_gradient(prob, ins, nz, dz, dk, w, phi=phi, phi_field=pf)
    assert np.linalg.norm(gdk - gdk0) > 0.1 * np.linalg.norm(gdk)


@pytest.mark.parametrize("three", [False, True])
def test_gradient_under_map_changing_along_z(three):
    """A map that changes along z (three segments).  Pins: maps uniform on
    each segment give the gradient of the per-step profile with each step's
    segment value added (1e-12); three segments holding one map give the
    static-map gradient (1e-12); with three different maps the gradient
    matches central differences of the z-resolved objective."""
    rng = np.random.default_rng(53 + three)
    if three:
        g = wl.Grid(8, 8, 16, 6 * UM, 6 * UM, 30 * FS)
        f = _fields3()
        x, y, t = g.axes()
        env = np.exp(-(x[None, None] ** 2 + y[None, :, None] ** 2) / (15 * UM) ** 2 - (t[:, None, None] / (120 * FS)) ** 2)
        ins = [8e7 * env + 0j, 2e7 * env * np.exp(0.3j), 1e6 * (rng.standard_normal(env.shape) + 0j)]
        nz, dz, w, pf = 12, 30 * UM, np.array([0.0, 1.0, 0.5]), 0
        dk = rng.normal(300.0, 200.0, nz)
    else:
        g, f, ins = _small_shg()
        x, y, _ = g.axes()
        nz, dz, pf = 16, 40 * UM, 1
        wF = np.sum(np.abs(ins[1]) ** 2)
        w = np.array([f[0].n / (f[1].n * wF), 0.0])
        dk = rng.normal(0, 0.1, nz) / MM
    prob = oracle.make_problem(g, f, wl.D_EFF)
    edges = [3.3 * dz, 8.6 * dz]
    seg = np.searchsorted(edges, (np.arange(nz) + 0.5) * dz, side="right")
    phi = rng.normal(0, 0.2, g.nt)
    # uniform segments == step profile
    vals = np.array([900.0, -1500.0, 600.0])
    uni = np.stack([np.full((g.ny, g.nx), v) for v in vals])
    Ju, gphu, gdku = oracle.adjoint_gradient(prob, ins, nz, dz, dk, w, phi=phi, phi_field=pf, z_edges=edges, maps=uni)
    Jp, gphp, gdkp = oracle.adjoint_gradient(prob, ins, nz, dz, dk + vals[seg], w, phi=phi, phi_field=pf)
    assert Ju == pytest.approx(Jp, rel=1e-12)
    assert np.linalg.norm(gdku - gdkp) <= 1e-12 * np.linalg.norm(gdkp)
    assert np.linalg.norm(gphu - gphp) <= 1e-12 * np.linalg.norm(gphp)
    # one map on every segment == the static map
    m = 4e6 * x[None, :] + 3e3 * np.exp(-(x[None, :] ** 2 + y[:, None] ** 2) / (12 * UM) ** 2) + 0 * y[:, None]
    Js, gphs, gdks = oracle.adjoint_gradient(prob, ins, nz, dz, dk, w, phi=phi, phi_field=pf, dk_map=m)
    J3, gph3, gdk3 = oracle.adjoint_gradient(prob, ins, nz, dz, dk, w, phi=phi, phi_field=pf, z_edges=edges,
                                             maps=np.stack([m, m, m]))
    assert J3 == pytest.approx(Js, rel=1e-12)
    assert np.linalg.norm(gdk3 - gdks) <= 1e-12 * np.linalg.norm(gdks)
    assert np.linalg.norm(gph3 - gphs) <= 1e-12 * np.linalg.norm(gphs)
    # three different maps against central differences
    maps = np.stack([m, 2000.0 - 0.7 * m, 0.5 * m - 800.0])
    J, gphi, gdk = oracle.adjoint_gradient(prob, ins, nz, dz, dk, w, phi=phi, phi_field=pf, z_edges=edges, maps=maps)
    assert J == pytest.approx(oracle.objective(prob, ins, nz, dz, dk, w, phi, pf, z_edges=edges, maps=maps), rel=1e-14)
    hk = 1.0
    for j in (0, 3, 4, nz - 1):  # around the first edge and at the ends
        e = np.zeros(nz)
        e[j] = hk
        fd = (oracle.objective(prob, ins, nz, dz, dk + e, w, phi, pf, z_edges=edges, maps=maps) -
              oracle.objective(prob, ins, nz, dz, dk - e, w, phi, pf, z_edges=edges, maps=maps)) / (2 * hk)
        assert abs(gdk[j] - fd) <= 1e-6 * abs(fd) + 1e-9 * abs(J), (j, gdk[j], fd)
    def fd_phi(p, h):
        e = np.zeros(g.nt)
        e[p] = h
        return (oracle.objective(prob, ins, nz, dz, dk, w, phi + e, pf, z_edges=edges, maps=maps) -
                oracle.objective(prob, ins, nz, dz, dk, w, phi - e, pf, z_edges=edges, maps=maps)) / (2 * h)

    for p in (0, g.nt // 2, g.nt - 1):  # the zero-frequency bin has the largest curvature: Richardson over h, h/2
        fd = (4 * fd_phi(p, 5e-4) - fd_phi(p, 1e-3)) / 3
        assert abs(gphi[p] - fd) <= 1e-6 * abs(fd) + 1e-9 * abs(J), (p, gphi[p], fd)
    assert np.linalg.norm(gdk - gdks) > 0.05 * np.linalg.norm(gdk)


def _centred_omega(nt, dt):
    """Omega_p = 2 pi (p - NT/2) / (NT dt): the centred order of the spectral-phase vector."""
    return 2 * np.pi * (np.arange(nt) - nt // 2) / (nt * dt)


@pytest.mark.parametrize("nt,shift", [(64, 5), (64, -7), (48, 11), (48, -1), (256, 100)])
@pytest.mark.parametrize("sign", [+1, -1])
def test_spectral_phase_linear_phase_is_an_exact_circular_shift(nt, shift, sign):
    """A linear spectral phase phi(Omega) = Omega m dt multiplies each DFT bin
    by e^{+2 pi i k m / NT}; the inverse transform then returns the pulse
    advanced by exactly m samples: out[t] = in[(t + m) mod NT] (sign -1 delays
    it).  Fixes the sign of phi, the centred index of each bin (an off-by-one
    turns the shift into a shift times a constant phase and breaks the Nyquist
    bin) and the 1/NT of the inverse."""
    dt = 7 * FS
    g = wl.Grid(4, 3, nt, UM, UM, dt)
    prob = oracle.make_problem(g, wl.shg_fields(), wl.D_EFF)
    rng = np.random.default_rng(abs(1000 * nt + 31 * shift) + (sign > 0))
    a = rng.standard_normal((nt, 3, 4)) + 1j * rng.standard_normal((nt, 3, 4))
    phi = _centred_omega(nt, dt) * shift * dt
    out = oracle.spectral_phase(prob, a, phi, sign)
    want = np.roll(a, -sign * shift, axis=0)
    assert np.abs(out - want).max() < 1e-13 * np.abs(a).max()


@pytest.mark.parametrize("beta_over_tau2", [0.7, -1.3])
def test_spectral_phase_quadratic_phase_gives_the_chirped_gaussian(beta_over_tau2):
    """phi(Omega) = beta Omega^2 / 2 on A = exp(-tau^2/tau0^2).  With the
    forward transform e^{-i Omega tau}, A~(Omega) = sqrt(pi) tau0
    exp(-Omega^2 tau0^2 / 4); times e^{i beta Omega^2/2} and transformed back,
    A'(tau) = tau0 / sqrt(tau0^2 - 2 i beta) exp(-tau^2 / (tau0^2 - 2 i beta))
    (principal root).  The window holds the chirped pulse to e^{-50} and the
    spectrum to e^{-300}, so the discrete result equals the closed form to
    rounding.  The sign of beta's imaginary part pins the sign of phi."""
    nt, dt = 512, 2 * FS
    tau0 = 12 * dt
    beta = beta_over_tau2 * tau0**2
    g = wl.Grid(2, 2, nt, UM, UM, dt)
    prob = oracle.make_problem(g, wl.shg_fields(), wl.D_EFF)
    tau = (np.arange(nt) - nt // 2) * dt
    a = np.broadcast_to(np.exp(-(tau / tau0) ** 2)[:, None, None], (nt, 2, 2)).astype(np.complex128)
    phi = beta * _centred_omega(nt, dt) ** 2 / 2
    out = oracle.spectral_phase(prob, a, phi, +1)
    q = tau0**2 - 2j * beta
    want = tau0 / np.sqrt(q) * np.exp(-tau**2 / q)
    assert np.abs(out[:, 1, 0] - want).max() < 1e-9
    # the conjugate chirp (sign -1) is the closed form with beta -> -beta
    back = oracle.spectral_phase(prob, a, phi, -1)
    qm = tau0**2 + 2j * beta
    assert np.abs(back[:, 0, 1] - tau0 / np.sqrt(qm) * np.exp(-tau**2 / qm)).max() < 1e-9
