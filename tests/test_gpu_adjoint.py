"""GPU adjoint (checkpointed reverse sweep) against the FP64 oracle gradient,
finite differences of the GPU forward, and through torch.autograd."""
import numpy as np
import pytest

import oracle
from paper_2609_08384_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GRAD_TOL = 1e-3  # relative L2 over the whole gradient vector


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2609_08384_gb300 import build
    build.build()


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def _shg_case(n, nt, nz, dz, seed, intensity=3e13):
    g = wl.Grid(n, n, nt, 12.5 * wl.UM, 12.5 * wl.UM, 50 * wl.FS)
    f = wl.shg_fields()
    a0 = wl.peak_amplitude(intensity, wl.N_F)
    F = wl.focused_pulse(g, f[1], a0, 4 * n / 32 * 25 * wl.UM, 8 * nt / 64 * 50 * wl.FS, nz * dz)
    ins = [np.zeros_like(F).astype(np.complex64), F.astype(np.complex64)]
    rng = np.random.default_rng(wl.SEED_BASE + seed)
    phi = rng.normal(0, 0.1, nt)
    dk = rng.normal(0, 0.1, nz) / wl.MM
    return g, f, ins, phi, dk


def _gpu_grad(g, f, ins, phi, dk, nz, dz, w, interval=0, phi_field=1, dk_map=None, z_edges=None, maps=None):
    import paper_2609_08384_gb300 as br
    s = br.Solver(g, f, wl.D_EFF, 0.0)
    if dk_map is not None:
        s.set_dk_map(dk_map)
    if maps is not None:
        s.set_dk_map_z(z_edges, maps)
    J = s.adjoint_forward([torch.from_numpy(a).cuda() for a in ins], dk, nz, dz, w, phi=phi, phi_field=phi_field,
                          checkpoint_interval=interval)
    gphi, gdk = s.adjoint_backward(1.0)
    s.close()
    return J, gphi, gdk


@pytest.mark.parametrize("n,nt,nz", [(32, 64, 60), (64, 128, 24)])
def test_shg_gradient_matches_oracle(n, nt, nz):
    dz = 5 * wl.UM * (400 / nz) * 0.25
    g, f, ins, phi, dk = _shg_case(n, nt, nz, dz, 50 + n)
    w = np.array([f[0].n / (f[1].n * float(np.sum(np.abs(ins[1].astype(np.complex128)) ** 2))), 0.0])
    J, gphi, gdk = _gpu_grad(g, f, ins, phi, dk, nz, dz, w)
    prob = oracle.make_problem(g, f, wl.D_EFF)
    Jr, gphi_r, gdk_r = oracle.adjoint_gradient(prob, [a.astype(np.complex128) for a in ins], nz, dz, dk, w,
                                                phi=phi, phi_field=1)
    assert Jr > 1e-3
    assert abs(J / Jr - 1) < 1e-4
    assert rel_l2(gphi, gphi_r) < GRAD_TOL
    assert rel_l2(gdk, gdk_r) < GRAD_TOL


def test_three_field_gradient_matches_oracle():
    g = wl.Grid(24, 16, 32, 6 * wl.UM, 6 * wl.UM, 30 * wl.FS)
    fields = [wl.FieldParams(wl.LAM_P, wl.N_P, delta=1e-10, k2=2e-25, rho=2e-3),
              wl.FieldParams(wl.LAM_S, wl.N_S, k2=1e-25),
              wl.FieldParams(wl.LAM_I, wl.N_I, delta=-1e-10, k2=5e-26, rho=1e-3, alpha=20.0)]
    x, y, t = g.axes()
    env = np.exp(-(x[None, None] ** 2 + y[None, :, None] ** 2) / (25 * wl.UM) ** 2 - (t[:, None, None] / (150 * wl.FS)) ** 2)
    rng = np.random.default_rng(7)
    ins = [(8e7 * env).astype(np.complex64), (2e7 * env * np.exp(0.3j)).astype(np.complex64),
           (1e6 * rng.standard_normal(env.shape)).astype(np.complex64)]
    nz, dz = 16, 25 * wl.UM
    dk = rng.normal(300.0, 200.0, nz)
    phi = rng.normal(0, 0.2, g.nt)
    w = np.array([0.0, 1e-15, 5e-16])
    J, gphi, gdk = _gpu_grad(g, fields, ins, phi, dk, nz, dz, w, phi_field=0)
    prob = oracle.make_problem(g, fields, wl.D_EFF)
    Jr, gphi_r, gdk_r = oracle.adjoint_gradient(prob, [a.astype(np.complex128) for a in ins], nz, dz, dk, w,
                                                phi=phi, phi_field=0)
    assert abs(J / Jr - 1) < 1e-4
    assert rel_l2(gphi, gphi_r) < GRAD_TOL
    assert rel_l2(gdk, gdk_r) < GRAD_TOL


def test_checkpoint_interval_does_not_change_the_gradient():
    nz, dz = 30, 20 * wl.UM
    g, f, ins, phi, dk = _shg_case(32, 64, nz, dz, 60)
    w = np.array([1e-20, 0.0])
    res = [_gpu_grad(g, f, ins, phi, dk, nz, dz, w, interval=k) for k in (0, 7, nz, 1)]
    for J, gp, gd in res[1:]:
        assert J == res[0][0]
        assert np.array_equal(gp, res[0][1]) and np.array_equal(gd, res[0][2])


def test_adjoint_gradient_full_size_directional_derivative():
    """SHG efficiency on 128x128x256 over 400 steps of 5 um, with respect to
    the 256-entry spectral phase and the 400-entry mismatch profile: the
    adjoint's directional derivative along the gradient matches a central
    difference of the GPU forward."""
    import paper_2609_08384_gb300 as br
    p = wl.problem_adjoint()
    f = p.fields
    a0 = wl.peak_amplitude(1e13, wl.N_F)
    F = wl.focused_pulse(p.grid, f[1], a0, 50 * wl.UM, 200 * wl.FS, p.length).astype(np.complex64)
    ins = [np.zeros_like(F), F]
    phi, dk = p.spectral_phase, p.dk_profile
    s = br.Solver(p.grid, f, p.d_eff, 0.0)
    dev = [torch.from_numpy(a).cuda() for a in ins]
    w = s.shg_efficiency_weights(dev)
    # the library's weights are those of the definition eta = E_SH(L)/E_F(0)
    # (its sum takes FP32 squares of the complex64 field into FP64: ~1e-9)
    w_def = f[0].n / (f[1].n * float(np.sum(np.abs(F.astype(np.complex128)) ** 2)))
    assert abs(w[0] / w_def - 1) < 1e-7 and w[1] == 0.0
    J = s.adjoint_forward(dev, dk, p.nz, p.dz, w, phi=phi)
    gphi, gdk = s.adjoint_backward(1.0)
    assert 0.01 < J < 1.0
    # scale mismatch steps to the unit of the draw (1/mm) so both blocks count
    d_phi, d_dk = gphi, gdk * (1.0 / wl.MM)
    norm = np.sqrt(np.sum(d_phi ** 2) + np.sum(d_dk ** 2))
    d_phi, d_dk = d_phi / norm, d_dk / norm
    slope = float(np.dot(gphi, d_phi) + np.dot(gdk, d_dk * (1.0 / wl.MM)))
    def cd(eps):
        Jp = s.adjoint_forward(dev, dk + eps * d_dk / wl.MM, p.nz, p.dz, w, phi=phi + eps * d_phi)
        Jm = s.adjoint_forward(dev, dk - eps * d_dk / wl.MM, p.nz, p.dz, w, phi=phi - eps * d_phi)
        return (Jp - Jm) / (2 * eps)

    # steps that move eta by ~0.8% and ~0.4%; Richardson removes the O(eps^2) term
    eps = 0.008 * J / slope
    f1, f2 = cd(eps), cd(0.5 * eps)
    rich = (4 * f2 - f1) / 3
    s.close()
    assert abs(rich / slope - 1) < GRAD_TOL, (f1, f2, rich, slope)


def test_autograd_function():
    import paper_2609_08384_gb300 as br
    nz, dz = 20, 20 * wl.UM
    g, f, ins, phi, dk = _shg_case(32, 64, nz, dz, 70)
    s = br.Solver(g, f, wl.D_EFF, 0.0)
    dev = [torch.from_numpy(a).cuda() for a in ins]
    w = s.shg_efficiency_weights(dev)
    Eta = br.shg_efficiency_function()
    tphi = torch.tensor(phi, dtype=torch.float64, requires_grad=True)
    tdk = torch.tensor(dk, dtype=torch.float64, requires_grad=True)
    eta = Eta.apply(tphi, tdk, s, dev, nz, dz, w, 0)
    eta.backward()
    J, gphi, gdk = _gpu_grad(g, f, ins, phi, dk, nz, dz, w)
    assert float(eta.detach()) == J
    assert np.array_equal(tphi.grad.numpy(), gphi) and np.array_equal(tdk.grad.numpy(), gdk)
    # the incoming gradient scales the result (FP32 rounding of the scaled adjoint aside)
    tphi.grad = None
    tdk.grad = None
    (3.0 * Eta.apply(tphi, tdk, s, dev, nz, dz, w, 0)).backward()
    assert rel_l2(tphi.grad.numpy(), 3.0 * gphi) < 1e-4 and rel_l2(tdk.grad.numpy(), 3.0 * gdk) < 1e-4
    s.close()


def test_field_streams_do_not_change_the_gradient():
    """The adjoint's linear passes on per-field streams give the same bits."""
    import paper_2609_08384_gb300 as br
    nz, dz = 20, 20 * wl.UM
    g, f, ins, phi, dk = _shg_case(32, 64, nz, dz, 61)
    w = np.array([1e-20, 3e-21])
    out = []
    for split in (0, 1):
        s = br.Solver(g, f, wl.D_EFF, 0.0)
        s.set_option(br.BRAHMS_OPT_FIELD_STREAMS, split)
        J = s.adjoint_forward([torch.from_numpy(a).cuda() for a in ins], dk, nz, dz, w, phi=phi, checkpoint_interval=6)
        out.append((J,) + tuple(s.adjoint_backward(1.0)))
        s.close()
    assert out[0][0] == out[1][0]
    assert np.array_equal(out[0][1], out[1][1]) and np.array_equal(out[0][2], out[1][2])


def _fanout_map(g, slope=4e6, bump=3e3, width=30 * wl.UM):
    x, y, _ = g.axes()
    return slope * x[None, :] + bump * np.exp(-(x[None, :] ** 2 + y[:, None] ** 2) / width**2)


@pytest.mark.parametrize("three", [False, True])
def test_gradient_under_mismatch_map_matches_oracle(three):
    """A fan-out map plus a bump: the recomputation, the recording x-pass and
    the reverse x-pass take per-point stage phases; gradients against the
    oracle's adjoint under the same map."""
    if three:
        g = wl.Grid(24, 16, 32, 6 * wl.UM, 6 * wl.UM, 30 * wl.FS)
        f = [wl.FieldParams(wl.LAM_P, wl.N_P, delta=1e-10, k2=2e-25, rho=2e-3),
             wl.FieldParams(wl.LAM_S, wl.N_S, k2=1e-25),
             wl.FieldParams(wl.LAM_I, wl.N_I, delta=-1e-10, k2=5e-26, rho=1e-3, alpha=20.0)]
        x, y, t = g.axes()
        env = np.exp(-(x[None, None] ** 2 + y[None, :, None] ** 2) / (25 * wl.UM) ** 2 - (t[:, None, None] / (150 * wl.FS)) ** 2)
        rng = np.random.default_rng(9)
        ins = [(8e7 * env).astype(np.complex64), (2e7 * env * np.exp(0.3j)).astype(np.complex64),
               (1e6 * rng.standard_normal(env.shape)).astype(np.complex64)]
        nz, dz, pf = 16, 25 * wl.UM, 0
        dk = rng.normal(300.0, 200.0, nz)
        phi = rng.normal(0, 0.2, g.nt)
        w = np.array([0.0, 1e-15, 5e-16])
        m = _fanout_map(g, slope=2e7, bump=2e4, width=15 * wl.UM)
    else:
        nz = 60
        dz = 5 * wl.UM * (400 / nz) * 0.25
        g, f, ins, phi, dk = _shg_case(32, 64, nz, dz, 83)
        w = np.array([f[0].n / (f[1].n * float(np.sum(np.abs(ins[1].astype(np.complex128)) ** 2))), 0.0])
        pf = 1
        m = _fanout_map(g)
    J, gphi, gdk = _gpu_grad(g, f, ins, phi, dk, nz, dz, w, phi_field=pf, dk_map=m)
    prob = oracle.make_problem(g, f, wl.D_EFF)
    ins128 = [a.astype(np.complex128) for a in ins]
    Jr, gphi_r, gdk_r = oracle.adjoint_gradient(prob, ins128, nz, dz, dk, w, phi=phi, phi_field=pf, dk_map=m)
    assert abs(J / Jr - 1) < 1e-4
    assert rel_l2(gphi, gphi_r) < GRAD_TOL
    assert rel_l2(gdk, gdk_r) < GRAD_TOL
    # the map is felt: the map-free oracle gradient is far off
    _, _, gdk0 = oracle.adjoint_gradient(prob, ins128, nz, dz, dk, w, phi=phi, phi_field=pf)
    assert rel_l2(gdk0, gdk_r) > 20 * GRAD_TOL


def test_checkpoint_interval_does_not_change_the_gradient_under_a_map():
    nz, dz = 30, 20 * wl.UM
    g, f, ins, phi, dk = _shg_case(32, 64, nz, dz, 61)
    w = np.array([1e-20, 0.0])
    m = _fanout_map(g)
    res = [_gpu_grad(g, f, ins, phi, dk, nz, dz, w, interval=k, dk_map=m) for k in (0, 7, 1)]
    for J, gp, gd in res[1:]:
        assert J == res[0][0]
        assert np.array_equal(gp, res[0][1]) and np.array_equal(gd, res[0][2])


@pytest.mark.parametrize("with_map", [False, True])
def test_store_all_forward_gives_the_same_gradient(with_map):
    """checkpoint_interval < 0: the forward records every step and the backward
    recomputes nothing; J and both gradients are bit-identical to the
    checkpointed run."""
    nz, dz = 30, 20 * wl.UM
    g, f, ins, phi, dk = _shg_case(32, 64, nz, dz, 62)
    w = np.array([1e-20, 0.0])
    m = _fanout_map(g) if with_map else None
    ref = _gpu_grad(g, f, ins, phi, dk, nz, dz, w, interval=0, dk_map=m)
    got = _gpu_grad(g, f, ins, phi, dk, nz, dz, w, interval=-1, dk_map=m)
    assert got[0] == ref[0]
    assert np.array_equal(got[1], ref[1]) and np.array_equal(got[2], ref[2])


@pytest.mark.parametrize("three", [False, True])
def test_gradient_under_map_changing_along_z_matches_oracle(three):
    """Three z-segments with different maps: the adjoint's recomputation and
    reverse sweep form each step's map phase from the segments' step counts;
    the gradient matches the oracle's z-resolved gradient with the default
    checkpoints, an interval of 7 steps and every step recorded."""
    if three:
        g = wl.Grid(24, 16, 32, 6 * wl.UM, 6 * wl.UM, 30 * wl.FS)
        f = [wl.FieldParams(wl.LAM_P, wl.N_P, delta=1e-10, k2=2e-25, rho=2e-3),
             wl.FieldParams(wl.LAM_S, wl.N_S, k2=1e-25),
             wl.FieldParams(wl.LAM_I, wl.N_I, delta=-1e-10, k2=5e-26, rho=1e-3, alpha=20.0)]
        x, y, t = g.axes()
        env = np.exp(-(x[None, None] ** 2 + y[None, :, None] ** 2) / (25 * wl.UM) ** 2 - (t[:, None, None] / (150 * wl.FS)) ** 2)
        rng = np.random.default_rng(19)
        ins = [(8e7 * env).astype(np.complex64), (2e7 * env * np.exp(0.3j)).astype(np.complex64),
               (1e6 * rng.standard_normal(env.shape)).astype(np.complex64)]
        nz, dz, pf = 16, 25 * wl.UM, 0
        dk = rng.normal(300.0, 200.0, nz)
        phi = rng.normal(0, 0.2, g.nt)
        w = np.array([0.0, 1e-15, 5e-16])
        m = _fanout_map(g, slope=2e7, bump=2e4, width=15 * wl.UM)
    else:
        nz = 60
        dz = 5 * wl.UM * (400 / nz) * 0.25
        g, f, ins, phi, dk = _shg_case(32, 64, nz, dz, 89)
        w = np.array([f[0].n / (f[1].n * float(np.sum(np.abs(ins[1].astype(np.complex128)) ** 2))), 0.0])
        pf = 1
        m = _fanout_map(g)
    maps = np.stack([m, 0.5 * m.max() - 0.8 * m, 0.4 * m])
    edges = [0.31 * nz * dz, 0.72 * nz * dz]
    prob = oracle.make_problem(g, f, wl.D_EFF)
    ins128 = [a.astype(np.complex128) for a in ins]
    Jr, gphi_r, gdk_r = oracle.adjoint_gradient(prob, ins128, nz, dz, dk, w, phi=phi, phi_field=pf, z_edges=edges,
                                                maps=maps)
    errs = {}
    for interval in (0, 7, -1):
        J, gphi, gdk = _gpu_grad(g, f, ins, phi, dk, nz, dz, w, interval=interval, phi_field=pf, z_edges=edges,
                                 maps=maps)
        errs[interval] = (abs(J / Jr - 1), rel_l2(gphi, gphi_r), rel_l2(gdk, gdk_r))
        assert errs[interval][0] < 1e-4, errs
        assert errs[interval][1] < GRAD_TOL and errs[interval][2] < GRAD_TOL, errs
    # the z-resolution is felt: the gradient under the first segment's map alone is far off
    _, _, gdk1 = oracle.adjoint_gradient(prob, ins128, nz, dz, dk, w, phi=phi, phi_field=pf, dk_map=maps[0])
    assert rel_l2(gdk1, gdk_r) > 20 * GRAD_TOL
