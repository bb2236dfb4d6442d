"""Failure detection and error paths on the GPU, without faulting it.

Every failure here is made the allowed way: a bounded device wait given a
zero limit (so it runs out on purpose and the kernel returns an error status
the host reads), an allocation that the library's fault-injection hook makes
report failure on the host, a call out of order, or a non-finite input.
After each, the same context or batch must work again and give the same
numbers as a fresh one."""
import ctypes
import threading

import numpy as np
import pytest

from paper_2609_08384_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2609_08384_gb300 import build
    build.build()


def _br():
    import paper_2609_08384_gb300 as br
    return br


def _opg_small():
    g = wl.Grid(32, 24, 256, 12.5 * wl.UM, 12.5 * wl.UM, 40 * wl.FS)
    fields = [wl.FieldParams(wl.LAM_P, wl.N_P, delta=1e-10, k2=2e-25, rho=2e-3),
              wl.FieldParams(wl.LAM_S, wl.N_S, k2=1e-25),
              wl.FieldParams(wl.LAM_I, wl.N_I, delta=-1e-10, k2=5e-26, rho=1e-3)]
    a0 = wl.peak_amplitude(1e13, wl.N_P)
    rng = np.random.default_rng(77)
    init = [wl.focused_pulse(g, fields[0], a0, 60 * wl.UM, 1000 * wl.FS, 2 * wl.MM),
            wl.complex_noise(g, 1e-3 * a0, rng), wl.complex_noise(g, 1e-3 * a0, rng)]
    return g, fields, [torch.from_numpy(a.astype(np.complex64)).cuda() for a in init]


@pytest.mark.parametrize("form", [16, 1], ids=["double_buffered", "prefetching"])
def test_tma_tau_wait_limit_runs_out_and_the_context_recovers(form):
    """TMA tau-pass with a zero wait limit: the waits for the tiles' copies run
    out, the kernel lets its copies land and returns, the next synchronising
    call reports E_TIMEOUT; with the default limit and the fields set again
    the same context propagates bit-identically to the plain tau-pass."""
    br = _br()
    g, fields, dev = _opg_small()
    s = br.Solver(g, fields, wl.D_EFF, 20.0)
    ref = br.Solver(g, fields, wl.D_EFF, 20.0)
    ref.set_fields(dev)
    ref.propagate(6, 10 * wl.UM)
    want = ref.get_fields()
    ref.close()
    s.set_option(br.BRAHMS_OPT_TMA_TAU, form)
    assert s.get_option(br.BRAHMS_OPT_TMA_WAIT_US) == 2000000
    s.set_option(br.BRAHMS_OPT_TMA_WAIT_US, 0)
    s.set_fields(dev)
    s.propagate(6, 10 * wl.UM)
    with pytest.raises(br.BrahmsError) as ei:
        s.sync()
    assert ei.value.status == br.BRAHMS_E_TIMEOUT
    s.set_option(br.BRAHMS_OPT_TMA_WAIT_US, 2000000)
    s.set_fields(dev)
    s.propagate(6, 10 * wl.UM)
    got = s.get_fields()
    for f in range(3):
        assert np.array_equal(got[f], want[f]), f
    with pytest.raises(br.BrahmsError):
        s.set_option(br.BRAHMS_OPT_TMA_WAIT_US, -1)
    s.close()


def _batch(br, problems, mode=0):
    b = br.Batch()
    b.set_mode(mode)
    for p in problems:
        i = b.add(p.grid, p.fields, p.d_eff, p.dk, p.nz, p.dz)
        b.set_fields(i, [torch.from_numpy(a.astype(np.complex64)).cuda() for a in wl.inputs_shg(p)])
    return b


def test_batch_wait_limit_runs_out_and_the_batch_recovers():
    """Persistent batched kernel (the form with device-side waits) with a zero
    wait limit: some CTA finds the previous pass of an instance unfinished,
    its wait runs out, every CTA returns and brahms_batch_sync reports
    E_TIMEOUT.  With the default limit and the fields set again the same
    batch runs clean and matches a fresh batch bit for bit."""
    br = _br()
    probs = [wl.problem_batch_member(64, 128, 50.0, 1.0 * wl.MM, 40),
             wl.problem_batch_member(32, 64, -30.0, 0.5 * wl.MM, 25)]
    fresh = _batch(br, probs, mode=2)
    fresh.run()
    fresh.sync()
    want = [fresh.get_fields(i) for i in range(2)]
    fresh.close()
    b = _batch(br, probs, mode=2)
    b.set_timeout(0.0)
    b.run()
    with pytest.raises(br.BrahmsError) as ei:
        b.sync()
    assert ei.value.status == br.BRAHMS_E_TIMEOUT
    b.set_timeout(5.0)
    for i, p in enumerate(probs):
        b.set_fields(i, [torch.from_numpy(a.astype(np.complex64)).cuda() for a in wl.inputs_shg(p)])
    b.run()
    b.sync()
    for i in range(2):
        got = b.get_fields(i)
        for f in range(2):
            assert np.array_equal(got[f], want[i][f]), (i, f)
    with pytest.raises(br.BrahmsError):
        b.set_timeout(-1.0)
    b.close()


def _raw_init(lib, br, g, fields):
    ctx = ctypes.c_void_p()
    fp = (br.FieldParams * 3)(*[br.field_params(f) for f in fields])
    s = lib.brahms_init_grid(ctypes.byref(ctx), g.nx, g.ny, g.nt, g.dx, g.dy, g.dt, len(fields), fp, wl.D_EFF,
                             0.0, None, 0, None)
    return s, ctx


def test_allocation_failures_report_oom_and_leave_usable_state():
    """The fault-injection hook makes the next allocations fail on the host:
    a context without a caller workspace, the adjoint's checkpoints, the
    thermal buffers and a batch instance each report E_OOM, and the next
    attempt succeeds."""
    br = _br()
    lib = br.load()
    g = wl.Grid(32, 32, 64, 12.5 * wl.UM, 12.5 * wl.UM, 50 * wl.FS)
    fields = wl.shg_fields()
    br.fail_next_allocations(1)
    s, ctx = _raw_init(lib, br, g, fields)
    assert s == br.BRAHMS_E_OOM and not ctx.value
    assert br.pending_allocation_failures() == 0
    s, ctx = _raw_init(lib, br, g, fields)
    assert s == br.BRAHMS_OK
    lib.brahms_free(ctx)

    # thermal model buffers
    sol = br.Solver(g, fields, wl.D_EFF, 0.0)
    br.fail_next_allocations(1)
    with pytest.raises(br.BrahmsError) as ei:
        sol.heat_set(np.zeros((g.ny, g.nx)))
    assert ei.value.status == br.BRAHMS_E_OOM
    sol.heat_set(np.ones((g.ny, g.nx)))
    sol.close()

    # the planes of a map with z-segments: E_OOM, then zero maps in effect and a usable context
    sol = br.Solver(g, fields, wl.D_EFF, 0.0)
    zf = [torch.zeros(g.nt, g.ny, g.nx, dtype=torch.complex64).cuda() for _ in range(2)]
    sol.set_fields(zf)
    br.fail_next_allocations(1)
    with pytest.raises(br.BrahmsError) as ei:
        sol.set_dk_map_z([1e-4, 2e-4], np.ones((3, g.ny, g.nx)))
    assert ei.value.status == br.BRAHMS_E_OOM
    sol.propagate(2, 10 * wl.UM)
    sol.set_dk_map_z([1e-4, 2e-4], np.ones((3, g.ny, g.nx)))
    sol.propagate(2, 10 * wl.UM)
    sol.sync()
    sol.close()

    # a batch instance
    b = br.Batch()
    br.fail_next_allocations(1)
    p = wl.problem_batch_member(32, 64, 10.0, 0.5 * wl.MM, 10)
    with pytest.raises(br.BrahmsError) as ei:
        b.add(p.grid, p.fields, p.d_eff, p.dk, p.nz, p.dz)
    assert ei.value.status == br.BRAHMS_E_OOM
    i = b.add(p.grid, p.fields, p.d_eff, p.dk, p.nz, p.dz)
    b.set_fields(i, [torch.from_numpy(a.astype(np.complex64)).cuda() for a in wl.inputs_shg(p)])
    b.run()
    b.sync()
    b.close()
    br.fail_next_allocations(0)


def _shg_adjoint_case():
    g = wl.Grid(32, 32, 64, 12.5 * wl.UM, 12.5 * wl.UM, 50 * wl.FS)
    fields = wl.shg_fields()
    F = wl.focused_pulse(g, fields[1], wl.peak_amplitude(1e13, wl.N_F), 50 * wl.UM, 200 * wl.FS,
                         1 * wl.MM).astype(np.complex64)
    dev = [torch.zeros_like(torch.from_numpy(F)).cuda(), torch.from_numpy(F).cuda()]
    rng = np.random.default_rng(5)
    return g, fields, dev, rng.normal(0, 0.1, 64), rng.normal(0, 100.0, 20)


def test_adjoint_backward_runs_only_on_its_forward():
    """brahms_adjoint_backward refuses (E_STATE) after a forward that failed
    (checkpoint allocation made to fail) and after any call that changed the
    fields, the profile or the map; it may run twice for one forward, with
    the same result."""
    br = _br()
    g, fields, dev, phi, dk = _shg_adjoint_case()
    nz, dz = 20, 50 * wl.UM
    s = br.Solver(g, fields, wl.D_EFF, 0.0)
    w = s.shg_efficiency_weights(dev)
    J = s.adjoint_forward(dev, dk, nz, dz, w, phi=phi)
    gphi, gdk = s.adjoint_backward(1.0)
    gphi2, gdk2 = s.adjoint_backward(1.0)
    assert np.array_equal(gphi, gphi2) and np.array_equal(gdk, gdk2)
    # a failed forward: the checkpoint memory (larger interval count) cannot be had
    br.fail_next_allocations(1)
    with pytest.raises(br.BrahmsError) as ei:
        s.adjoint_forward(dev, dk, nz, dz, w, phi=phi, checkpoint_interval=-1)
    assert ei.value.status == br.BRAHMS_E_OOM
    with pytest.raises(br.BrahmsError) as ei:
        s.adjoint_backward(1.0)
    assert ei.value.status == br.BRAHMS_E_STATE
    # each state-changing call voids the forward
    changes = [lambda: s.propagate(1, dz), lambda: s.set_fields(dev), lambda: s.set_dk_profile(dk),
               lambda: s.set_dk_map(np.zeros((g.ny, g.nx))), lambda: s.set_dk_map(None)]
    for change in changes:
        # (the last forward runs under the zero map the change before set)
        assert abs(s.adjoint_forward(dev, dk, nz, dz, w, phi=phi) / J - 1) < 1e-5
        change()
        with pytest.raises(br.BrahmsError) as ei:
            s.adjoint_backward(1.0)
        assert ei.value.status == br.BRAHMS_E_STATE
    assert s.adjoint_forward(dev, dk, nz, dz, w, phi=phi) == J
    g3, d3 = s.adjoint_backward(1.0)
    assert np.array_equal(g3, gphi) and np.array_equal(d3, gdk)
    s.close()


def test_failed_thermal_solve_keeps_the_user_map():
    """A thermal solve whose temperature overflows reports E_NONFINITE and
    leaves the map of brahms_set_dk_map in effect: the next propagation equals
    one under that map alone, bit for bit."""
    br = _br()
    g = wl.Grid(32, 32, 64, 12.5 * wl.UM, 12.5 * wl.UM, 50 * wl.FS)
    fields = wl.shg_fields()
    F = wl.focused_pulse(g, fields[1], wl.peak_amplitude(1e13, wl.N_F), 50 * wl.UM, 200 * wl.FS, 1 * wl.MM)
    dev = [torch.zeros(F.shape, dtype=torch.complex64).cuda(), torch.from_numpy(F.astype(np.complex64)).cuda()]
    x = (np.arange(g.nx) - g.nx // 2) * g.dx
    umap = np.broadcast_to(3e5 * x[None, :], (g.ny, g.nx)).copy()
    ref = br.Solver(g, fields, wl.D_EFF, 0.0)
    ref.set_dk_map(umap)
    ref.set_fields(dev)
    ref.propagate(20, 20 * wl.UM)
    want = ref.get_fields()
    ref.close()
    s = br.Solver(g, fields, wl.D_EFF, 0.0)
    s.set_dk_map(umap)
    s.heat_set(np.full((g.ny, g.nx), 1e300))
    with pytest.raises(br.BrahmsError) as ei:
        s.thermal_map(1e-300, 1.0)
    assert ei.value.status == br.BRAHMS_E_NONFINITE
    s.set_fields(dev)
    s.propagate(20, 20 * wl.UM)
    got = s.get_fields()
    for f in range(2):
        assert np.array_equal(got[f], want[f]), f
    s.close()


def test_contexts_created_and_run_from_two_host_threads():
    """Two host threads each create a context on the same GPU (the launch
    configuration is a per-device, thread-safe record) and propagate; both
    match a context run on the main thread bit for bit."""
    br = _br()
    g, fields, dev = _opg_small()
    main = br.Solver(g, fields, wl.D_EFF, 20.0)
    main.set_fields(dev)
    main.propagate(5, 10 * wl.UM)
    want = main.get_fields()
    main.close()
    torch.cuda.synchronize()
    out, errs = [None, None], []

    def work(k):
        try:
            torch.cuda.set_device(0)
            st = torch.cuda.Stream()
            with torch.cuda.stream(st):
                s = br.Solver(g, fields, wl.D_EFF, 20.0, stream=st)
                s.set_fields(dev)
                s.propagate(5, 10 * wl.UM)
                out[k] = s.get_fields()
                s.close()
        except Exception as e:  # noqa: BLE001
            errs.append(e)

    th = [threading.Thread(target=work, args=(k,)) for k in range(2)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    assert not errs, errs
    for k in range(2):
        for f in range(3):
            assert np.array_equal(out[k][f], want[f]), (k, f)
