"""Batched form (one graph launch: grouped per-shape launches, or one
persistent cooperative kernel) against the single-instance path and the FP64
oracle."""
import numpy as np
import pytest

import oracle
from paper_2609_08384_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2609_08384_gb300 import build
    build.build()


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def _mixed_problems(seed=5, nz_range=(4, 14)):
    rng = np.random.default_rng(wl.SEED_BASE + seed)
    shapes = [(32, 64), (64, 128), (32, 64), (96, 192), (64, 128), (128, 256), (96, 192)]
    probs = []
    for nxy, nt in shapes:
        dk = float(rng.uniform(-200, 200))
        nz = int(rng.integers(*nz_range))
        L = float(rng.uniform(0.5, 5.0)) * wl.MM
        probs.append(wl.problem_batch_member(nxy, nt, dk, L, nz))
    return probs


GROUPED, PERSISTENT = 1, 2


def _run_batch(probs, inputs, tune=False, mode=None):
    import paper_2609_08384_gb300 as br
    b = br.Batch()
    if mode is not None:
        b.set_mode(mode)
    for p, inp in zip(probs, inputs):
        i = b.add(p.grid, p.fields, p.d_eff, p.dk, p.nz, p.dz)
        b.set_fields(i, [torch.from_numpy(a.astype(np.complex64)).cuda() for a in inp])
    if tune:
        b.tune(4)
    b.run()
    b.sync()
    out = [b.get_fields(i) for i in range(len(probs))]
    info = b.info()
    info["mode"] = b.mode()
    sched = [b.schedule(s) for s in range(4)]
    b.close()
    return out, info, sched


def _plain(p, inp):
    import paper_2609_08384_gb300 as br
    s = br.Solver(p.grid, p.fields, p.d_eff, p.dk)
    s.set_fields([torch.from_numpy(a.astype(np.complex64)).cuda() for a in inp])
    s.propagate(p.nz, p.dz)
    out = s.get_fields()
    s.close()
    return out


@pytest.mark.parametrize("mode", [GROUPED, PERSISTENT], ids=["grouped", "persistent"])
def test_batch_matches_single_instance_and_oracle(mode):
    probs = _mixed_problems()
    inputs = [wl.inputs_shg(p) for p in probs]
    out, info, _ = _run_batch(probs, inputs, mode=mode)
    assert info["instances"] == len(probs) and info["mode"] == mode
    assert (info["grid"] >= 152) if mode == PERSISTENT else (info["launches"] > 4 * max(p.nz for p in probs))
    for p, inp, o in zip(probs, inputs, out):
        ref = _plain(p, inp)
        for f in range(2):
            # same kernels and tables; only the FP64 phase bookkeeping differs
            assert rel_l2(o[f], ref[f]) < 1e-6, (p.name, f)
    for k in (0, 3):  # one small and one radix-3 instance against the oracle
        p, inp, o = probs[k], inputs[k], out[k]
        prob = oracle.problem_from(p)
        ref, _ = oracle.propagate(prob, [a.astype(np.complex64).astype(np.complex128) for a in inp], p.nz, p.dz, p.dk)
        for f in range(2):
            assert rel_l2(o[f], ref[f]) < 1e-4, (p.name, f)


def test_grouped_form_is_bit_identical_to_the_single_instance_path():
    """The grouped form runs the single-instance kernels on the same tables
    with the same stage factors (formed on the host with the same phase
    accumulation), so every instance gives brahms_propagate's bits."""
    probs = _mixed_problems(seed=9)
    inputs = [wl.inputs_shg(p) for p in probs]
    out, _, _ = _run_batch(probs, inputs, mode=GROUPED)
    for p, inp, o in zip(probs, inputs, out):
        ref = _plain(p, inp)
        for f in range(2):
            assert np.array_equal(o[f], ref[f]), (p.name, f)


def test_grouped_and_persistent_forms_agree():
    """The two forms run the same kernel code on the same tables: the results
    agree bit for bit (up to the FP64 phase bookkeeping, which both share)."""
    probs = _mixed_problems(seed=8)
    inputs = [wl.inputs_shg(p) for p in probs]
    g, _, _ = _run_batch(probs, inputs, mode=GROUPED)
    q, _, _ = _run_batch(probs, inputs, mode=PERSISTENT)
    for x, y in zip(g, q):
        for f in range(2):
            assert rel_l2(x[f], y[f]) < 1e-6


def test_grouped_batch_takes_shapes_outside_the_persistent_four():
    """Non-square grids and 3 * 2^k lengths outside the persistent kernel's
    shapes: the grouped form runs them, each instance equal to the
    single-instance path; two of them against the oracle.  Several
    instances of one shape with different step counts exercise the shrinking
    prefix of running instances; the persistent form refuses the set."""
    import paper_2609_08384_gb300 as br
    # (8, 6, 4): an instance's rows do not fill whole x-pass CTAs, so its
    # x-passes run one instance per launch
    shapes = [(48, 32, 96), (48, 32, 96), (96, 64, 48), (24, 48, 64), (48, 32, 96), (64, 96, 12), (8, 6, 4)]
    rng = np.random.default_rng(11)
    probs = []
    for k, (nx, ny, nt) in enumerate(shapes):
        g = wl.Grid(nx, ny, nt, 12.5 * wl.UM, 12.5 * wl.UM, 50 * wl.FS)
        probs.append(wl.Problem(f"shg_{nx}x{ny}x{nt}_{k}", g, wl.shg_fields(), wl.D_EFF,
                                float(rng.uniform(-200, 200)), float(rng.uniform(0.5, 2.0)) * wl.MM,
                                int(rng.integers(5, 17))))
    inputs = [wl.inputs_shg(p) for p in probs]
    out, info, _ = _run_batch(probs, inputs)
    assert info["mode"] == GROUPED
    for p, inp, o in zip(probs, inputs, out):
        ref = _plain(p, inp)
        for f in range(2):
            assert rel_l2(o[f], ref[f]) < 1e-6, (p.name, f)
    for k in (0, 3):
        p, inp, o = probs[k], inputs[k], out[k]
        prob = oracle.problem_from(p)
        ref, _ = oracle.propagate(prob, [a.astype(np.complex64).astype(np.complex128) for a in inp], p.nz, p.dz, p.dk)
        for f in range(2):
            assert rel_l2(o[f], ref[f]) < 1e-4, (p.name, f)
    b = br.Batch()
    b.add(probs[0].grid, probs[0].fields, probs[0].d_eff, probs[0].dk, probs[0].nz, probs[0].dz)
    with pytest.raises(br.BrahmsError) as ei:
        b.set_mode(PERSISTENT)
    assert ei.value.status == br.BRAHMS_E_SIZE
    b.close()


def test_batch_repeat_is_deterministic_and_tuner_keeps_results():
    probs = _mixed_problems(seed=6)
    inputs = [wl.inputs_shg(p) for p in probs]
    a, _, _ = _run_batch(probs, inputs)
    b, _, _ = _run_batch(probs, inputs)
    for x, y in zip(a, b):
        for f in range(2):
            assert np.array_equal(x[f], y[f])
    c, _, sched = _run_batch(probs, inputs, tune=True)
    for s in sched:
        assert all(v in (1, 2, 4, 8, 16, 32, 64) for v in s[:3]) and s[3] in (1, 2)
    for x, y in zip(a, c):
        for f in range(2):
            assert np.array_equal(x[f], y[f])  # the schedule changes who computes, not what


def test_batch_64_instance_sweep_energy():
    """The 64-run SHG sweep (grids from {64^2x128, 96^2x192, 128^2x256},
    dk in [-200, 200] 1/m, L in [0.5, 5] mm, 200-800 steps): every instance
    conserves its total energy sum n|A|^2 (lossless), and a sample of
    instances matches the single-instance path."""
    probs = wl.problems_batched()
    inputs = [wl.inputs_shg(p) for p in probs]
    out, info, _ = _run_batch(probs, inputs)
    assert info["instances"] == 64
    for p, inp, o in zip(probs, inputs, out):
        n = [f.n for f in p.fields]
        e0 = sum(n[f] * np.sum(np.abs(inp[f].astype(np.complex64)) ** 2) for f in range(2))
        e1 = sum(n[f] * np.sum(np.abs(o[f].astype(np.complex128)) ** 2) for f in range(2))
        assert abs(e1 / e0 - 1) < 1e-5, p.name
        assert np.sum(np.abs(o[0]) ** 2) > 0  # some SH generated
    for k in (0, 17, 41):
        ref = _plain(probs[k], inputs[k])
        for f in range(2):
            assert rel_l2(out[k][f], ref[f]) < 1e-5
