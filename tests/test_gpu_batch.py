"""Batched persistent form (one cooperative launch, graph-captured) against
the single-instance path and the FP64 oracle."""
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


def _run_batch(probs, inputs, tune=False):
    import paper_2609_08384_gb300 as br
    b = br.Batch()
    for p, inp in zip(probs, inputs):
        i = b.add(p.grid, p.fields, p.d_eff, p.dk, p.nz, p.dz)
        b.set_fields(i, [torch.from_numpy(a.astype(np.complex64)).cuda() for a in inp])
    if tune:
        b.tune(4)
    b.run()
    b.sync()
    out = [b.get_fields(i) for i in range(len(probs))]
    info = b.info()
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


def test_batch_matches_single_instance_and_oracle():
    probs = _mixed_problems()
    inputs = [wl.inputs_shg(p) for p in probs]
    out, info, _ = _run_batch(probs, inputs)
    assert info["instances"] == len(probs) and info["grid"] >= 152
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
