"""GPU path against the FP64 oracle over the workloads' own step counts.

The expected values are the oracle's, written by tests/golden/make_long_parity.py
(which calls only oracle/) into tests/golden/long_*.npz: per field the
oracle's energy and power trace over the whole grid and its values at 8192
stored points (half uniform, half among the largest), plus a fingerprint of
the inputs, which is checked first so that a machine whose generators give
other inputs fails instead of comparing different problems.

Cases:
  - SFG, 3 x 128x128x256, all 500 steps of 10 um (the SFG workload);
  - OPG, 3 x 256x256x512, the first 50 of its 1000 steps, and the whole
    1000-step run;
  - one batched instance of each compiled-in batch shape, 220-640 steps;
  - the adjoint workload's gradient on its full 128x128x256 grid over its
    first 40 steps against the oracle's gradient;
  - the full adjoint workload (400 steps): directional derivatives of the
    GPU gradient against FP64 central differences of the oracle objective.
Tolerances: fields 1e-4 relative L2 per field, per-field energy and power
trace 2e-4 (a field within 1e-4 has its energy within ~2e-4), gradients
1e-3 relative."""
import json
import os

import numpy as np
import pytest

from paper_2609_08384_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
GOLD = os.path.join(ROOT, "tests", "golden")
FIELD_TOL = 1e-4
ENERGY_PARITY_TOL = 2e-4
GRAD_TOL = 1e-3

_LOG = []


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2609_08384_gb300 import build
    build.build()
    yield
    path = os.environ.get("BRAHMS_PARITY_LOG")
    if path and _LOG:
        with open(path, "a") as f:
            for rec in _LOG:
                f.write(json.dumps(rec) + "\n")


def _gold(name):
    path = os.path.join(GOLD, f"long_{name}.npz")
    assert os.path.exists(path), f"missing oracle values {path} (tests/golden/make_long_parity.py {name})"
    with np.load(path) as z:
        return {k: z[k] for k in z.files}


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def _check_inputs(d, init, pre=""):
    for f, a in enumerate(init):
        a = np.ascontiguousarray(a, dtype=np.complex64).ravel()
        n2 = float(np.sum(np.abs(a.astype(np.complex128)) ** 2))
        want = float(d[f"{pre}in_norm2_{f}"])
        assert (n2 == want == 0.0) or abs(n2 / want - 1) < 1e-6, f"input {f} differs from the oracle's"
        v, w = a[d[f"{pre}in_idx_{f}"]], d[f"{pre}in_val_{f}"]
        assert np.abs(v - w).max() <= 1e-6 * max(np.abs(w).max(), 1e-30), f"input {f} differs from the oracle's"


def _compare(name, d, got, e_gpu, power, pre=""):
    nf = len(got)
    errs, eerr, perr = [], [], []
    for f in range(nf):
        g = got[f].ravel()[d[f"{pre}idx_{f}"]]
        errs.append(rel_l2(g, d[f"{pre}val_{f}"]))
        eerr.append(abs(e_gpu[f] / d[f"{pre}energy"][f] - 1))
        perr.append(rel_l2(power[f], d[f"{pre}power"][f]))
    _LOG.append({"test": name, "field_rel_l2_sampled": errs, "energy_rel": eerr, "power_rel_l2": perr})
    for f in range(nf):
        assert errs[f] < FIELD_TOL, (name, f, errs)
        assert eerr[f] < ENERGY_PARITY_TOL, (name, f, eerr)
        assert perr[f] < ENERGY_PARITY_TOL, (name, f, perr)


def _run_plain(p, init, nz):
    import paper_2609_08384_gb300 as br
    s = br.Solver(p.grid, p.fields, p.d_eff, p.dk)
    s.set_fields([torch.from_numpy(np.ascontiguousarray(a, dtype=np.complex64)).cuda() for a in init])
    s.propagate(nz, p.dz)
    got = s.get_fields()
    e, _ = s.energy()
    power, _ = s.diagnostics()
    z, phi = s.get_z()
    s.close()
    return got, e, power, z, phi


def test_sfg_128x128x256_all_500_steps():
    d = _gold("sfg_128x128x256_500")
    p = wl.problem_sfg()
    init = wl.inputs_sfg(p)
    _check_inputs(d, init)
    got, e, power, z, phi = _run_plain(p, init, p.nz)
    assert int(d["nz"]) == p.nz and abs(z - p.length) < 1e-12 and abs(phi - float(d["phi"])) < 1e-9
    _compare("sfg_128x128x256_500", d, got, e, power)


def test_opg_256x256x512_first_50_steps():
    d = _gold("opg_256x256x512_50")
    p = wl.problem_opg()
    init = wl.inputs_opg(p)
    _check_inputs(d, init)
    got, e, power, _, _ = _run_plain(p, init, 50)
    _compare("opg_256x256x512_50", d, got, e, power)


def test_opg_256x256x512_whole_1000_step_run():
    """The whole OPG workload, 1000 steps over 10 mm, against the oracle's
    single long host run (16410 s on 8 host cores; the duration is recorded
    in the file)."""
    d = _gold("opg_256x256x512_1000")
    p = wl.problem_opg()
    init = wl.inputs_opg(p)
    _check_inputs(d, init)
    got, e, power, z, phi = _run_plain(p, init, p.nz)
    assert int(d["nz"]) == p.nz and abs(z - p.length) < 1e-12
    _compare("opg_256x256x512_1000", d, got, e, power)


def test_batched_instances_of_every_shape_over_their_full_runs():
    import paper_2609_08384_gb300 as br
    d = _gold("batch_shg_4shapes")
    members = [tuple(m) for m in d["members"]]
    b = br.Batch()
    probs = []
    for m, (nx, nt, dk, length, nz) in enumerate(members):
        p = wl.problem_batch_member(int(nx), int(nt), dk, length * wl.MM, int(nz))
        init = wl.inputs_shg(p)
        _check_inputs(d, init, pre=f"m{m}_")
        i = b.add(p.grid, p.fields, p.d_eff, p.dk, p.nz, p.dz)
        b.set_fields(i, [torch.from_numpy(a.astype(np.complex64)).cuda() for a in init])
        probs.append(p)
    b.run()
    b.sync()
    for m, p in enumerate(probs):
        got = b.get_fields(m)
        # energies and power traces of the batched result through a context's reductions
        s = br.Solver(p.grid, p.fields, p.d_eff, p.dk)
        s.set_fields([torch.from_numpy(a).cuda() for a in got])
        e, _ = s.energy()
        power, _ = s.diagnostics()
        s.close()
        _compare(f"batch_{p.grid.nx}x{p.grid.ny}x{p.grid.nt}_{p.nz}", d, got, e, power, pre=f"m{m}_")
    b.close()


def _adjoint_inputs():
    p = wl.problem_adjoint()
    F = wl.focused_pulse(p.grid, p.fields[1], wl.peak_amplitude(1e13, wl.N_F), 50 * wl.UM, 200 * wl.FS,
                         p.length).astype(np.complex64)
    return p, [np.zeros_like(F), F]


def test_adjoint_gradient_full_grid_against_oracle_gradient():
    """The adjoint workload's grid (SHG 128x128x256) and inputs over the first
    40 of its steps: J, dJ/dphi and dJ/d dk against the oracle's gradient."""
    import paper_2609_08384_gb300 as br
    d = _gold("adjoint_128x128x256_40")
    p, ins = _adjoint_inputs()
    _check_inputs(d, ins)
    nz = int(d["nz"])
    s = br.Solver(p.grid, p.fields, p.d_eff, 0.0)
    dev = [torch.from_numpy(a).cuda() for a in ins]
    w = s.shg_efficiency_weights(dev)
    # the library sums FP32 squares of the complex64 field in FP64 (~1e-9)
    assert np.allclose(w, d["weights"], rtol=1e-7, atol=0)
    J = s.adjoint_forward(dev, p.dk_profile[:nz], nz, p.dz, w, phi=p.spectral_phase)
    gphi, gdk = s.adjoint_backward(1.0)
    s.close()
    errs = dict(J=abs(J / float(d["J"]) - 1), phi=rel_l2(gphi, d["grad_phi"]), dk=rel_l2(gdk, d["grad_dk"]))
    _LOG.append({"test": "adjoint_128x128x256_40", **errs})
    assert errs["J"] < FIELD_TOL, errs
    assert errs["phi"] < GRAD_TOL and errs["dk"] < GRAD_TOL, errs


def test_adjoint_gradient_full_workload_against_fp64_differences():
    """The full adjoint workload (400 steps, 256 phase and 400 mismatch
    entries): the GPU gradient's directional derivatives along two seeded
    directions against FP64 central differences of the oracle's objective
    (h = 1e-3 in rad and 1/mm; Richardson over h and h/2 along the first)."""
    import paper_2609_08384_gb300 as br
    d = _gold("adjoint_128x128x256_400_fd")
    p, ins = _adjoint_inputs()
    _check_inputs(d, ins)
    s = br.Solver(p.grid, p.fields, p.d_eff, 0.0)
    dev = [torch.from_numpy(a).cuda() for a in ins]
    w = s.shg_efficiency_weights(dev)
    J = s.adjoint_forward(dev, p.dk_profile, p.nz, p.dz, w, phi=p.spectral_phase)
    gphi, gdk = s.adjoint_backward(1.0)
    s.close()

    def slope(v):
        return float(np.dot(gphi, v[:256]) + np.dot(gdk, v[256:]) / wl.MM)

    fd0 = d["fd0"]
    rich0 = (4 * fd0[1] - fd0[0]) / 3
    errs = dict(J=abs(J / float(d["J"]) - 1), dir0=abs(slope(d["dir0"]) / rich0 - 1),
                dir1=abs(slope(d["dir1"]) / float(d["fd1"][0]) - 1),
                fd_richardson_change=abs(fd0[0] / rich0 - 1))
    _LOG.append({"test": "adjoint_128x128x256_400_fd", **errs})
    assert errs["J"] < FIELD_TOL, errs
    assert errs["dir0"] < GRAD_TOL and errs["dir1"] < GRAD_TOL, errs
