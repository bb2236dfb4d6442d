"""GPU diagnostics (temporal power trace, energy spectrum over Omega) against
the oracle's, through the C ABI.

On the same complex64 fields the power traces agree to the GPU's FP32
squares of point pairs (summed in FP64; 1e-7 of the peak); the spectrum's
tau transform is FP32 on the GPU (1e-5 of the peak bin).  After a propagation
the fields themselves differ by the propagation's FP32 error (2e-4)."""
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


def _br():
    import paper_2609_08384_gb300 as br
    return br


def _c64(a):
    return np.ascontiguousarray(a, dtype=np.complex64)


def _fields(g, nf, seed):
    rng = np.random.default_rng(wl.SEED_BASE + 300 + seed)
    x, y, t = g.axes()
    out = []
    for f in range(nf):
        w = (0.15 + 0.05 * f) * g.nx * g.dx
        tau = (0.1 + 0.03 * f) * g.nt * g.dt
        env = np.exp(-(x[None, None, :] ** 2 + y[None, :, None] ** 2) / w**2 - (t[:, None, None] / tau) ** 2
                     - 1j * 0.7 * (t[:, None, None] / tau) ** 2)
        noise = rng.standard_normal(env.shape) + 1j * rng.standard_normal(env.shape)
        out.append(_c64(3e7 * (env + 1e-3 * noise)))
    return out


SHAPES = [(32, 32, 64, 3), (24, 48, 96, 2), (64, 16, 512, 3), (16, 8, 4096, 2), (24, 6, 12, 3), (64, 64, 1, 2),
          (48, 1, 32, 3)]


@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: "x".join(map(str, s)))
def test_diagnostics_match_oracle_on_same_fields(shape):
    nx, ny, nt, nf = shape
    g = wl.Grid(nx, ny, nt, 3e-6, 4e-6, 20e-15)
    fp = [wl.FieldParams(wl.LAM_P, wl.N_P), wl.FieldParams(wl.LAM_S, wl.N_S), wl.FieldParams(wl.LAM_I, wl.N_I)][:nf]
    arrs = _fields(g, nf, nx + ny + nt)
    br = _br()
    s = br.Solver(g, fp, wl.D_EFF, 0.0)
    s.set_fields([torch.from_numpy(a).cuda() for a in arrs])
    p_gpu, s_gpu = s.diagnostics()
    e_gpu, _ = s.energy()
    again = s.get_fields()
    s.close()
    prob = oracle.make_problem(g, fp, wl.D_EFF)
    a128 = [a.astype(np.complex128) for a in arrs]
    p_ref = oracle.power_trace(prob, a128)
    s_ref = oracle.spectrum(prob, a128)
    for f in range(nf):
        assert np.array_equal(again[f], arrs[f])  # the state is untouched
        assert np.max(np.abs(p_gpu[f] - p_ref[f])) <= 1e-7 * p_ref[f].max()
        assert np.max(np.abs(s_gpu[f] - s_ref[f])) <= 1e-5 * s_ref[f].max()
        assert p_gpu[f].sum() * g.dt == pytest.approx(e_gpu[f], rel=1e-12)
        assert s_gpu[f].sum() == pytest.approx(e_gpu[f], rel=1e-6)


def test_diagnostics_after_full_size_opg_steps():
    """OPG 256x256x512: two z-steps on both sides, then the diagnostics."""
    br = _br()
    p = wl.problem_opg()
    init = wl.inputs_opg(p)
    s = br.Solver(p.grid, p.fields, p.d_eff, p.dk)
    s.set_fields([torch.from_numpy(_c64(a)).cuda() for a in init])
    s.propagate(2, p.dz)
    p_gpu, s_gpu = s.diagnostics()
    s.close()
    prob = oracle.problem_from(p)
    ref, _ = oracle.propagate(prob, [_c64(a).astype(np.complex128) for a in init], 2, p.dz, p.dk)
    p_ref = oracle.power_trace(prob, ref)
    s_ref = oracle.spectrum(prob, ref)
    for f in range(3):
        assert np.max(np.abs(p_gpu[f] - p_ref[f])) <= 2e-4 * p_ref[f].max()
        assert np.max(np.abs(s_gpu[f] - s_ref[f])) <= 2e-4 * s_ref[f].max()
