"""The allocation-free energy entry point (brahms_energy_static) against the
context-based brahms_energy, on two calls in a row.

brahms_energy_static exists for callers that cannot let the library allocate
device memory (their GPU memory belongs to another allocator, or their host
forbids a library's own cudaMalloc, or they cannot afford the synchronisation
cudaMalloc/cudaFree may cause); it keeps its partial sums in a fixed array
inside the library instead."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ENERGY_TOL = 1e-5  # the energy tolerance of the GPU parity tests


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2609_08384_gb300 import build
    build.build()


def _static_energy(lib, fields, grid, fps, stream):
    import paper_2609_08384_gb300 as br
    out = torch.zeros(len(fields), dtype=torch.float64, device="cuda")
    ptrs = (ctypes.c_void_p * len(fields))(*[ctypes.c_void_p(t.data_ptr()) for t in fields])
    fpa = (br.FieldParams * 3)(*[br.field_params(f) for f in fps])
    rc = lib.brahms_energy_static(ptrs, len(fields), grid.nx, grid.ny, grid.nt, grid.dx, grid.dy, grid.dt,
                                  fpa, ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream.cuda_stream))
    assert rc == br.BRAHMS_OK, br.status_string(rc)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def test_energy_static_matches_brahms_energy_twice():
    import paper_2609_08384_gb300 as br
    from paper_2609_08384_gb300 import workloads as wl

    lib = br.load()
    g = wl.Grid(64, 48, 96, 4 * wl.UM, 4 * wl.UM, 30 * wl.FS)
    fps = [wl.FieldParams(wl.LAM_P, wl.N_P, delta=1e-10, k2=2e-25, rho=2e-3),
           wl.FieldParams(wl.LAM_S, wl.N_S, k2=1e-25),
           wl.FieldParams(wl.LAM_I, wl.N_I, delta=-1e-10, rho=1e-3)]
    rng = np.random.default_rng(123)
    init = [(rng.standard_normal((96, 48, 64)) + 1j * rng.standard_normal((96, 48, 64))).astype(np.complex64) * 3e7
            for _ in range(3)]
    s = br.Solver(g, fps, wl.D_EFF, 50.0)
    stream = s.stream
    s.set_fields([torch.from_numpy(a).cuda() for a in init])
    for call in range(2):
        e_ref, _ = s.energy()
        dev = s.get_fields(on_device=True)
        e_static = _static_energy(lib, dev, g, fps, stream)
        assert np.all(np.abs(e_static / e_ref - 1) < ENERGY_TOL), (call, e_static, e_ref)
        # change the fields before the second call
        s.propagate(3, 5 * wl.UM)
    # outside the stated limits the call refuses with E_SIZE
    ptrs = (ctypes.c_void_p * 4)(*([ctypes.c_void_p(dev[0].data_ptr())] * 4))
    fpa = (br.FieldParams * 4)(*[br.field_params(fps[0])] * 4)
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    rc = lib.brahms_energy_static(ptrs, 4, g.nx, g.ny, g.nt, g.dx, g.dy, g.dt, fpa,
                                  ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream.cuda_stream))
    assert rc == br.BRAHMS_E_SIZE
    s.close()
