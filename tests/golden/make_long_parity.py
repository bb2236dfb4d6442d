"""Writes the oracle's expected values for the long-horizon GPU parity tests
(tests/test_gpu_long_parity.py) into tests/golden/long_*.npz.

Only the oracle computes here: the inputs come from the seeded generators in
paper_2609_08384_gb300/workloads.py (no method arithmetic), the propagation,
energies, power traces, gradients and objectives from oracle/.  The fields
of a 3D run are too large to store whole, so each file keeps, per field:
  - the oracle's FP64 energy and power trace P(tau) (sums over the whole grid);
  - the oracle's values (rounded to complex64, relative rounding 6e-8) at
    4096 uniformly drawn points and 4096 points drawn among the 2 % of
    largest magnitude, with their flat indices;
  - a fingerprint of the input (its FP64 norm and 64 sampled values), which
    the test checks before it compares, so that a machine whose generator
    gives other inputs fails loudly instead of comparing different problems.

Usage: python tests/golden/make_long_parity.py [case ...]   (all by default)
Cases and their cost on 8 host cores are listed in CASES.
"""
from __future__ import annotations

import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2609_08384_gb300 import workloads as wl  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))
N_UNIFORM, N_LARGE, N_FINGER = 4096, 4096, 64

# the instances of the batch test: one per compiled-in batch shape, nz >= 200
BATCH_MEMBERS = [
    # nx (= ny), nt, dk (1/m), L (mm), nz
    (32, 64, 150.0, 4.5, 640),
    (64, 128, -120.0, 3.0, 420),
    (96, 192, 60.0, 2.2, 300),
    (128, 256, -180.0, 1.3, 220),
]


def c64(arrs):
    return [np.ascontiguousarray(a, dtype=np.complex64) for a in arrs]


def fingerprint(init, rng):
    out = {}
    for f, a in enumerate(init):
        a = a.ravel()
        idx = np.sort(rng.choice(a.size, N_FINGER, replace=False))
        out[f"in_norm2_{f}"] = np.array(np.sum(np.abs(a.astype(np.complex128)) ** 2))
        out[f"in_idx_{f}"] = idx.astype(np.int64)
        out[f"in_val_{f}"] = a[idx]
    return out


def samples(ref, rng):
    out = {}
    for f, a in enumerate(ref):
        a = a.ravel()
        uni = rng.choice(a.size, N_UNIFORM, replace=False)
        mag = np.abs(a)
        top = np.argpartition(mag, a.size - max(N_LARGE, a.size // 50))[a.size - max(N_LARGE, a.size // 50):]
        big = rng.choice(top, N_LARGE, replace=False)
        idx = np.unique(np.concatenate([uni, big]))
        out[f"idx_{f}"] = idx.astype(np.int64)
        out[f"val_{f}"] = a[idx].astype(np.complex64)
    return out


def propagate_case(name, p, init, nz, dks, seed):
    rng = np.random.default_rng(seed)
    init = c64(init)
    prob = oracle.problem_from(p)
    t0 = time.time()
    ref, phi = oracle.propagate(prob, [a.astype(np.complex128) for a in init], nz, p.dz, dks)
    secs = time.time() - t0
    e, ph = oracle.energy(prob, ref)
    e_in, _ = oracle.energy(prob, [a.astype(np.complex128) for a in init])
    out = dict(nz=np.array(nz), dz=np.array(p.dz), dks=np.asarray(dks, dtype=np.float64), phi=np.array(phi),
               energy=np.asarray(e), energy_in=np.asarray(e_in), power=oracle.power_trace(prob, ref),
               oracle_seconds=np.array(secs), oracle_threads=np.array(oracle.get_threads()))
    out.update(fingerprint(init, rng))
    out.update(samples(ref, rng))
    return out, secs


def case_sfg():
    p = wl.problem_sfg()
    return propagate_case("sfg", p, wl.inputs_sfg(p), p.nz, np.full(p.nz, p.dk), 101)


def case_opg50():
    p = wl.problem_opg()
    return propagate_case("opg50", p, wl.inputs_opg(p), 50, np.full(50, p.dk), 102)


def case_opg1000():
    """The whole OPG workload: 1000 steps of 10 um over 10 mm (about five
    hours of the oracle on 8 host cores)."""
    p = wl.problem_opg()
    return propagate_case("opg1000", p, wl.inputs_opg(p), p.nz, np.full(p.nz, p.dk), 103)


def case_batch():
    out, total = {}, 0.0
    for m, (nx, nt, dk, length, nz) in enumerate(BATCH_MEMBERS):
        p = wl.problem_batch_member(nx, nt, dk, length * wl.MM, nz)
        o, secs = propagate_case(f"batch{m}", p, wl.inputs_shg(p), nz, np.full(nz, dk), 200 + m)
        total += secs
        out.update({f"m{m}_{k}": v for k, v in o.items()})
    out["members"] = np.array(BATCH_MEMBERS, dtype=np.float64)
    return out, total


def adjoint_inputs():
    """The adjoint workload: SHG 128x128x256 with the fundamental a focused
    1 GW/cm^2, 200 fs pulse and the SH zero; J = E_SH(L)/E_F(0) through the
    weights w_SH = n_SH/(n_F sum |A_F(0)|^2), w_F = 0."""
    p = wl.problem_adjoint()
    f = p.fields
    F = wl.focused_pulse(p.grid, f[1], wl.peak_amplitude(1e13, wl.N_F), 50 * wl.UM, 200 * wl.FS,
                         p.length).astype(np.complex64)
    ins = [np.zeros_like(F), F]
    s = float(np.sum(np.abs(F.astype(np.complex128)) ** 2))
    w = np.array([f[0].n / (f[1].n * s), 0.0])
    return p, ins, w


def case_adjoint40():
    """Oracle gradient on the full adjoint grid over the first 40 of its steps."""
    p, ins, w = adjoint_inputs()
    prob = oracle.problem_from(p)
    nz = 40
    dk = p.dk_profile[:nz]
    t0 = time.time()
    J, gphi, gdk = oracle.adjoint_gradient(prob, [a.astype(np.complex128) for a in ins], nz, p.dz, dk, w,
                                           phi=p.spectral_phase, phi_field=1)
    secs = time.time() - t0
    out = dict(nz=np.array(nz), dz=np.array(p.dz), J=np.array(J), grad_phi=gphi, grad_dk=gdk, weights=w,
               oracle_seconds=np.array(secs), oracle_threads=np.array(oracle.get_threads()))
    out.update(fingerprint(ins, np.random.default_rng(301)))
    return out, secs


def case_adjoint400_fd():
    """FP64 central differences of the oracle objective at the full adjoint
    workload (400 steps): along two seeded unit directions v in the scaled
    parameters (phi in rad, dk in 1/mm), with h = 1e-3 (the workload's step)
    and, along the first, also h/2 for a Richardson estimate."""
    p, ins, w = adjoint_inputs()
    prob = oracle.problem_from(p)
    x = [a.astype(np.complex128) for a in ins]
    rng = np.random.default_rng(302)
    dirs = []
    for _ in range(2):
        v = rng.standard_normal(256 + p.nz)
        dirs.append(v / np.linalg.norm(v))
    phi, dk = p.spectral_phase, p.dk_profile

    def J(v, h):
        return oracle.objective(prob, x, p.nz, p.dz, dk + h * v[256:] / wl.MM, w, phi=phi + h * v[:256],
                                phi_field=1)

    t0 = time.time()
    J0 = J(dirs[0], 0.0)
    t_one = time.time() - t0
    h = 1e-3
    fd = []
    for d, v in enumerate(dirs):
        hs = [h, h / 2] if d == 0 else [h]
        fd.append([(J(v, s) - J(v, -s)) / (2 * s) for s in hs])
    secs = time.time() - t0
    out = dict(nz=np.array(p.nz), dz=np.array(p.dz), J=np.array(J0), weights=w, h=np.array(h),
               dir0=dirs[0], dir1=dirs[1], fd0=np.array(fd[0]), fd1=np.array(fd[1]),
               objective_seconds=np.array(t_one), oracle_seconds=np.array(secs),
               oracle_threads=np.array(oracle.get_threads()))
    out.update(fingerprint(ins, np.random.default_rng(303)))
    return out, secs


CASES = {
    # name: (function, approximate cost on 8 x86 cores)
    "sfg_128x128x256_500": (case_sfg, "18 min"),
    "opg_256x256x512_50": (case_opg50, "15 min"),
    "opg_256x256x512_1000": (case_opg1000, "5 h"),
    "batch_shg_4shapes": (case_batch, "8 min"),
    "adjoint_128x128x256_40": (case_adjoint40, "4 min"),
    "adjoint_128x128x256_400_fd": (case_adjoint400_fd, "60 min"),
}


def main(argv):
    oracle.set_threads(os.cpu_count() or 1)
    names = argv or list(CASES)
    for name in names:
        fn, _ = CASES[name]
        t0 = time.time()
        out, secs = fn()
        path = os.path.join(HERE, f"long_{name}.npz")
        np.savez_compressed(path, **out)
        print(f"{name}: oracle {secs:.1f} s, total {time.time() - t0:.1f} s -> {os.path.basename(path)} "
              f"({os.path.getsize(path) / 1e3:.0f} kB)", flush=True)


if __name__ == "__main__":
    main(sys.argv[1:])
