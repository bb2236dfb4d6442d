"""Benchmark of the split-step chi(2) solver.

Default workload: OPG, 3 complex64 fields on a 256x256x512 grid (~33.5 M
points per field), 1000 z-steps of 10 um (walk-off, GVM and GVD on all
fields, seed-drawn noise on signal and idler).  One bench step = upload of
the resident input into the solver state, 1000 split steps, energy readout.

Metric: grid-point * field * z-steps per second.  The JSON line also carries
the roofline of the dominant kernel (CUDA events around every launch, on the
solver's stream), an end-to-end figure through the C ABI with host buffers,
SM clocks sampled during the timed region, and the FP64 CPU oracle timed on
this host's cores on a bounded sample of the same workload.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
Multi-GPU (torchrun): every rank runs an independent replica ("replicas
only": a single split-step instance does not shard on one node here).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "grid-point·field·z-steps/sec and % of HBM roofline, plain vs batched vs adjoint"
UNIT = "grid-point·field·z-steps/s"
KINDS = ("xpass_nl", "ypass_fwd", "tpass_prop", "ypass_inv", "other")
# bytes the four passes of a z-step read and write per grid point and field (16 each)
DESIGN_BYTES = 64
FALLBACK_HBM_GBS = 6800.0
# FP32 peak derived from the unit counts: 152 SMs x 128 FP32 lanes x 2 flop (FMA)
# at the maximum SM clock (MEASURED_PEAKS.json sm_max_mhz, 2070 MHz on this pool)
SMS, FP32_LANES = 152, 128


def _fp32_peak_tflops():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    mhz = 2070.0
    if os.path.exists(p):
        with open(p) as f:
            mhz = float(json.load(f).get("sm_max_mhz", mhz))
    return SMS * FP32_LANES * 2 * mhz * 1e6 / 1e12, mhz


def alg_flops_per_point_field(kind, problem):
    """Algorithmic FP32 flops per grid point per field of one launch.
    FFTs count 5 n log2 n per transform of length n; complex multiply 6,
    complex add 2.  The x-pass runs two RK4 half steps: per point, 4
    right-hand sides (F=3: 6 complex products, F=2: 4), 3 stage inputs and
    the weighted sum: 222 flops (F=3) or 148 (F=2) per RK4."""
    import math
    g, F = problem.grid, problem.nfields
    rk4 = 222.0 if F == 3 else 148.0
    if kind == "xpass_nl":
        return 2 * 5 * math.log2(g.nx) + 2 * rk4 / F
    if kind in ("ypass_fwd", "ypass_inv"):
        return 5 * math.log2(g.ny)
    if kind == "tpass_prop":
        return 2 * 5 * math.log2(g.nt) + 6
    return 0.0


def _env_int(k, d):
    try:
        return int(os.environ.get(k, d))
    except ValueError:
        return d


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return FALLBACK_HBM_GBS, "fallback"


# the sources that define the four pass kernels whose DRAM traffic is recorded
KERNEL_SOURCES = ("fft_core.cuh", "kernels.cuh", "k_xpass.cu", "k_axis.cu")


def _kernel_hash():
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2609_08384_gb300", "csrc")
    for fn in KERNEL_SOURCES:
        with open(os.path.join(csrc, fn), "rb") as f:
            h.update(fn.encode() + f.read())
    return h.hexdigest()[:16]


def _traffic(kind):
    """DRAM bytes per launch of `kind` from the committed ncu summary, or None
    when the kernels changed since the counters were taken."""
    p = os.path.join(ROOT, "profiles", "dram_traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    if d.get("kernel_hash") != _kernel_hash():
        return None
    v = d.get("bytes_per_launch", {}).get(kind)
    return float(v) if v is not None else None


class ClockSampler:
    """nvidia-smi SM clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"brahms_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                c = [x.strip() for x in line.split(",")]
                if len(c) < 9:
                    continue
                try:
                    sm.append(float(c[1]))
                    mx = max(mx, float(c[2]))
                except ValueError:
                    continue
                for n, v in zip(names, c[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def cpu_baseline(problem, inputs, nz_sample=1):
    """The FP64 oracle as it stands, on this host's cores, on nz_sample split
    steps of the same workload."""
    import oracle

    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    oracle.set_threads(cores)
    prob = oracle.problem_from(problem)
    t0 = time.perf_counter()
    oracle.propagate(prob, inputs, nz_sample, problem.dz, problem.dk)
    dt = time.perf_counter() - t0
    units = problem.grid.npoints * problem.nfields * nz_sample
    out = {"value": units / dt, "unit": UNIT, "cores": int(cores), "kind": "oracle",
           "sample": f"{nz_sample} split step(s) of the {problem.name} workload "
                     f"({problem.nfields} fields, FP64), {dt:.1f} s"}
    # one thread, on a bounded sample: one step of the 128x128x256 SFG grid
    from paper_2609_08384_gb300 import workloads as wl
    ps = wl.problem_sfg()
    ins = [np.ascontiguousarray(a, dtype=np.complex64).astype(np.complex128) for a in wl.inputs_sfg(ps)]
    oracle.set_threads(1)
    t0 = time.perf_counter()
    oracle.propagate(oracle.problem_from(ps), ins, 1, ps.dz, ps.dk)
    dt1 = time.perf_counter() - t0
    oracle.set_threads(cores)
    out["one_thread"] = {"value": ps.grid.npoints * ps.nfields / dt1, "unit": UNIT, "cores": 1,
                         "sample": f"1 split step of the {ps.name} workload (3 fields, FP64), {dt1:.1f} s"}
    return out


def make_workload(name):
    from paper_2609_08384_gb300 import workloads as wl
    if name == "opg":
        p = wl.problem_opg()
        return p, wl.inputs_opg(p)
    if name == "sfg":
        p = wl.problem_sfg()
        return p, wl.inputs_sfg(p)
    if name == "shg":
        p = wl.problem_shg_small()
        return p, wl.inputs_shg_small(p)
    raise ValueError(name)


def _dist_init(n_gpus):
    world = _env_int("WORLD_SIZE", 1)
    rank = _env_int("RANK", 0)
    local = _env_int("LOCAL_RANK", 0)
    dist = None
    if world > 1:
        import torch.distributed as dist  # noqa: F811
        import torch
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        dist.init_process_group(backend)
    return world, rank, local, dist


def _barrier(dist):
    if dist is not None:
        dist.barrier()


def _max_over_ranks(dist, v, device):
    if dist is None:
        return v
    import torch
    t = torch.tensor([v], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def batched_form(dev, reps=2, small=False):
    """A sweep in one persistent graph-captured launch (after the autotuner),
    against the same instances run one after another through the
    single-instance path.  Both are timed with CUDA events on their stream
    and include the upload of the resident inputs.  Default: the 64-run SHG
    sweep; small=True: 256 runs of 32x32x64 SHG (200-800 steps each)."""
    import torch

    import paper_2609_08384_gb300 as br
    from paper_2609_08384_gb300 import workloads as wl

    probs = wl.problems_batched_small() if small else wl.problems_batched()
    ins = [[torch.from_numpy(np.ascontiguousarray(a, dtype=np.complex64)).to(dev) for a in wl.inputs_shg(p)]
           for p in probs]
    units = float(sum(p.grid.npoints * 2 * p.nz for p in probs))
    stream = torch.cuda.Stream(device=dev)
    b = br.Batch(stream=stream)
    for p, x in zip(probs, ins):
        i = b.add(p.grid, p.fields, p.d_eff, p.dk, p.nz, p.dz)
        b.set_fields(i, x)
    t_tune = time.perf_counter()
    b.tune(16)
    t_tune = time.perf_counter() - t_tune
    sched = {s: b.schedule(s) for s in range(4)}
    mode = {1: "grouped", 2: "persistent"}.get(b.mode(), "?")

    def one():
        for i, x in enumerate(ins):
            b.set_fields(i, x)
        b.run()

    one()
    b.sync()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        one()
    e1.record(stream)
    b.sync()
    ms_batch = e0.elapsed_time(e1) / reps
    info = b.info()
    b.close()
    # the same instances, one at a time through the single-instance path
    solvers = [br.Solver(p.grid, p.fields, p.d_eff, p.dk, stream=stream, device=dev) for p in probs]
    for s_, x in zip(solvers, ins):
        s_.set_fields(x)
    torch.cuda.synchronize(dev)
    e0.record(stream)
    for s_, p, x in zip(solvers, probs, ins):
        s_.set_fields(x)
        s_.propagate(p.nz, p.dz)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms_seq = e0.elapsed_time(e1)
    for s_ in solvers:
        s_.close()
    return {"value": units / (ms_batch / 1e3), "unit": UNIT, "ms": ms_batch, "instances": len(probs),
            "form": mode, "kernel_launches_per_run": info["launches"] / (reps + 1),
            "persistent_grid": info["grid"], "schedule_by_shape": sched, "tune_s": t_tune,
            "sequential_single_instance": {"value": units / (ms_seq / 1e3), "ms": ms_seq},
            "speedup_vs_sequential": ms_seq / ms_batch,
            "moved_GB_per_s_design": 64.0 * units / (ms_batch / 1e3) / 1e9,
            "workload": ("256 SHG runs, 32^2x64, 200-800 steps, 2 fields" if small else
                         "64 SHG runs, grids {64^2x128, 96^2x192, 128^2x256}, 200-800 steps, 2 fields")}


def cw_form(dev, reps=2):
    """cw focused SHG (nt = 1) at the Boyd-Kleinman optimum, 1024x1024, 1000
    steps: the reduced-dimensional path (x-pass, y-passes, pointwise linear
    step); CUDA events on the solver stream, resident inputs."""
    import torch

    import paper_2609_08384_gb300 as br
    from paper_2609_08384_gb300 import workloads as wl

    p = wl.problem_cw_shg()
    ins = [torch.from_numpy(np.ascontiguousarray(a, dtype=np.complex64)).to(dev) for a in wl.inputs_cw_shg(p)]
    stream = torch.cuda.Stream(device=dev)
    s = br.Solver(p.grid, p.fields, p.d_eff, p.dk, stream=stream, device=dev)
    s.set_fields(ins)
    s.propagate(20, p.dz)
    s.sync()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        s.set_fields(ins)
        s.propagate(p.nz, p.dz)
    e1.record(stream)
    s.sync()
    ms = e0.elapsed_time(e1) / reps
    e, _ = s.energy()
    s.close()
    units = float(p.grid.npoints * 2 * p.nz)
    return {"value": units / (ms / 1e3), "unit": UNIT, "ms": ms, "shg_efficiency": float(e[0] / e.sum()),
            "workload": "cw focused SHG 1024x1024 (nt = 1), w0 20 um, L = 2.84 b, dk b/2 = -0.57, 1000 steps"}


def dk_map_form(dev, inputs, nz=200):
    """OPG with a fan-out mismatch map (dk(x) = 2000 1/m per 100 um of x):
    the per-point stage phases of the x-pass; CUDA events on the solver stream."""
    import torch

    import paper_2609_08384_gb300 as br
    from paper_2609_08384_gb300 import workloads as wl

    p = wl.problem_opg()
    x, _, _ = p.grid.axes()
    m = np.tile(2e7 * x, (p.grid.ny, 1))
    stream = torch.cuda.Stream(device=dev)
    s = br.Solver(p.grid, p.fields, p.d_eff, p.dk, stream=stream, device=dev)
    s.set_dk_map(m)
    s.set_fields(inputs)
    s.propagate(10, p.dz)
    s.sync()
    s.timing(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    s.propagate(nz, p.dz)
    e1.record(stream)
    s.sync()
    ms = e0.elapsed_time(e1)
    kind_ms, kind_n = s.timing(False)
    s.close()
    units = float(p.grid.npoints * p.nfields * nz)
    return {"value": units / (ms / 1e3), "unit": UNIT, "ms": ms,
            "xpass_us_per_launch": float(kind_ms[0] / max(1, kind_n[0]) * 1e3),
            "workload": f"OPG 256x256x512, {nz} steps, fan-out mismatch map dk(x) = 2e7 x (1/m)"}


def diagnostics_form(solver, problem, reps=3):
    """Power trace plus spectrum of the resident OPG fields (each reads the
    state once): wall time per call including the small device-to-host copy."""
    import torch
    solver.sync()
    solver.diagnostics()
    t0 = time.perf_counter()
    for _ in range(reps):
        solver.diagnostics()
    ms = (time.perf_counter() - t0) / reps * 1e3
    nbytes = 2 * 8.0 * problem.grid.npoints * problem.nfields
    return {"ms_per_call": ms, "alg_GB_per_s": nbytes / (ms / 1e3) / 1e9,
            "workload": "power trace + tau spectrum of the 3 x 256x256x512 OPG state"}


def thermal_form(solver, problem, dev, reps=5):
    """Thermal model: the heat load of the resident OPG state (one pass over the
    3 x 256x256x512 fields) timed with CUDA events on the solver stream, and the
    FP64 transverse Poisson solve with its map install (wall time per call,
    including the 4-byte status read) on 256x256, 1024x1024 and 4096x4096."""
    import torch

    import paper_2609_08384_gb300 as br
    from paper_2609_08384_gb300 import workloads as wl

    g = problem.grid
    st = solver.stream
    solver.heat_accumulate(1e6, 1.0)
    solver.sync()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(reps):
        solver.heat_accumulate(1e6, 1.0)
    e1.record(st)
    solver.sync()
    us = e0.elapsed_time(e1) / reps * 1e3
    nbytes = 8.0 * g.npoints * problem.nfields + 16.0 * g.nx * g.ny
    out = {"heat_load_us": us, "heat_load_alg_GB_per_s": nbytes / (us / 1e6) / 1e9,
           "heat_load_workload": "3 x 256x256x512 OPG state, one pass"}

    def solve_ms(s):
        s.thermal_map(1.0, 0.0, want_temperature=False)
        t0 = time.perf_counter()
        for _ in range(reps):
            s.thermal_map(1.0, 0.0, want_temperature=False)
        return (time.perf_counter() - t0) / reps * 1e3

    out[f"solve_ms_{g.nx}x{g.ny}"] = solve_ms(solver)
    solver.set_dk_map(None)
    rng = np.random.default_rng(wl.SEED_BASE + 7)
    for n in (1024, 4096):
        gg = wl.Grid(n, n, 1, 1e-6, 1e-6, 1e-15)
        s = br.Solver(gg, wl.shg_fields(), wl.D_EFF, 0.0, stream=torch.cuda.Stream(device=dev), device=dev)
        s.heat_set(rng.random((n, n)) * 1e9)
        out[f"solve_ms_{n}x{n}"] = solve_ms(s)
        s.close()
    return out


def adjoint_form(dev, store_all=True):
    """SHG efficiency gradient on 128x128x256 over 400 steps (256-entry spectral
    phase, 400-entry mismatch profile), sqrt(nz) checkpointing: the time of the
    checkpointed forward plus the reverse sweep, against the plain forward of
    the same propagation.  CUDA events on the solver stream.  store_all also
    times the form that records every step (54 GB of states)."""
    import torch

    import paper_2609_08384_gb300 as br
    from paper_2609_08384_gb300 import workloads as wl

    p = wl.problem_adjoint()
    a0 = wl.peak_amplitude(1e13, wl.N_F)
    F = wl.focused_pulse(p.grid, p.fields[1], a0, 50 * wl.UM, 200 * wl.FS, p.length).astype(np.complex64)
    dev_in = [torch.zeros_like(torch.from_numpy(F)).to(dev), torch.from_numpy(F).to(dev)]
    stream = torch.cuda.Stream(device=dev)
    s = br.Solver(p.grid, p.fields, p.d_eff, 0.0, stream=stream, device=dev)
    w = s.shg_efficiency_weights(dev_in)
    e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    s.adjoint_forward(dev_in, p.dk_profile, p.nz, p.dz, w, phi=p.spectral_phase)
    s.adjoint_backward(1.0)
    torch.cuda.synchronize(dev)
    e[0].record(stream)
    J = s.adjoint_forward(dev_in, p.dk_profile, p.nz, p.dz, w, phi=p.spectral_phase)
    e[1].record(stream)
    s.adjoint_backward(1.0)
    e[2].record(stream)
    torch.cuda.synchronize(dev)
    s.set_dk_profile(p.dk_profile)
    s.set_fields(dev_in)
    torch.cuda.synchronize(dev)
    e[3].record(stream)
    s.propagate(p.nz, p.dz)
    e0 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    torch.cuda.synchronize(dev)
    ms_fwd, ms_bwd, ms_plain = e[0].elapsed_time(e[1]), e[1].elapsed_time(e[2]), e[3].elapsed_time(e0)
    units = float(p.grid.npoints * 2 * p.nz)
    out = {"value": units / ((ms_fwd + ms_bwd) / 1e3), "unit": UNIT, "eta": J,
           "ms_forward_checkpointed": ms_fwd, "ms_backward": ms_bwd, "ms_plain_forward": ms_plain,
           "gradient_cost_vs_plain_forward": (ms_fwd + ms_bwd) / ms_plain,
           # bytes moved by design per grid point, field and step (the per-segment
           # checkpoint copies left out): forward 4 passes (64 B); backward the
           # recording recomputation (64 B + 2 writes of 8 B) and the reverse
           # passes (64 B + 2 reads of 8 B)
           "moved_GB_per_s_design": 224.0 * units / ((ms_fwd + ms_bwd) / 1e3) / 1e9,
           "workload": "SHG 128x128x256, 400 steps of 5 um, d eta / d(phi[256], dk[400])"}
    if not store_all:
        s.close()
        return out
    # every step recorded in the forward (2 nz states, 54 GB here): no recomputation in the backward
    s.adjoint_forward(dev_in, p.dk_profile, p.nz, p.dz, w, phi=p.spectral_phase, checkpoint_interval=-1)
    s.adjoint_backward(1.0)
    torch.cuda.synchronize(dev)
    e[0].record(stream)
    s.adjoint_forward(dev_in, p.dk_profile, p.nz, p.dz, w, phi=p.spectral_phase, checkpoint_interval=-1)
    e[1].record(stream)
    s.adjoint_backward(1.0)
    e[2].record(stream)
    torch.cuda.synchronize(dev)
    ms_fwd_all, ms_bwd_all = e[0].elapsed_time(e[1]), e[1].elapsed_time(e[2])
    s.close()
    out["store_all"] = {"value": units / ((ms_fwd_all + ms_bwd_all) / 1e3), "ms_forward_recording": ms_fwd_all,
                        "ms_backward": ms_bwd_all,
                        "gradient_cost_vs_plain_forward": (ms_fwd_all + ms_bwd_all) / ms_plain,
                        # recording forward (80 B) and reverse passes (80 B)
                        "moved_GB_per_s_design": 160.0 * units / ((ms_fwd_all + ms_bwd_all) / 1e3) / 1e9,
                        "state_memory_GB": 2 * p.nz * p.grid.npoints * 2 * 8 / 1e9}
    return out


def e2e_pipelined(solvers, host_in, host_out, problem, steps):
    """End to end through the C ABI with two contexts on two streams, one host
    thread each (the calls release the GIL): problem k's propagation waits on
    the device for problem k-1's to finish, so propagations never share the
    GPU, while problem k's host->device copy and problem k-1's device->host
    read overlap them.  Returns seconds for `steps` problems."""
    import threading

    import torch

    done = [torch.cuda.Event() for _ in range(steps)]
    enqueued = [threading.Event() for _ in range(steps)]
    errors = []

    def worker(i):
        try:
            s = solvers[i]
            for k in range(i, steps, 2):
                s.set_fields(host_in[i])
                if k > 0:
                    enqueued[k - 1].wait()
                    s.stream.wait_event(done[k - 1])
                s.propagate(problem.nz, problem.dz)
                done[k].record(s.stream)
                enqueued[k].set()
                s.get_fields(out=host_out[i])
        except Exception as e:  # noqa: BLE001
            errors.append(e)
            for ev in enqueued:
                ev.set()

    th = [threading.Thread(target=worker, args=(i,)) for i in range(2)]
    t0 = time.perf_counter()
    for t in th:
        t.start()
    for t in th:
        t.join()
    dt = time.perf_counter() - t0
    if errors:
        raise errors[0]
    return dt


def run_reference(args):
    world, rank, local, dist = _dist_init(args.gpus)
    if rank != 0:
        return 0
    problem, inputs = make_workload(args.config)
    import oracle
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    oracle.set_threads(cores)
    prob = oracle.problem_from(problem)
    sample = 1
    for _ in range(args.warmup):
        oracle.propagate(prob, inputs, sample, problem.dz, problem.dk)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.propagate(prob, inputs, sample, problem.dz, problem.dk)
    dt = time.perf_counter() - t0
    units = problem.grid.npoints * problem.nfields * sample * args.steps
    v = units / dt
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": _config(problem, args),
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": int(cores), "kind": "oracle",
                             "sample": f"{sample} split step of the {problem.name} workload per bench step"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def _config(problem, args):
    g = problem.grid
    return {"workload": f"{problem.name}_f{problem.nfields}_nz{problem.nz}",
            "grid_xyt": [g.nx, g.ny, g.nt], "fields": problem.nfields, "nz": problem.nz,
            "dz_m": problem.dz, "parallelism": f"replicas x{args.gpus}" if args.gpus > 1 else "single instance",
            "l2": "state (%.0f MB) larger than the 126 MB L2; no flush" % (
                problem.grid.npoints * problem.nfields * 8 / 1e6)}


def run_ours(args):
    import torch

    import paper_2609_08384_gb300 as br

    world, rank, local, dist = _dist_init(args.gpus)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    problem, inputs = make_workload(args.config)
    g = problem.grid
    units_per_step = g.npoints * problem.nfields * problem.nz
    stream = torch.cuda.Stream(device=dev)
    with torch.cuda.stream(stream):
        solver = br.Solver(g, problem.fields, problem.d_eff, problem.dk, stream=stream, device=dev)
        dev_in = [torch.from_numpy(np.ascontiguousarray(a, dtype=np.complex64)).to(dev) for a in inputs]
    torch.cuda.synchronize(dev)

    def step():
        solver.set_fields(dev_in)
        solver.propagate(problem.nz, problem.dz)
        return solver.energy()

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)

    clocks = ClockSampler(local)
    launches0 = solver.launch_count()
    # events around every 10th launch of each kind: the per-launch averages of
    # the timed region at a tenth of the events' own cost (about 1 % when
    # every launch is bracketed)
    solver.timing(True, every=10)
    _barrier(dist)
    torch.cuda.synchronize(dev)
    clocks.start()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        step()
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    clk = clocks.stop()
    _barrier(dist)
    ms = ev0.elapsed_time(ev1)
    kind_ms, kind_n = solver.timing(False)
    launches = solver.launch_count() - launches0
    ms_max = _max_over_ranks(dist, ms, dev)
    value = world * units_per_step * args.steps / (ms_max / 1e3)

    # roofline of the dominant kernel.  HBM view (the reported roofline):
    # algorithmic bytes = one read and one write of every field's state per
    # launch (16 B per grid point per field) against the measured copy
    # bandwidth.  ALU view (roofline_other_bound): algorithmic FP32 flops per
    # launch against the FP32 FMA rate measured on this GPU by the library's
    # probe (brahms_fp32_fma_rate), the nominal unit-count peak beside it.
    main = int(np.argmax(kind_ms[:4]))
    alg_bytes = 16.0 * g.npoints * problem.nfields
    avg_s = kind_ms[main] / max(1, kind_n[main]) / 1e3
    peak, peak_kind = _peaks()
    achieved = alg_bytes / avg_s / 1e9
    traffic = _traffic(KINDS[main])
    roof_hbm = {"bound": "hbm", "kernel": KINDS[main], "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": traffic, "peak_source": f"{peak_kind} hbm_gbs (copy)",
                "alg_bytes_per_launch": alg_bytes}
    fp_nominal, mhz = _fp32_peak_tflops()
    with torch.cuda.stream(stream):
        fp_peak = br.fp32_fma_rate(stream)
    alg_flops = alg_flops_per_point_field(KINDS[main], problem) * g.npoints * problem.nfields
    roof_alu = {"bound": "alu", "kernel": KINDS[main], "achieved": alg_flops / avg_s / 1e12, "peak": fp_peak,
                "unit": "TFLOP/s", "frac": alg_flops / avg_s / 1e12 / fp_peak, "traffic": traffic,
                "peak_source": "measured: brahms_fp32_fma_rate (16 FMA chains per thread on every SM)",
                "nominal_peak": fp_nominal,
                "nominal_source": f"{SMS} SMs x {FP32_LANES} FP32 lanes x 2 flop x {mhz:.0f} MHz",
                "alg_flops_per_launch": alg_flops}
    roofline = roof_hbm
    roofline_other = roof_alu
    total_k = float(np.sum(kind_ms))
    def _rate(k, per_unit):
        return float(per_unit / (kind_ms[k] / max(1, kind_n[k]) / 1e3)) if k < 4 and kind_n[k] else None

    kernels = {KINDS[k]: {"ms_timed": float(kind_ms[k]), "launches_timed": int(kind_n[k]),
                          "us_per_launch": float(1e3 * kind_ms[k] / max(1, kind_n[k])),
                          "share": float(kind_ms[k] / total_k) if total_k else 0.0,
                          "GB_per_s_alg": (_rate(k, alg_bytes) or 0) / 1e9 if k < 4 else None,
                          "TFLOP_per_s_alg": (_rate(k, alg_flops_per_point_field(KINDS[k], problem) * g.npoints *
                                                    problem.nfields) or 0) / 1e12 if k < 4 else None}
               for k in range(5)}
    step_alg_gbs = 16.0 * units_per_step * args.steps / (ms / 1e3) / 1e9

    # end to end through the C ABI with pinned host buffers: first one context
    # (copy in, propagate, copy out, one problem after another), then two
    # contexts whose copies overlap the other's propagation
    host_in = [torch.from_numpy(np.ascontiguousarray(a, dtype=np.complex64)).pin_memory() for a in inputs]
    host_out = [torch.empty_like(h).pin_memory() for h in host_in]
    e2e_steps = max(1, min(args.steps, 3))
    torch.cuda.synchronize(dev)
    _barrier(dist)
    ph = {"set_fields_host_ms": 0.0, "propagate_enqueue_host_ms": 0.0, "get_fields_host_ms": 0.0,
          "propagate_device_ms": 0.0}
    pe = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(e2e_steps)]
    t0 = time.perf_counter()
    for k in range(e2e_steps):
        ta = time.perf_counter()
        solver.set_fields(host_in)
        pe[k][0].record(stream)
        tb = time.perf_counter()
        solver.propagate(problem.nz, problem.dz)
        pe[k][1].record(stream)
        tc = time.perf_counter()
        solver.get_fields(out=host_out)
        td = time.perf_counter()
        ph["set_fields_host_ms"] += 1e3 * (tb - ta)
        ph["propagate_enqueue_host_ms"] += 1e3 * (tc - tb)
        ph["get_fields_host_ms"] += 1e3 * (td - tc)
    t_e2e = time.perf_counter() - t0
    for k in range(e2e_steps):
        ph["propagate_device_ms"] += pe[k][0].elapsed_time(pe[k][1])
    ph = {key: v / e2e_steps for key, v in ph.items()}
    t_e2e = _max_over_ranks(dist, t_e2e, dev)
    nbytes = g.npoints * problem.nfields * 8
    serial = {"value": world * units_per_step * e2e_steps / t_e2e, "steps": e2e_steps, "phases_ms_per_step": ph,
              "form": "one context: copy in, propagate, copy out, one problem after another"}
    stream2 = torch.cuda.Stream(device=dev)
    with torch.cuda.stream(stream2):
        solver2 = br.Solver(g, problem.fields, problem.d_eff, problem.dk, stream=stream2, device=dev)
    pipe_in = [host_in, [torch.empty_like(h).pin_memory().copy_(h) for h in host_in]]
    pipe_out = [host_out, [torch.empty_like(h).pin_memory() for h in host_in]]
    pipe_steps = max(2, min(args.steps, 4))
    torch.cuda.synchronize(dev)
    _barrier(dist)
    t_pipe = e2e_pipelined([solver, solver2], pipe_in, pipe_out, problem, pipe_steps)
    t_pipe = _max_over_ranks(dist, t_pipe, dev)
    solver2.close()
    e2e = {"value": world * units_per_step * pipe_steps / t_pipe, "unit": UNIT,
           "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes, "steps": pipe_steps,
           "form": "two contexts on two streams: each problem's host->device copy and the previous problem's "
                   "device->host read overlap a propagation; propagations run one after another",
           "serial": serial}
    def want(name):
        return not args.no_forms and (args.forms is None or name in args.forms.split(","))

    forms = {"plain": value}
    if want("diagnostics"):
        forms["diagnostics"] = diagnostics_form(solver, problem)
    if want("thermal"):
        forms["thermal"] = thermal_form(solver, problem, dev)
    solver.close()
    if want("cw_focused_shg"):
        forms["cw_focused_shg"] = cw_form(dev)
    if want("dk_map") and problem.name.startswith("opg"):
        forms["dk_map"] = dk_map_form(dev, dev_in)
    if want("batched"):
        forms["batched"] = batched_form(dev)
    if want("batched_small_grids"):
        forms["batched_small_grids"] = batched_form(dev, small=True)
    if want("adjoint"):
        forms["adjoint"] = adjoint_form(dev)
    elif want("adjoint_checkpointed"):
        forms["adjoint"] = adjoint_form(dev, store_all=False)

    if rank != 0:
        return 0
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(problem, inputs, 1)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": _config(problem, args), "roofline": roofline, "roofline_other_bound": roofline_other,
            "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": int(launches), "clocks": clk, "kernels": kernels, "kernel_timing_every": 10,
            "step_hbm": {"alg_GB_per_s": step_alg_gbs, "alg_bytes_per_point_field_step": 16,
                         "design_bytes_per_point_field_step": DESIGN_BYTES,
                         "design_GB_per_s": DESIGN_BYTES * value / 1e9,
                         "design_frac_of_peak": DESIGN_BYTES * value / 1e9 / peak,
                         "note": "design bytes: what the pass structure reads and writes by construction "
                                 "(the ncu DRAM counters of every pass equal them, profiles/); not a measured rate"},
            "forms": forms}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default="opg", choices=["opg", "sfg", "shg"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-forms", action="store_true", help="skip the batched and adjoint forms")
    ap.add_argument("--forms", default=None,
                    help="comma-separated subset of the forms (diagnostics, thermal, cw_focused_shg, dk_map, "
                         "batched, batched_small_grids, adjoint, adjoint_checkpointed); default all but "
                         "adjoint_checkpointed (adjoint includes it)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
