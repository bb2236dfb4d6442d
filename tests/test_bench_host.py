"""Host-side logic of bench.py on CPU: max-over-ranks timing with two gloo
ranks, the reference arm under torch.distributed.run, and the roofline
bookkeeping."""
import json
import math
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    w, r, _, d = bench._dist_init(world)
    v = bench._max_over_ranks(d, 10.0 + 5.0 * r, "cpu")
    bench._barrier(d)
    q.put((r, w, v))
    d.destroy_process_group()


def test_max_over_ranks_with_gloo():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + os.getpid() % 1000
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res == [(0, 2, 15.0), (1, 2, 15.0)]


def test_reference_arm_under_torchrun_two_ranks():
    port = 29600 + os.getpid() % 1000
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", "--impl", "reference",
           "--gpus", "2", "--steps", "1", "--warmup", "0", "--config", "shg"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["n_gpus"] == 2
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["unit"] == "grid-point·field·z-steps/s" and d["higher_is_better"] is True


def test_algorithmic_flop_counts():
    sys.path.insert(0, ROOT)
    import bench
    from paper_2609_08384_gb300 import workloads as wl
    p = wl.problem_opg()
    # two 256-point transforms (5 n log2 n each) and two RK4 steps of 3 fields
    assert bench.alg_flops_per_point_field("xpass_nl", p) == pytest.approx(80 + 2 * 222 / 3)
    assert bench.alg_flops_per_point_field("ypass_fwd", p) == pytest.approx(40)
    assert bench.alg_flops_per_point_field("tpass_prop", p) == pytest.approx(2 * 5 * math.log2(512) + 6)
    peak, mhz = bench._fp32_peak_tflops()
    assert peak == pytest.approx(152 * 128 * 2 * mhz * 1e6 / 1e12)
