"""The bench's multi-rank path on CPU with the gloo backend, world size 2:
the max-over-ranks timing and whole-job rate, and the reference arm under
torch.distributed.run (rank 0 alone runs and prints one JSON line, the
other rank exits 0 without work).  Rendezvous on 127.0.0.1."""
import json
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t = bench.max_over_ranks(1.5 + rank, dist)          # rank 1 is the slow one
        rate = bench.whole_job_rate(world, 1000, 4, t)
        out.put((rank, t, rate))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_rate_gloo():
    world, port = 2, free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(world))
    for rank, t, rate in res:
        assert t == 2.5                                     # the slowest rank's time
        assert rate == world * 1000 * 4 / 2.5               # all ranks' cells over it


def test_single_process_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.25) == 3.25
    assert bench.whole_job_rate(1, 10, 2, 4.0) == 5.0


def test_reference_arm_under_torchrun_two_ranks():
    port = free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port),
           os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2", "--steps", "1",
           "--warmup", "1", "--size", "24"]
    env = dict(os.environ, OMP_NUM_THREADS="2")
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=ROOT, env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1                                  # rank 0 only
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle"
    assert d["e2e"]["h2d_bytes_per_step"] == 0


def test_reference_arm_twelve_point_scheme():
    """The reference arm (the oracle) runs the TENO12-AA workload too, on the
    same workload description as our arm."""
    sys.path.insert(0, ROOT)
    import bench
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--scheme", "12",
           "--steps", "1", "--warmup", "1", "--size", "24"]
    env = dict(os.environ, OMP_NUM_THREADS="2")
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=ROOT, env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    d = json.loads([l for l in r.stdout.splitlines() if l.startswith("{")][-1])
    assert d["impl"] == "reference" and d["value"] > 0
    assert d["config"]["scheme"] == 12
    assert d["config"]["workload"] == bench.workload_desc(24, 12)


def test_flop_accounting_reads_the_s6_code():
    """The roofline's FP64 count per face classifies decision bytes the way
    the kernels write them: S6 of the twelve-point scheme as bits 0-4 zero,
    S3..S5 as L - 2 in bits 0-1, the fallback as 0 with cut-off bits."""
    import numpy as np
    sys.path.insert(0, ROOT)
    import bench
    fl = np.array([0x20, 0xE1, 0x42, 0x63, 0x04, 0x1C, 0x00], np.uint8)
    assert bench.selection_class(fl, 6).tolist() == [4, 1, 2, 3, 0, 0, 4]
    assert bench.selection_class(fl, 5).tolist() == [0, 1, 2, 3, 0, 0, 0]
    # S6: the common part, one indicator of 11 non-zero shifted values
    # (11 + 121 + 21 flops), its test (8) and its 12-point scheme (23)
    assert bench.recon_flops(6, 4) == 101 + 153 + 8 + 23
    # the executed count: a decided S6 value is one multiply and 11 fmas
    t0, _ = bench.face_fp64_instructions(3, 6, [0, 0, 0, 0, 0], 0.0)
    t1, _ = bench.face_fp64_instructions(3, 6, [0, 0, 0, 0, 1.0], 0.0)
    assert (t1["dmul"] - t0["dmul"], t1["dfma"] - t0["dfma"]) == (10, 110)
    # the S5 path of TENO12 first tests S6, then S5
    assert bench.recon_flops(6, 3) == 101 + 153 + 8 + (9 + 81 + 17) + 8 + 19
