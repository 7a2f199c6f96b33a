"""The multi-rank path of the benchmark on CPU: two gloo ranks (world size 2), as torchrun
would start them.  Each rank times its own independent field (weak scaling); the job time is
the maximum over ranks, the throughput counts every rank's points, and only rank 0 runs and
prints the CPU-oracle reference arm."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = bench.max_over_ranks(10.0 + 5.0 * rank, world, "cpu")   # rank 1 is the slow one
        val = bench.job_throughput(world, 18, 64 ** 3, 4, ms)

        class A:
            size, steps, warmup, P = 64, 1, 0, 4
        ref = bench.run_reference(A, rank, world)
        dist.barrier()
        q.put((rank, ms, val, None if ref is None else (ref["impl"], ref["n_gpus"], ref["value"] > 0)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_max_time_and_weak_scaling_value():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=240)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=5) for _ in range(world))
    for rank, ms, val, ref in got:
        assert ms == 15.0                         # the slowest rank sets the job time
        assert val == pytest.approx(2 * 18 * 64 ** 3 * 4 / 15e-3 / 1e9)
        if rank == 0:
            assert ref == ("reference", 2, True)
        else:
            assert ref is None                    # only rank 0 runs the reference arm


def test_reference_arm_json_line_on_cpu():
    """`bench.py --impl reference` needs no GPU: it prints one JSON line with the contract's keys."""
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0", "--size", "64"], capture_output=True, text=True, timeout=600,
                         cwd=root)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
