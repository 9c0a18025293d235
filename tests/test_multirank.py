"""The multi-rank host logic of bench.py on CPU: two gloo ranks, each with its
own independent instances (replicas), reduce the time by max and the
end-to-end throughput by sum.  No GPU is used."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, lr = bench.dist_env()
    ms_local = 10.0 + 5.0 * rank  # rank 1 is the slow one
    ms = bench.reduce_over_ranks(ms_local, dist, "max")
    e2e = bench.reduce_over_ranks(100.0 * (rank + 1), dist, "sum")
    value = bench.job_throughput(w, 3, 1000, 20, ms)
    q.put((r, w, lr, ms, e2e, value))
    dist.destroy_process_group()


def test_two_gloo_ranks_reduce_like_the_bench():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r, (rank, w, lr, ms, e2e, value) in enumerate(out):
        assert (rank, w, lr) == (r, 2, r)
        assert ms == 15.0  # max over ranks
        assert e2e == 300.0  # sum over ranks
        assert value == pytest.approx(2 * 3 * 1000 * 20 / 0.015)


def test_single_process_defaults():
    import bench
    assert bench.reduce_over_ranks(7.0, None) == 7.0
    assert bench.job_throughput(1, 3, 10, 2, 1000.0) == pytest.approx(60.0)


@pytest.mark.parametrize("workload", ["small_64x48x48", "surrogate_1536"])
def test_reference_arm_prints_its_json_line(workload):
    """bench.py --impl reference times the CPU oracle and prints one JSON line
    with the contract's keys (no GPU needed); on a batched workload it samples
    the batch's first instance."""
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference",
                          "--steps", "2", "--warmup", "1", "--workload", workload],
                         capture_output=True, text=True, timeout=300, cwd=root)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference"
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "cpu_baseline", "e2e", "config"):
        assert key in line, key
    assert line["value"] > 0 and line["cpu_baseline"]["cores"] == (os.cpu_count() or 1)
    assert line["e2e"]["h2d_bytes_per_step"] == 0
