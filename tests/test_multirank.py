"""The benchmark's multi-rank logic on CPU ranks (gloo, world size 2): the max-over-ranks time
and the whole-job weak-scaling value every rank computes, and the reference arm's non-zero
ranks, which exit without work."""
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    dev = torch.device("cpu")
    local_seconds = 2.0 + rank                      # rank 1 is the slow one
    mx = bench.allreduce_max(local_seconds, world, dev)
    value = bench.weak_scaling_value(1000.0, local_seconds, world, dev)
    bench.barrier(world)
    with open(os.path.join(out_dir, f"rank{rank}.txt"), "w") as f:
        f.write(f"{mx} {value}\n")
    dist.destroy_process_group()


def test_max_over_ranks_and_weak_scaling_value(tmp_path):
    world = 2
    port = _free_port()
    ctx = torch.multiprocessing.get_context("spawn")
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, str(tmp_path))) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    for r in range(world):
        mx, value = (float(v) for v in (tmp_path / f"rank{r}.txt").read_text().split())
        assert mx == 3.0                              # the slowest rank's time on every rank
        assert value == pytest.approx(world * 1000.0 / 3.0)


def test_single_rank_value_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.allreduce_max(1.5, 1, None) == 1.5
    assert bench.weak_scaling_value(300.0, 1.5, 1, None) == pytest.approx(200.0)


def test_reference_arm_other_ranks_exit_without_work():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "1"], env=env, capture_output=True, text=True, timeout=300,
                       cwd=ROOT)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""
