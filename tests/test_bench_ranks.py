"""Host logic of bench.py's multi-rank path (one replica of the workload per rank), with
two gloo ranks on the CPU: every rank takes the slowest rank's time, the whole-job value
counts every rank's cells, and the reference arm prints on rank 0 only."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank(rank, world, port, q):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = bench.max_over_ranks(torch, dist, 10.0 + 5.0 * rank, "cpu")
    value = bench.job_mlups(world, 1000, 4, ms)
    q.put((rank, ms, value))
    dist.destroy_process_group()


def test_max_over_ranks_and_job_value_with_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + os.getpid() % 1000
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, value in out:
        assert ms == 15.0                                  # the slower rank's time
        assert value == pytest.approx(2 * 1000 * 4 / 15e-3 / 1e6)


def test_max_over_ranks_without_a_group_is_the_own_time():
    import torch
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(torch, None, 12.5, "cpu") == 12.5


@pytest.mark.parametrize("rank", [0, 1])
def test_reference_arm_prints_on_rank_zero_only(rank):
    env = dict(os.environ, RANK=str(rank), WORLD_SIZE="2", LOCAL_RANK=str(rank))
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "1"], capture_output=True, text=True, env=env, timeout=600)
    assert r.returncode == 0, r.stderr
    lines = [ln for ln in r.stdout.splitlines() if ln.strip().startswith("{")]
    if rank == 0:
        line = json.loads(lines[-1])
        assert line["impl"] == "reference" and line["unit"] == "MLUPS" and line["value"] > 0
    else:
        assert not lines


def test_launch_count_per_step_of_each_layout():
    """gpu_launches is the bench's claim: the step kernel, the edge kernel of the split
    layouts, and the pressure pass unless layout 10 does the pressure columns itself
    (lattices without a body force)."""
    sys.path.insert(0, ROOT)
    import bench
    assert bench.launches_per_step(0, pressure=True) == 2
    assert bench.launches_per_step(2, pressure=True) == 3
    assert bench.launches_per_step(10, pressure=True) == 1
    assert bench.launches_per_step(10, pressure=True, force=True) == 2
    assert bench.launches_per_step(5, pressure=False) == 1
