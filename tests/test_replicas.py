"""The N > 1 benchmark path on CPU: world-size-2 gloo ranks run the same host logic that
bench.py runs over NCCL (independent replicas, one max-over-ranks reduction of the timed
region, whole-job rate over all ranks)."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, ms_of_rank, out_dir):
    import datetime
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world),
                      RANK=str(rank), LOCAL_RANK=str(rank))
    w, r, local = bench.dist_env()
    dist.init_process_group("gloo", timeout=datetime.timedelta(seconds=60))
    dist.barrier()
    ms = bench.max_over_ranks(ms_of_rank[r], w, "cpu")
    value = bench.whole_job_rate(w, 5, ms)
    seeds = bench.replica_seeds(r)
    dist.barrier()
    dist.destroy_process_group()
    with open(os.path.join(out_dir, f"rank{r}.txt"), "w") as f:
        f.write(f"{w} {r} {local} {ms!r} {value!r} {seeds[0]} {seeds[1]}\n")


@pytest.mark.parametrize("world", [2, 3])
def test_replicas_take_the_slowest_rank_and_count_every_rank(tmp_path, world):
    import torch.multiprocessing as mp
    ms_of_rank = [120.0, 250.5, 80.25][:world]
    ctx = mp.get_context("spawn")
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, ms_of_rank, str(tmp_path))) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    rows = [open(tmp_path / f"rank{r}.txt").read().split() for r in range(world)]
    slowest = max(ms_of_rank)
    seeds = set()
    for r, row in enumerate(rows):
        w, rr, local, ms, value, s0, s1 = row
        assert (int(w), int(rr), int(local)) == (world, r, r)
        # every rank learns the slowest rank's time; the rate counts all ranks' steps
        assert float(ms) == slowest
        assert float(value) == pytest.approx(world * 5 / (slowest / 1e3), rel=1e-15)
        seeds.add((int(s0), int(s1)))
    # independent replicas: no two ranks share a matrix or a sampling seed
    assert len(seeds) == world
    assert len({s[0] for s in seeds}) == world and len({s[1] for s in seeds}) == world


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(42.5, 1, "cpu") == 42.5
    assert bench.whole_job_rate(1, 4, 2000.0) == 2.0
