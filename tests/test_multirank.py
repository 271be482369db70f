"""The multi-rank host logic of bench.py on CPU: two gloo ranks (127.0.0.1) run the
rank helpers the benchmark uses under torchrun.  Each rank tracks its own
sequences (weak scaling, no data-path collective); the only collectives are the
timing barrier and the max / sum reductions that form the whole-job rate."""
import json
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench

    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, _ = bench.dist_env()
    units, secs = 10.0 * (rank + 1), 1.0 + 0.5 * rank  # rank r: 10 (r + 1) units in 1 + r/2 s
    res = dict(rank=r, world=w, t_max=bench.max_over_ranks(secs, w), units=bench.sum_over_ranks(units, w),
               rate=bench.job_rate(units, secs, w))
    bench.barrier(w)
    dist.destroy_process_group()
    with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
        json.dump(res, f)


def test_two_gloo_ranks_reduce_the_job_rate(tmp_path):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp

    world = 2
    mp.spawn(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    got = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(world)]
    for r, g in enumerate(got):
        assert (g["rank"], g["world"]) == (r, world)
        # every rank sees the same reductions: 30 units, slowest rank 1.5 s, 20 units/s
        assert g["t_max"] == 1.5 and g["units"] == 30.0 and g["rate"] == pytest.approx(20.0)


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.max_over_ranks(2.5, 1) == 2.5 and bench.sum_over_ranks(3.0, 1) == 3.0
    assert bench.job_rate(12.0, 4.0, 1) == 3.0


def test_ranks_track_disjoint_sequences():
    sys.path.insert(0, ROOT)
    import bench
    from paper_2105_05600_gb300 import synth

    spec = synth.CONFIGS["learned"]
    used = set()
    for rank in range(8):
        mine = set(bench.rank_seeds(spec["train_seeds"], rank)) | set(bench.rank_seeds(spec["test_seeds"], rank))
        assert len(mine) == len(spec["train_seeds"]) + len(spec["test_seeds"])
        assert not (mine & used)
        used |= mine
        # the batched workload: 16 sequences per rank, seeded 100 * rank + i
        seeds = {sp["seed"] for sp in synth.batched_specs(16, seed=100 * rank)}
        assert len(seeds) == 16 and not (seeds & {sp["seed"] for r2 in range(rank)
                                                  for sp in synth.batched_specs(16, seed=100 * r2)})
