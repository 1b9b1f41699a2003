"""The multi-GPU path is replicas only (instances are independent; no
exchange on the data path).  Its host logic -- which instances a rank solves
and how the ranks' timings and pass counts combine into the whole-job line --
runs here as world_size-2 gloo process groups on CPU."""
import os
import socket

import numpy as np
import torch.distributed as dist
import torch.multiprocessing as mp

import bench
from qpgen import make_batch


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, per_rank, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        start = bench.shard_start(rank, per_rank)
        data = make_batch("small", per_rank, seed=0, start=start)
        # rank r: a slower step and fewer passing instances
        ms = 10.0 + 5.0 * rank
        passed = per_rank - rank
        ms_max, total = bench.combine_ranks(ms, passed)
        e2e = bench.max_over_ranks(1.0 + rank)
        out[rank] = (start, data.q.copy(), ms_max, total, e2e)
    finally:
        dist.destroy_process_group()


def test_two_ranks_shard_and_combine():
    world, per_rank = 2, 3
    with mp.Manager() as man:
        out = man.dict()
        mp.spawn(_worker, args=(world, _free_port(), per_rank, out), nprocs=world, join=True)
        res = dict(out)
    whole = make_batch("small", world * per_rank, seed=0)
    for r in range(world):
        start, q, ms_max, total, e2e = res[r]
        assert start == r * per_rank
        # each rank's shard is exactly its slice of the one seeded workload
        np.testing.assert_array_equal(q, whole.q[start:start + per_rank])
        assert ms_max == 15.0            # the slowest rank's step time
        assert total == 2 * per_rank - 1  # passed instances of all ranks
        assert e2e == 2.0
    # disjoint shards that cover the whole job
    starts = sorted(res[r][0] for r in range(world))
    assert starts == [0, per_rank]


def test_reference_arm_other_ranks_do_no_work(capsys):
    class A:
        pass

    bench.run_reference(A(), rank=1, world=2)
    assert capsys.readouterr().out == ""


def test_reference_arm_rank0_prints_one_line(capsys):
    """Rank 0 of the reference arm (the FP64 oracle on the host cores) prints
    one JSON line with the main arm's metric and unit, and its CPU-baseline
    and e2e records (no host-device copies)."""
    import json

    class A:
        workload, batch, steps, warmup, gpus, kappa_relax = "small", 8, 1, 0, 1, 1e-4

    bench.run_reference(A(), rank=0, world=1)
    lines = [ln for ln in capsys.readouterr().out.splitlines() if ln.strip()]
    assert len(lines) == 1
    rec = json.loads(lines[0])
    assert rec["impl"] == "reference"
    assert rec["metric"] == bench.METRIC and rec["unit"] == bench.UNIT
    assert rec["higher_is_better"] is True and rec["value"] > 0
    assert rec["config"]["workload"] == "small" and rec["config"]["sample_per_step"] >= 1
    assert rec["cpu_baseline"]["kind"] == "oracle" and rec["cpu_baseline"]["cores"] >= 1
    assert rec["cpu_baseline"]["value"] == rec["value"]
    assert rec["e2e"] == {"value": rec["value"], "unit": rec["unit"],
                          "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
