"""Multi-process host logic of bench.py --gpus N, on CPU with the gloo
backend (world size 2): the maximum of the per-rank times is the same on
every rank, the flame batch is split without loss or overlap, and the
whole-job rate counts every rank's nodes over the slowest rank's time."""
import os
import socket

import pytest

from paper_2101_01702_gb300 import replicas
import workload as w


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    lengths, _ = w.batched_flames_lengths()
    shards = replicas.shard_lengths(lengths, world)
    mine = shards[rank]
    ms = 10.0 + 5.0 * rank                       # the slower rank sets the job time
    ms_max = replicas.max_over_ranks(ms, dist, "cpu")
    nodes = [sum(int(lengths[k]) for k in shards[r]) * 16 for r in range(world)]
    rate = replicas.whole_job_mlups(nodes, 100, ms_max)
    dist.barrier()
    with open(os.path.join(out_dir, f"rank{rank}.txt"), "w") as f:
        f.write(f"{ms_max} {rate} {','.join(map(str, mine))}\n")
    dist.destroy_process_group()


def test_two_gloo_ranks(tmp_path):
    import torch.multiprocessing as mp
    world, port = 2, _free_port()
    mp.start_processes(_rank_main, args=(world, port, str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    got = [(tmp_path / f"rank{r}.txt").read_text().split() for r in range(world)]
    assert float(got[0][0]) == float(got[1][0]) == 15.0
    assert float(got[0][1]) == float(got[1][1])
    idx = sorted(int(k) for g in got for k in g[2].split(","))
    lengths, _ = w.batched_flames_lengths()
    assert idx == list(range(len(lengths)))      # every flame exactly once
    loads = [sum(int(lengths[int(k)]) for k in g[2].split(",")) for g in got]
    assert max(loads) - min(loads) <= max(lengths)
    total = sum(loads) * 16
    assert float(got[0][1]) == pytest.approx(total * 100 / 15e-3 / 1e6)


def test_sharding_single_rank_and_more_ranks_than_flames():
    assert replicas.shard_lengths([5, 3, 9], 1) == [[0, 1, 2]]
    sh = replicas.shard_lengths([5, 3], 4)
    assert sorted(k for s in sh for k in s) == [0, 1] and sum(1 for s in sh if not s) == 2
    with pytest.raises(ValueError):
        replicas.shard_lengths([1], 0)
    assert replicas.max_over_ranks(3.5) == 3.5
