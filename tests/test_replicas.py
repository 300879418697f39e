"""Host logic of the multi-GPU form (independent replicas sharded by query) with two CPU ranks
over gloo: disjoint query shards, and the whole-job figure as the units all ranks processed over
the slowest rank's time."""
import json
import os
import socket

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

from paper_2511_22793_gb300 import synth
from paper_2511_22793_gb300.replicas import job_totals, rank_queries, throughput


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir, per_rank):
    import torch.distributed as tdist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    tdist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = rank_queries(synth.make_tx(per_rank * world, seed=2), per_rank, rank, world)
        shards = [None] * world
        tdist.all_gather_object(shards, mine.tolist())
        # rank r processed 1000 (r + 1) units in 2 + r milliseconds
        units, ms = job_totals(1000 * (rank + 1), 2.0 + rank)
        with open(os.path.join(out_dir, "rank%d.json" % rank), "w") as f:
            json.dump({"shards": shards, "units": units, "ms": ms}, f)
        tdist.barrier()
    finally:
        tdist.destroy_process_group()


@pytest.mark.parametrize("per_rank", [1, 3])
def test_two_gloo_ranks(tmp_path, per_rank):
    world = 2
    mp.spawn(_rank_main, args=(world, _free_port(), str(tmp_path), per_rank), nprocs=world, join=True)
    res = [json.load(open(tmp_path / ("rank%d.json" % r))) for r in range(world)]
    full = synth.make_tx(per_rank * world, seed=2)
    for r in range(world):
        assert res[r]["units"] == 1000 + 2000
        assert res[r]["ms"] == 3.0
        assert res[r]["shards"] == res[0]["shards"]
    shards = [np.array(s, dtype=np.float32) for s in res[0]["shards"]]
    # disjoint, and together exactly the seeded list
    assert np.array_equal(np.concatenate(shards), full)
    assert len({tuple(row) for s in shards for row in s.tolist()}) == per_rank * world
    assert throughput(res[0]["units"], res[0]["ms"]) == pytest.approx(3000 / 3e-3)


def test_single_rank_is_local_and_matches_the_one_rank_list():
    assert job_totals(123, 4.5) == (123, 4.5)
    one = rank_queries(synth.make_tx(4, seed=2), 4, 0, 1)
    # the first rows of a longer list are the rows of the shorter one (same seeded stream)
    assert np.array_equal(one, synth.make_tx(8, seed=2)[:4])


def test_bad_shards_raise():
    q = synth.make_tx(4, seed=2)
    with pytest.raises(ValueError):
        rank_queries(q, 3, 0, 2)
    with pytest.raises(ValueError):
        rank_queries(q, 1, 2, 2)
    with pytest.raises(ValueError):
        throughput(10, 0.0)
