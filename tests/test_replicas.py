"""Host logic of the multi-GPU replica mode (independent systems per rank, no data-path collective),
run with two gloo ranks on the CPU: the partition of a sweep, the max-over-ranks job time and the
gather of per-rank reports."""
import os
import socket
import tempfile

import pytest

from paper_1705_08849_gb300 import replicas


def test_block_partition_covers_each_unit_once():
    for n in range(0, 40):
        for world in range(1, 9):
            owned = []
            sizes = []
            for rank in range(world):
                lo, hi = replicas.block(n, world, rank)
                assert 0 <= lo <= hi <= n
                owned.extend(range(lo, hi))
                sizes.append(hi - lo)
            assert owned == list(range(n))  # contiguous, in rank order, each unit once
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        replicas.block(4, 2, 2)


def test_single_process_fallbacks():
    assert replicas.max_over_ranks(3.5) == 3.5
    assert replicas.gather_to_rank0({"a": 1}) == [{"a": 1}]


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_path):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        lo, hi = replicas.block(7, world, rank)
        t = replicas.max_over_ranks(10.0 * rank + 1.0)
        reports = replicas.gather_to_rank0({"rank": rank, "block": [lo, hi], "time_ms": 10.0 * rank + 1.0})
        if rank == 0:
            import json
            with open(out_path, "w") as fh:
                json.dump({"max": t, "reports": reports}, fh)
        else:
            assert reports is None
            assert t == 11.0
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
    import json

    import torch.multiprocessing as mp
    with tempfile.TemporaryDirectory() as d:
        out = os.path.join(d, "rank0.json")
        mp.start_processes(_rank_main, args=(2, _free_port(), out), nprocs=2, join=True, start_method="spawn")
        with open(out) as fh:
            r = json.load(fh)
    assert r["max"] == 11.0
    assert [x["rank"] for x in r["reports"]] == [0, 1]
    assert [x["block"] for x in r["reports"]] == [[0, 4], [4, 7]]
