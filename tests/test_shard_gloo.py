"""Multi-process ensemble path on CPU ranks (gloo, world size 2): instances
are partitioned across ranks, each rank advances its own (here with the
oracle, standing in for a rank's GPU), and the gathered states equal a
single-process run instance by instance."""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1805_08846_gb300 import inputs
from paper_1805_08846_gb300.shard import gather_by_instance, partition_instances


def test_partition_balances_and_covers():
    cells = [5, 100, 7, 64, 64, 3, 40, 41]
    parts = partition_instances(cells, 3)
    flat = sorted(i for p in parts for i in p)
    assert flat == list(range(len(cells)))
    loads = [sum(cells[i] for i in p) for p in parts]
    assert max(loads) - min(loads) <= max(cells)
    assert partition_instances(cells, 1) == [list(range(len(cells)))]
    with pytest.raises(ValueError):
        partition_instances(cells, 0)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle
        probs = inputs.sw_ensemble(B=5, nmin=12, nmax=40)
        parts = partition_instances([p.ncells for p in probs], world)
        local = {}
        for i in parts[rank]:
            r = oracle.Oracle(probs[i]).run_steps(probs[i].q0, 4)
            local[i] = (r["q"], r["t"])
        merged = gather_by_instance(local, world)
        if rank == 0:
            np.savez(os.path.join(out_dir, "merged.npz"),
                     **{f"q{i}": merged[i][0] for i in merged},
                     **{f"t{i}": np.array(merged[i][1]) for i in merged})
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_rank_ensemble_equals_single_process(tmp_path):
    import oracle
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world,
                       join=True, start_method="spawn")
    merged = np.load(os.path.join(tmp_path, "merged.npz"))
    probs = inputs.sw_ensemble(B=5, nmin=12, nmax=40)
    for i, p in enumerate(probs):
        r = oracle.Oracle(p).run_steps(p.q0, 4)
        np.testing.assert_array_equal(merged[f"q{i}"], r["q"])
        assert float(merged[f"t{i}"]) == r["t"]
