"""Host-side multi-rank logic of the replica runs, on CPU with the gloo backend (world size 2)."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "WORLD_SIZE": str(world),
                       "RANK": str(rank), "LOCAL_RANK": str(rank)})
    from paper_2405_05213_gb300 import replicas
    ws = replicas.init("gloo")
    replicas.barrier()
    t = replicas.max_over_ranks(1.0 + rank)  # rank 1 is the slower one
    out[rank] = (ws, t, replicas.aggregate_throughput(100.0, t, ws))
    import torch.distributed as dist
    dist.destroy_process_group()


def test_max_over_ranks_and_aggregate_gloo():
    world = 2
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0] == res[1]
    ws, t, thr = res[0]
    assert ws == 2 and t == 2.0 and thr == pytest.approx(100.0)


def test_single_rank_defaults(monkeypatch):
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    from paper_2405_05213_gb300 import replicas
    assert replicas.dist_env() == (1, 0, 0)
    assert replicas.init("gloo") == 1
    assert replicas.max_over_ranks(3.5) == 3.5
