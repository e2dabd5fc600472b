"""The multi-rank bookkeeping of bench.py (replicas only: one independent
system per rank, timing collectives only) with two gloo ranks on the CPU."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist

    from paper_2204_13595_gb300 import replicas, systems
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ws, r, lr = replicas.world()
        seed = replicas.rank_seed(3, r)
        s = systems.water(300, seed=seed)
        replicas.barrier(ws)
        ms = 10.0 + 5.0 * r                      # a per-rank "time": rank 1 is slower
        mx = replicas.max_over_ranks(ms, ws)
        value = replicas.throughput(ws, 1, mx)
        out.put((r, ws, lr, seed, float(s.pos.sum()), mx, value))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_replicas_and_max_time():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, ws0, l0, seed0, x0, mx0, v0), (r1, ws1, l1, seed1, x1, mx1, v1) = res
    assert (r0, r1) == (0, 1) and ws0 == ws1 == 2 and (l0, l1) == (0, 1)
    # independent replicas: distinct seeds and systems, same size (weak scaling)
    assert seed0 == 3 and seed1 == 4 and x0 != x1
    # every rank sees the slowest rank's time; whole-job throughput = 2 units / max time
    assert mx0 == mx1 == 15.0
    assert v0 == v1 == pytest.approx(2 * 1e3 / 15.0)


def test_single_process_defaults(monkeypatch):
    from paper_2204_13595_gb300 import replicas
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    assert replicas.world() == (1, 0, 0)
    assert replicas.max_over_ranks(7.5, 1) == 7.5
    assert replicas.throughput(1, 1, 8.0) == pytest.approx(125.0)
