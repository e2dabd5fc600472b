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


def _rho_rank_main(rank, world, port, out):
    import numpy as np
    import torch
    import torch.distributed as dist

    import oracle
    from paper_2204_13595_gb300 import systems
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        s = systems.water(1000, seed=8)
        pr = oracle.make_params(s.L, s.alpha, s.r_c, s.r_s, s.p, s.P, s.seed, k_e=s.k_e, eps=s.eps, sigma=s.sigma)
        m = oracle.sample_k_params(pr, 5)               # drawn on every rank from the same counters
        own = (np.floor(s.pos[:, 0] / s.L * world).astype(int) % world) == rank   # a slab of the box
        part = oracle.rho(s.pos[own], s.q[own], s.L, m)
        t = torch.tensor(np.stack([part.real, part.imag]), dtype=torch.float64)
        dist.all_reduce(t)                               # the one exchange of the Fourier part
        mm = torch.tensor(m, dtype=torch.int64)
        m0 = mm.clone()
        dist.broadcast(m0, 0)
        out.put((rank, int(own.sum()), bool(torch.equal(mm, m0)), t.numpy().copy()))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_sum_rho_partials():
    """The Fourier part's exchange under a domain decomposition (Sec. 3: one
    all-reduce of rho per step): each rank sums rho(k) over the atoms of its
    slab of the box for k samples it draws itself from the shared counters; the
    all-reduced sum equals rho over all atoms, and the samples agree without
    being sent."""
    import numpy as np
    import torch.multiprocessing as mp

    import oracle
    from paper_2204_13595_gb300 import systems
    oracle.build()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rho_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=120) for _ in procs), key=lambda x: x[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    s = systems.water(1000, seed=8)
    pr = oracle.make_params(s.L, s.alpha, s.r_c, s.r_s, s.p, s.P, s.seed, k_e=s.k_e, eps=s.eps, sigma=s.sigma)
    full = oracle.rho(s.pos, s.q, s.L, oracle.sample_k_params(pr, 5))
    assert res[0][1] + res[1][1] == s.n and min(res[0][1], res[1][1]) > 0
    assert res[0][2] and res[1][2]
    for _, _, _, t in res:
        assert np.allclose(t[0] + 1j * t[1], full, rtol=0, atol=1e-12 * np.abs(s.q).sum())
