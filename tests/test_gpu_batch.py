"""Batched execution (rbe_batch_*): many replicas of uneven size stepped by one
launch per stage, with the pair kernel as one persistent launch over a
(replica, slot) queue and one MD step replayed as a CUDA graph.  Every
replica must equal, bit for bit, its own single-system path (rbe_forces /
rbe_step on the same context), and through it the oracle."""
import numpy as np
import pytest

from gpu_util import cond_err, oracle, params, rbe, systems

pytestmark = pytest.mark.gpu


def _suite(nrep=8, n_max=8000, seed0=100):
    return systems.batch_replicas(nrep=nrep, n_min=1000, n_max=n_max, seed0=seed0)


def _dev(s):
    import torch
    t = lambda a, dt=torch.float64: torch.tensor(a, dtype=dt, device="cuda")
    return dict(pos=t(s.pos), vel=t(s.vel), mass=t(s.mass), q=t(s.q), typ=t(s.type, torch.int32),
                mol=None if s.mol is None else t(s.mol, torch.int32), F=torch.zeros((s.n, 3), dtype=torch.float64,
                                                                                    device="cuda"))


def _clone(d):
    return {k: (None if v is None else v.clone()) for k, v in d.items()}


def _make(suite, precision):
    ctxs = [rbe.Context.for_system(s, precision=precision) for s in suite]
    devs = [_dev(s) for s in suite]
    b = rbe.Batch(ctxs)
    b.bind([d["pos"] for d in devs], [d["q"] for d in devs], [d["typ"] for d in devs], [d["mol"] for d in devs],
           [d["F"] for d in devs], vel=[d["vel"] for d in devs], mass=[d["mass"] for d in devs],
           dt=[s.dt for s in suite], accel=[s.accel for s in suite])
    return ctxs, devs, b


def _looped_forces(ctx, d, step):
    import torch
    F = torch.empty_like(d["pos"])
    E = torch.zeros(rbe.NE, dtype=torch.float64, device="cuda")
    ctx.forces(step, d["pos"], d["q"], d["typ"], d["mol"], F, E)
    assert ctx.sync_status() == 0
    return F, E.cpu().numpy()


@pytest.mark.parametrize("precision", [rbe.FP64, rbe.MIXED])
def test_batched_forces_equal_single_system_bitwise(precision):
    import torch
    suite = _suite()
    assert {s.name for s in suite} == {"electrolyte", "water"}
    ctxs, devs, b = _make(suite, precision)
    info = b.info()
    assert info["replicas"] == len(suite) and info["atoms"] == sum(s.n for s in suite)
    assert info["families"] == 2 and info["tasks"] >= len(suite)
    E = b.forces(5, energy=True)
    first, st = b.sync_status()
    assert first == 0 and not st.any()
    for r, (ctx, d) in enumerate(zip(ctxs, devs)):
        Fb = d["F"].clone()
        F1, E1 = _looped_forces(ctx, d, 5)
        assert torch.equal(Fb, F1), f"replica {r} ({suite[r].name}, n={suite[r].n})"
        assert np.array_equal(E[r], E1), r


def test_batched_replica_matches_oracle():
    """FP64 batched forces of an electrolyte and a water replica against the
    oracle (same draws), at the single-system tolerance."""
    suite = _suite(nrep=2, n_max=2000, seed0=40)
    ctxs, devs, b = _make(suite, rbe.FP64)
    b.forces(2)
    assert b.sync_status()[0] == 0
    for s, d in zip(suite, devs):
        ref = oracle.rbe_forces(s.pos, s.q, s.type, s.mol, params(s), 2)
        F = d["F"].cpu().numpy()
        if s.n_water_mol:
            F = F - oracle.water_bonded(s.pos, s.L, s.n_water_mol, *s.bonds)[1]
        assert cond_err(F, ref) < 1e-11, s.name


@pytest.mark.parametrize("precision", [rbe.FP64, rbe.MIXED])
def test_batched_steps_equal_looped_rbe_step_bitwise(precision):
    import torch
    suite = _suite(nrep=6, n_max=5000, seed0=200)
    ctxs, devs, b = _make(suite, precision)
    loop = [_clone(d) for d in devs]
    nsteps = 6
    b.forces(0)
    trace = torch.zeros((len(suite), nsteps, 2), dtype=torch.float64, device="cuda")
    b.step(0, nsteps, trace)
    assert b.sync_status()[0] == 0
    for r, (s, ctx, d) in enumerate(zip(suite, ctxs, loop)):
        ctx.forces(0, d["pos"], d["q"], d["typ"], d["mol"], d["F"])
        tr = torch.zeros((nsteps, 2), dtype=torch.float64, device="cuda")
        ctx.step(0, nsteps, s.dt, s.accel, d["pos"], d["vel"], d["mass"], d["q"], d["typ"], d["mol"], d["F"], tr)
        assert ctx.sync_status() == 0
        for k in ("pos", "vel", "F"):
            assert torch.equal(devs[r][k], d[k]), (r, k)
        assert torch.equal(trace[r], tr), r
    # the graph replays continue from where the first call stopped
    b.step(nsteps, 2)
    for r, (s, ctx, d) in enumerate(zip(suite, ctxs, loop)):
        ctx.step(nsteps, 2, s.dt, s.accel, d["pos"], d["vel"], d["mass"], d["q"], d["typ"], d["mol"], d["F"])
        assert torch.equal(devs[r]["pos"], d["pos"]) and torch.equal(devs[r]["F"], d["F"]), r


def test_autotune_keeps_bitwise_equality():
    import torch
    suite = _suite(nrep=6, n_max=12000, seed0=300)
    ctxs, devs, b = _make(suite, rbe.MIXED)
    res = b.autotune(step=1)
    assert len(res["families"]) == 2 and res["untuned_ms"] > 0
    for f in res["families"]:
        assert f["ms"] > 0 and f["ms"] <= res["untuned_ms"] * 1.5
    b.forces(4)
    for r, (ctx, d) in enumerate(zip(ctxs, devs)):
        Fb = d["F"].clone()
        F1, _ = _looped_forces(ctx, d, 4)
        assert torch.equal(Fb, F1), r


@pytest.mark.parametrize("apu,ups", [(16, 1), (96, 0), (32, 3)])
def test_tiling_changes_only_rounding(apu, ups):
    """The work-unit width and slot count change the order of the block
    partials only: lists, batches and per-atom sums are untouched, so FP64
    forces agree with the default tiling to rounding and both with the oracle."""
    s = _suite(nrep=2, n_max=6000, seed0=50)[1]
    d = _dev(s)
    c0 = rbe.Context.for_system(s)
    c1 = rbe.Context.for_system(s)
    c1.set_rbl_tiling(apu, ups)
    F0, E0 = _looped_forces(c0, d, 3)
    F1, E1 = _looped_forces(c1, d, 3)
    ref = oracle.rbe_forces(s.pos, s.q, s.type, s.mol, params(s), 3)
    Fb = oracle.water_bonded(s.pos, s.L, s.n_water_mol, *s.bonds)[1]
    assert cond_err(F1.cpu().numpy() - Fb, ref) < 1e-11
    assert np.max(np.abs(F1.cpu().numpy() - F0.cpu().numpy()) / ref["F_abs"]) < 1e-12
    assert np.allclose(E1, E0, rtol=1e-12, atol=0)


def test_batch_argument_errors():
    import torch
    suite = _suite(nrep=2, n_max=2000, seed0=60)
    c0 = rbe.Context.for_system(suite[0], precision=rbe.FP64)
    c1 = rbe.Context.for_system(suite[1], precision=rbe.MIXED)
    devs = [_dev(s) for s in suite]
    b = rbe.Batch([c0, c1])
    with pytest.raises(rbe.RbeError) as e:
        b.bind([d["pos"] for d in devs], [d["q"] for d in devs], [d["typ"] for d in devs],
               [d["mol"] for d in devs], [d["F"] for d in devs])
    assert e.value.code == rbe.EINVAL
    c1.set_precision(rbe.FP64)
    c1.set_debug(True, 8)
    with pytest.raises(rbe.RbeError):
        b.bind([d["pos"] for d in devs], [d["q"] for d in devs], [d["typ"] for d in devs],
               [d["mol"] for d in devs], [d["F"] for d in devs])
    c1.set_debug(False)
    b.bind([d["pos"] for d in devs], [d["q"] for d in devs], [d["typ"] for d in devs], [d["mol"] for d in devs],
           [d["F"] for d in devs])
    with pytest.raises(rbe.RbeError):       # no velocities bound
        b.step(0, 1)
    host = [d["pos"].cpu() for d in devs]
    with pytest.raises(rbe.RbeError):       # host arrays are refused
        b.bind(host, [d["q"] for d in devs], [d["typ"] for d in devs], [d["mol"] for d in devs],
               [d["F"] for d in devs])
    with pytest.raises(rbe.RbeError):       # the same context twice
        rbe.Batch([c0, c0])
    assert torch.cuda.is_available()


def test_full_suite_batched_equals_looped():
    """The 64-replica suite (1,000 to 50,000 atoms, electrolyte and water, each
    its own box, alpha and P) in mixed precision: batched forces equal each
    replica's single-system forces bit for bit."""
    import torch
    suite = systems.batch_replicas()
    ctxs, devs, b = _make(suite, rbe.MIXED)
    b.forces(9)
    assert b.sync_status()[0] == 0
    for r, (ctx, d) in enumerate(zip(ctxs, devs)):
        Fb = d["F"].clone()
        F1, _ = _looped_forces(ctx, d, 9)
        assert torch.equal(Fb, F1), r
