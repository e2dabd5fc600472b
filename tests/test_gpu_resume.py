"""Checkpoint and resume: every random draw is a function of (seed, step,
atom, slot), so a run of 2n steps equals n steps + save to host + load into a
fresh context + n steps, bit for bit (NVE, and with the Langevin thermostat
when its held force is saved too); a run split into calls on one context or
one batch equals one call."""
import numpy as np
import pytest

from gpu_util import rbe, systems

pytestmark = pytest.mark.gpu

WCA = 2.0 ** (1.0 / 6.0)


def _dev(s):
    import torch
    t = lambda a, dt=torch.float64: torch.tensor(a, dtype=dt, device="cuda")
    return dict(pos=t(s.pos), vel=t(s.vel), mass=t(s.mass), q=t(s.q), typ=t(s.type, torch.int32),
                mol=None if s.mol is None else t(s.mol, torch.int32),
                F=torch.zeros((s.n, 3), dtype=torch.float64, device="cuda"))


def _ctx(s, lang):
    c = rbe.Context.for_system(s, precision=rbe.MIXED)
    if lang:
        c.set_lj_cutoff(WCA)
        c.set_langevin(1.0, 0.5)
    return c


def _steps(c, s, d, step0, n):
    c.step(step0, n, s.dt, s.accel, d["pos"], d["vel"], d["mass"], d["q"], d["typ"], d["mol"], d["F"])
    assert c.sync_status() == 0


@pytest.mark.parametrize("name,lang", [("water", False), ("electrolyte", False), ("electrolyte", True)])
def test_save_load_resume_is_bitwise(name, lang):
    import torch
    s = systems.water(334, seed=6) if name == "water" else systems.electrolyte()
    a, b = _dev(s), _dev(s)
    ca, cb = _ctx(s, lang), _ctx(s, lang)
    for c, d in ((ca, a), (cb, b)):
        c.forces(0, d["pos"], d["q"], d["typ"], d["mol"], d["F"])
    _steps(ca, s, a, 0, 40)
    _steps(cb, s, b, 0, 20)
    # checkpoint to host memory
    ck = {k: b[k].cpu().numpy().copy() for k in ("pos", "vel", "F")}
    if lang:
        FL, st = cb.get_langevin_force(s.n)
        assert st == 20
    del cb
    # restart: a fresh context and fresh device arrays
    cc = _ctx(s, lang)
    c = _dev(s)
    for k in ("pos", "vel", "F"):
        c[k].copy_(torch.tensor(ck[k], device="cuda"))
    if lang:
        cc.set_langevin_force(FL, 20)
    _steps(cc, s, c, 20, 20)
    for k in ("pos", "vel", "F"):
        assert torch.equal(a[k], c[k]), k


def test_split_calls_equal_one_call_with_thermostat():
    import torch
    s = systems.electrolyte()
    a, b = _dev(s), _dev(s)
    ca, cb = _ctx(s, True), _ctx(s, True)
    for c, d in ((ca, a), (cb, b)):
        c.forces(0, d["pos"], d["q"], d["typ"], d["mol"], d["F"])
    _steps(ca, s, a, 0, 30)
    _steps(cb, s, b, 0, 7)
    _steps(cb, s, b, 7, 23)
    for k in ("pos", "vel", "F"):
        assert torch.equal(a[k], b[k]), k


def test_batched_split_equals_looped_one_call():
    import torch
    suite = systems.batch_replicas(nrep=3, n_min=1000, n_max=2500, seed0=900)
    A = [_dev(s) for s in suite]
    B = [{k: (None if v is None else v.clone()) for k, v in d.items()} for d in A]
    cA = [_ctx(s, s.name == "electrolyte") for s in suite]
    cB = [_ctx(s, s.name == "electrolyte") for s in suite]
    b = rbe.Batch(cA)
    b.bind([d["pos"] for d in A], [d["q"] for d in A], [d["typ"] for d in A], [d["mol"] for d in A],
           [d["F"] for d in A], vel=[d["vel"] for d in A], mass=[d["mass"] for d in A],
           dt=[s.dt for s in suite], accel=[s.accel for s in suite])
    b.forces(0)
    b.step(0, 5)
    b.step(5, 4)
    assert b.sync_status()[0] == 0
    for s, c, d, a in zip(suite, cB, B, A):
        c.forces(0, d["pos"], d["q"], d["typ"], d["mol"], d["F"])
        _steps(c, s, d, 0, 9)
        for k in ("pos", "vel", "F"):
            assert torch.equal(a[k], d[k]), (s.name, k)
