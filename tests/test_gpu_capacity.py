"""List capacity overflow and errors during rbe_step (include/rbe.h,
rbe_set_capacity and rbe_step).

A list longer than its capacity makes that evaluation's forces wrong, so the
library must not integrate on it: rbe_step stops at a latched error, and a
capacity overflow is retried once with capacities grown to the counts met.
Checked here against the oracle's integrator on the same draws: a run whose
capacities are far too small (32 core, 32 shell) ends where a run with the
automatic capacities ends; a run that meets a non-finite position stops at
the step whose force evaluation found it and reports that step; a waiting
rbe_forces call retries too, and rbe_sync_status sizes the next call.
"""
import numpy as np
import pytest

from gpu_util import cond_err, oracle, params, rbe, systems

pytestmark = pytest.mark.gpu


def _dev(a, dt=None):
    import torch
    return torch.tensor(a, dtype=dt or torch.float64, device="cuda")


def _start(s, step0):
    """Device arrays of s and F at (pos, step0) from a context with automatic
    capacities."""
    import torch
    pos, q, typ = _dev(s.pos), _dev(s.q), _dev(s.type, torch.int32)
    mol = None if s.mol is None else _dev(s.mol, torch.int32)
    F = torch.empty_like(pos)
    ref = rbe.Context.for_system(s)
    ref.forces(step0, pos, q, typ, mol, F)
    assert ref.sync_status() == 0
    ref.close()
    return pos, _dev(s.vel), _dev(s.mass), q, typ, mol, F


@pytest.mark.parametrize("precision", [rbe.FP64, rbe.MIXED])
def test_step_retries_capacity_overflow(precision):
    s = systems.electrolyte()
    step0, nsteps, dt = 4, 6, 0.002
    ctx = rbe.Context.for_system(s, precision=precision)
    ctx.set_capacity(32, 32)                      # below the tails of the ~16 / 115 mean counts
    pos, vel, mass, q, typ, mol, F = _start(s, step0)
    ctx.step(step0, nsteps, dt, 1.0, pos, vel, mass, q, typ, mol, F)   # raises if not recovered
    assert ctx.sync_status() == 0
    info = ctx.info()
    assert info["halt_step"] == -1
    assert info["core_cap"] > 32 and info["shell_cap"] > 32
    if precision == rbe.FP64:
        F0 = oracle.rbe_forces(s.pos, s.q, s.type, s.mol, params(s), step0)["F"]
        orc = oracle.vv_run(s.pos, s.vel, s.mass, s.q, s.type, s.mol, params(s), step0, nsteps, dt, 1.0, F0)
        assert orc["status"] == 0
        assert np.abs(pos.cpu().numpy() - orc["pos"]).max() < 1e-10 * s.L
        ref_F = oracle.rbe_forces(orc["pos"], s.q, s.type, s.mol, params(s), step0 + nsteps)
        assert cond_err(F.cpu().numpy(), ref_F) < 1e-11
    # the same trajectory as a run with automatic capacities (the lists and
    # batches are identical; only block partial sums may round differently)
    ref = rbe.Context.for_system(s, precision=precision)
    p2, v2, m2, q2, t2, mo2, F2 = _start(s, step0)
    ref.step(step0, nsteps, dt, 1.0, p2, v2, m2, q2, t2, mo2, F2)
    assert np.abs(pos.cpu().numpy() - p2.cpu().numpy()).max() < 1e-9 * s.L
    ctx.close()
    ref.close()


def test_step_stops_at_nonfinite_position_and_reports_the_step():
    import torch
    s = systems.electrolyte()
    step0, nsteps, dt = 10, 5, 0.002
    ctx = rbe.Context.for_system(s)
    pos, vel, mass, q, typ, mol, F = _start(s, step0)
    vel[7, 0] = float("inf")                      # the first drift makes a non-finite position
    p0, v0, F0 = pos.clone(), vel.clone(), F.clone()
    with pytest.raises(rbe.RbeError) as e:
        ctx.step(step0, nsteps, dt, 1.0, pos, vel, mass, q, typ, mol, F)
    assert e.value.code == rbe.ENONFINITE
    assert ctx.info()["halt_step"] == step0 + 1
    # the state is the one after the first half kick and drift of step 1: the
    # second half kick and every later step did nothing
    v_half = v0 + 0.5 * dt * F0 / mass[:, None]
    p_exp = p0 + dt * v_half
    ok = torch.isfinite(p_exp).all(1)
    assert torch.equal(pos[ok], p_exp[ok])
    assert torch.equal(vel[ok], v_half[ok])
    assert ctx.sync_status() == rbe.ENONFINITE    # still latched for the caller
    assert ctx.sync_status() == 0
    ctx.close()


def test_waiting_forces_call_retries_and_sync_status_grows_caps():
    s = systems.water(4000, seed=4)
    step = 3
    ref = oracle.rbe_forces(s.pos, s.q, s.type, s.mol, params(s), step)
    ctx = rbe.Context.for_system(s)
    ctx.set_capacity(32, 32)
    # host pointers: the call waits, reads the status and retries once
    F = np.zeros((s.n, 3))
    ctx.forces(step, s.pos, s.q, s.type.astype(np.int32), s.mol.astype(np.int32), F)
    assert ctx.sync_status() == 0
    assert cond_err(F, ref) < 1e-11
    # device pointers: the overflow is latched; rbe_sync_status reports it and
    # the next call runs with room for the counts met
    import torch
    c2 = rbe.Context.for_system(s)
    c2.set_capacity(32, 32)
    pos, q, typ, mol = _dev(s.pos), _dev(s.q), _dev(s.type, torch.int32), _dev(s.mol, torch.int32)
    Fd = torch.empty_like(pos)
    c2.forces(step, pos, q, typ, mol, Fd)
    assert c2.sync_status() == rbe.ECAPACITY
    c2.forces(step, pos, q, typ, mol, Fd)
    assert c2.sync_status() == 0
    assert cond_err(Fd.cpu().numpy(), ref) < 1e-11
    ctx.close()
    c2.close()
