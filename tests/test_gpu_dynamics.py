"""Velocity-Verlet driver (rbe_step) against the oracle's integrator on the
same draws, and the bonded water terms."""
import numpy as np
import pytest

from gpu_util import cond_err, gpu_forces, oracle, params, rbe, rel_err_components, systems

pytestmark = pytest.mark.gpu


def _run(s, nsteps, bonds):
    import torch
    ctx = rbe.Context.for_system(s) if bonds else rbe.Context(s.L, s.alpha, s.r_c, s.r_s, s.p, s.P, s.seed,
                                                              k_e=s.k_e, eps=s.eps, sigma=s.sigma)
    dev = lambda a, dt=torch.float64: torch.tensor(a, dtype=dt, device="cuda")
    pos, vel, mass, q = dev(s.pos), dev(s.vel), dev(s.mass), dev(s.q)
    typ = dev(s.type, torch.int32)
    mol = None if s.mol is None else dev(s.mol, torch.int32)
    F = torch.empty_like(pos)
    ctx.forces(0, pos, q, typ, mol, F)
    F0 = F.cpu().numpy()
    tr = torch.zeros((nsteps, 2), dtype=torch.float64, device="cuda")
    ctx.step(0, nsteps, s.dt, s.accel, pos, vel, mass, q, typ, mol, F, tr)
    assert ctx.sync_status() == 0
    return F0, pos.cpu().numpy(), vel.cpu().numpy(), F.cpu().numpy(), tr.cpu().numpy()


@pytest.mark.parametrize("kind", ["electrolyte", "water"])
def test_velocity_verlet_matches_oracle(kind):
    if kind == "electrolyte":
        s, nsteps, bonds = systems.electrolyte(), 20, False
    else:
        s, nsteps, bonds = systems.water(334, seed=6), 10, True
    F0, pos, vel, F, tr = _run(s, nsteps, bonds)
    water = (s.n_water_mol, *s.bonds) if bonds else None
    r0 = oracle.rbe_forces(s.pos, s.q, s.type, s.mol, params(s), 0)
    F0o, A = r0["F"], r0["F_abs"]
    if bonds:
        Fb = oracle.water_bonded(s.pos, s.L, s.n_water_mol, *s.bonds)[1]
        F0o, A = F0o + Fb, A + np.abs(Fb)
    # the FP64 bar of the parity tests: 1e-11 of each component's condition scale
    assert np.max(np.abs(F0 - F0o) / A) < 1e-11
    ref = oracle.vv_run(s.pos, s.vel, s.mass, s.q, s.type, s.mol, params(s), 0, nsteps, s.dt, s.accel, F0o,
                        water=water)
    assert np.max(np.abs(pos - ref["pos"])) < 1e-10 * s.L
    assert rel_err_components(vel, ref["vel"]) < 1e-9
    assert rel_err_components(F, ref["F"]) < 1e-9
    assert np.allclose(tr, ref["trace"], rtol=1e-10, atol=0)


def test_bonded_terms_in_forces():
    s = systems.water(334, seed=6)
    rng = np.random.default_rng(3)
    s.pos = s.pos + rng.normal(0, 0.02, s.pos.shape)
    out = gpu_forces(s, 4, bonds=True)
    ref = oracle.rbe_forces(s.pos, s.q, s.type, s.mol, params(s), 4)
    U, Fb = oracle.water_bonded(s.pos, s.L, s.n_water_mol, *s.bonds)
    ref = dict(ref, F=ref["F"] + Fb, F_abs=ref["F_abs"] + np.abs(Fb))
    assert cond_err(out["F"], ref) < 1e-11
    assert out["E"][rbe.E_BOND] == pytest.approx(U, rel=1e-12)
