"""Energy drift of NVE velocity Verlet on the 12,000-atom water box (4,000
flexible 3-site molecules, seed 4), FP64 and mixed precision, against the
oracle's integrator on identical draws.

The random batches make every step's force an unbiased but noisy estimate,
so an NVE run heats (the paper runs its water with a thermostat); each step's
energy is itself an estimate.  Drift is therefore compared as the slope of a
least-squares line through 100 steps of the kinetic energy (exact at each
step) and of the total-energy estimate, from a state thermalised by Langevin
dynamics (reading R14).  FP64: the GPU trajectory equals the oracle's to
rounding, so the slopes agree to 1e-9.  Mixed: the trajectory departs from the
FP64 one (rounding, then chaos and different list decisions), so its slopes
are compared with the spread of FP64 slopes over independent draws."""
import numpy as np
import pytest

from gpu_util import oracle, params, rbe, systems

pytestmark = pytest.mark.gpu

NEQ = 1000        # Langevin steps before the NVE segments
NSEG = 100        # NVE steps per segment


def _slope(y):
    t = np.arange(len(y), dtype=np.float64)
    return float(np.polyfit(t, y, 1)[0])


@pytest.fixture(scope="module")
def state():
    import torch
    s = systems.water(4000, seed=4)
    dev = lambda a, dt=torch.float64: torch.tensor(a, dtype=dt, device="cuda")
    d = dict(pos=dev(s.pos), vel=dev(s.vel), mass=dev(s.mass), q=dev(s.q), typ=dev(s.type, torch.int32),
             mol=dev(s.mol, torch.int32))
    F = torch.empty_like(d["pos"])
    c = rbe.Context.for_system(s, precision=rbe.MIXED)
    c.set_langevin(systems.KT_WATER, 100.0)
    c.forces(0, d["pos"], d["q"], d["typ"], d["mol"], F)
    c.step(0, NEQ, s.dt, s.accel, d["pos"], d["vel"], d["mass"], d["q"], d["typ"], d["mol"], F)
    assert c.sync_status() == 0
    return s, d["pos"].cpu().numpy(), d["vel"].cpu().numpy()


def _nve(s, P0, V0, precision, seed=None):
    import torch
    dev = lambda a, dt=torch.float64: torch.tensor(a, dtype=dt, device="cuda")
    c = rbe.Context.for_system(s, precision=precision, seed=seed)
    pos, vel = dev(P0), dev(V0)
    q, typ, mol, mass = dev(s.q), dev(s.type, torch.int32), dev(s.mol, torch.int32), dev(s.mass)
    F = torch.empty_like(pos)
    c.forces(NEQ, pos, q, typ, mol, F)
    tr = torch.zeros((NSEG, 2), dtype=torch.float64, device="cuda")
    c.step(NEQ, NSEG, s.dt, s.accel, pos, vel, mass, q, typ, mol, F, tr)
    assert c.sync_status() == 0
    return tr.cpu().numpy()


def test_nve_drift_against_oracle(state):
    s, P0, V0 = state
    pr = params(s)
    r0 = oracle.rbe_forces(P0, s.q, s.type, s.mol, pr, NEQ)
    F0 = r0["F"] + oracle.water_bonded(P0, s.L, s.n_water_mol, *s.bonds)[1]
    ref = oracle.vv_run(P0, V0, s.mass, s.q, s.type, s.mol, pr, NEQ, NSEG, s.dt, s.accel, F0,
                        water=(s.n_water_mol, *s.bonds))["trace"]
    K_o, E_o = ref[:, 1], ref.sum(1)
    f64 = _nve(s, P0, V0, rbe.FP64)
    mix = _nve(s, P0, V0, rbe.MIXED)
    # FP64: the same trajectory as the oracle, step by step
    assert np.max(np.abs(f64[:, 1] - K_o) / K_o) < 1e-10
    assert np.max(np.abs(f64.sum(1) - E_o)) < 1e-10 * K_o.mean()
    sK_o, sE_o = _slope(K_o), _slope(E_o)
    sK_64, sE_64 = _slope(f64[:, 1]), _slope(f64.sum(1))
    assert sK_o > 0 and sE_o > 0                     # the stochastic forces heat the NVE run
    assert abs(sK_64 - sK_o) < 1e-9 * abs(sK_o) and abs(sE_64 - sE_o) < 1e-9 * abs(sE_o)
    # mixed: slopes within the spread of FP64 slopes over independent draws
    spread = [_nve(s, P0, V0, rbe.FP64, seed=100 + k) for k in range(8)]
    sdK = np.std([_slope(t[:, 1]) for t in spread], ddof=1)
    sdE = np.std([_slope(t.sum(1)) for t in spread], ddof=1)
    sK_m, sE_m = _slope(mix[:, 1]), _slope(mix.sum(1))
    print(f"\nNVE slopes over {NSEG} steps (kJ/mol per step): K oracle {sK_o:.2f}, FP64 {sK_64:.2f}, "
          f"mixed {sK_m:.2f} (FP64 spread over draws {sdK:.2f}); E oracle {sE_o:.2f}, FP64 {sE_64:.2f}, "
          f"mixed {sE_m:.2f} (spread {sdE:.2f}); mixed K departs from the oracle by "
          f"{np.max(np.abs(mix[:, 1] - K_o) / K_o):.2e} (max over the segment)")
    assert abs(sK_m - sK_o) < 4 * sdK
    assert abs(sE_m - sE_o) < 4 * sdE


@pytest.mark.slow
def test_water_90k_thousand_fp64_steps_thermostatted():
    """The 90,000-atom water box (30,000 molecules, seed 2) for 1,000 FP64
    velocity-Verlet steps of 1 fs.  Unthermostatted, the stochastic forces heat
    this system until it diverges within that many steps (see the NVE slopes
    above), so the run uses the Langevin thermostat (100 fs): it must finish
    with no status error, finite state and a bounded kinetic temperature."""
    import torch
    s = systems.water(30000, seed=2)
    dev = lambda a, dt=torch.float64: torch.tensor(a, dtype=dt, device="cuda")
    pos, vel, mass, q = dev(s.pos), dev(s.vel), dev(s.mass), dev(s.q)
    typ, mol = dev(s.type, torch.int32), dev(s.mol, torch.int32)
    c = rbe.Context.for_system(s, precision=rbe.FP64)
    c.set_langevin(systems.KT_WATER, 100.0)
    F = torch.empty_like(pos)
    c.forces(0, pos, q, typ, mol, F)
    nsteps = 1000
    tr = torch.zeros((nsteps, 2), dtype=torch.float64, device="cuda")
    c.step(0, nsteps, s.dt, s.accel, pos, vel, mass, q, typ, mol, F, tr)
    assert c.sync_status() == 0
    t = tr.cpu().numpy()
    assert np.isfinite(t).all() and torch.isfinite(pos).all() and torch.isfinite(vel).all()
    kT_kin = t[:, 1] / (1.5 * s.n)
    print(f"\n90k water, 1,000 FP64 steps: kinetic kT {kT_kin[0]:.3f} -> {kT_kin[-1]:.3f} kJ/mol "
          f"(target {systems.KT_WATER})")
    assert kT_kin.max() < 10 * systems.KT_WATER
