"""Langevin thermostat (reading R14) on the GPU: the zero-temperature closed
form, trajectory parity with the oracle, batched = looped bit for bit, and
physical checks on the paper's 1:1 primitive-model electrolyte (Sec. 3.1:
5,120 ions at 0.01 sigma^-3, L = 80 sigma, WCA soft spheres, r_eta = 5 sigma,
r_c = 15 sigma, shell batch 10, alpha = 0.03, Fourier batch 100, dt = 0.002,
relaxation time 1): equipartition, and the mean potential energy per atom of
the IRBE against larger batches (the comparison of Table 1)."""
import math

import numpy as np
import pytest

from gpu_util import oracle, rbe, rel_err_components, systems

pytestmark = pytest.mark.gpu

WCA = 2.0 ** (1.0 / 6.0)


def _dev(s):
    import torch
    t = lambda a, dt=torch.float64: torch.tensor(a, dtype=dt, device="cuda")
    return dict(pos=t(s.pos), vel=t(s.vel), mass=t(s.mass), q=t(s.q), typ=t(s.type, torch.int32),
                mol=None if s.mol is None else t(s.mol, torch.int32),
                F=torch.zeros((s.n, 3), dtype=torch.float64, device="cuda"))


def test_zero_temperature_decay_closed_form():
    """Free particles at kT = 0: v_n = (1 - a)^2 (1 - 2a)^(n-1) v_0, a = dt/(2 tau)."""
    import torch
    n, L, dt, tau, accel = 300, 40.0, 0.01, 0.25, 0.7
    rng = np.random.default_rng(1)
    pos = torch.tensor(rng.random((n, 3)) * L, device="cuda")
    v0 = rng.normal(size=(n, 3))
    vel = torch.tensor(v0, device="cuda")
    mass = torch.full((n,), 2.5, dtype=torch.float64, device="cuda")
    q = torch.zeros(n, dtype=torch.float64, device="cuda")
    F = torch.zeros((n, 3), dtype=torch.float64, device="cuda")
    ctx = rbe.Context(L, 0.05, 3.0, 6.0, 10, 1, 5, eps=(0.0,), sigma=(1.0,))
    ctx.set_langevin(0.0, tau)
    nsteps = 30
    ctx.step(0, nsteps, dt, accel, pos, vel, mass, q, None, None, F)
    assert ctx.sync_status() == 0
    a = dt / (2 * tau)
    pred = (1 - a) ** 2 * (1 - 2 * a) ** (nsteps - 1) * v0
    assert np.allclose(vel.cpu().numpy(), pred, rtol=1e-12, atol=0)


def test_langevin_trajectory_matches_oracle():
    """20 thermostatted steps of the WCA electrolyte against the oracle's
    integrator on the same draws (forces differ by rounding only)."""
    import torch
    s = systems.electrolyte()
    kT, tau = 1.0, 0.5
    pr = oracle.make_params(s.L, s.alpha, s.r_c, s.r_s, s.p, s.P, s.seed, k_e=s.k_e, eps=s.eps, sigma=s.sigma,
                            shift_lj=1, lj_rc_factor=WCA, lang_kT=kT, lang_tau=tau)
    ctx = rbe.Context(s.L, s.alpha, s.r_c, s.r_s, s.p, s.P, s.seed, k_e=s.k_e, eps=s.eps, sigma=s.sigma,
                      shift_lj=True)
    ctx.set_lj_cutoff(WCA)
    ctx.set_langevin(kT, tau)
    d = _dev(s)
    ctx.forces(0, d["pos"], d["q"], d["typ"], None, d["F"])
    F0 = d["F"].cpu().numpy()
    nsteps = 20
    tr = torch.zeros((nsteps, 2), dtype=torch.float64, device="cuda")
    ctx.step(0, nsteps, s.dt, s.accel, d["pos"], d["vel"], d["mass"], d["q"], d["typ"], None, d["F"], tr)
    assert ctx.sync_status() == 0
    r0 = oracle.rbe_forces(s.pos, s.q, s.type, None, pr, 0)
    F0o = r0["F"]
    assert np.max(np.abs(F0 - F0o) / r0["F_abs"]) < 1e-11
    ref = oracle.vv_run(s.pos, s.vel, s.mass, s.q, s.type, None, pr, 0, nsteps, s.dt, s.accel, F0o)
    assert np.max(np.abs(d["pos"].cpu().numpy() - ref["pos"])) < 1e-10 * s.L
    assert rel_err_components(d["vel"].cpu().numpy(), ref["vel"]) < 1e-9
    assert np.allclose(tr.cpu().numpy(), ref["trace"], rtol=1e-10, atol=0)
    # the thermostat acted: the NVE run from the same state differs
    nve = oracle.make_params(s.L, s.alpha, s.r_c, s.r_s, s.p, s.P, s.seed, k_e=s.k_e, eps=s.eps, sigma=s.sigma,
                             shift_lj=1, lj_rc_factor=WCA)
    ref_nve = oracle.vv_run(s.pos, s.vel, s.mass, s.q, s.type, None, nve, 0, nsteps, s.dt, s.accel, F0o)
    assert np.max(np.abs(ref_nve["vel"] - ref["vel"])) > 1e-3


def test_batched_langevin_equals_looped():
    import torch
    suite = systems.batch_replicas(nrep=4, n_min=1000, n_max=3000, seed0=700)
    ctxs = [rbe.Context.for_system(s, precision=rbe.MIXED) for s in suite]
    for r, (s, c) in enumerate(zip(suite, ctxs)):
        if r != 1:
            c.set_langevin(1.0 if s.name == "electrolyte" else systems.KT_WATER, 0.5 if s.name == "electrolyte" else 100.0)
    A = [_dev(s) for s in suite]
    B = [{k: (None if v is None else v.clone()) for k, v in d.items()} for d in A]
    b = rbe.Batch(ctxs)
    b.bind([d["pos"] for d in A], [d["q"] for d in A], [d["typ"] for d in A], [d["mol"] for d in A],
           [d["F"] for d in A], vel=[d["vel"] for d in A], mass=[d["mass"] for d in A],
           dt=[s.dt for s in suite], accel=[s.accel for s in suite])
    assert b.info()["launches_per_step"] == 19
    b.forces(0)
    b.step(0, 8)
    assert b.sync_status()[0] == 0
    for s, c, d, a in zip(suite, ctxs, B, A):
        c.forces(0, d["pos"], d["q"], d["typ"], d["mol"], d["F"])
        c.step(0, 8, s.dt, s.accel, d["pos"], d["vel"], d["mass"], d["q"], d["typ"], d["mol"], d["F"])
        for k in ("pos", "vel", "F"):
            assert torch.equal(a[k], d[k]), k


def _paper_electrolyte(seed=21):
    """Sec. 3.1's 1:1 system: 2,560 + 2,560 ions, L = 80 sigma."""
    return systems.electrolyte(n=5120, L=80.0, seed=seed, r_c=5.0, r_s=15.0, p=10, P=100, dt=0.002)


def _paper_electrolyte_2to1(seed=22):
    """Sec. 3.1's 2:1 system: 1,280 divalent cations and 2,560 monovalent
    anions, L = 80 sigma."""
    return systems.electrolyte_2to1(n_cations=1280, L=80.0, seed=seed, r_c=5.0, r_s=15.0, p=10, P=100, dt=0.002)


def _langevin_run(s, p, P, nsteps, nequil, seed, kT=1.0, tau=1.0, every=100):
    """Potential energy per atom and the kinetic temperature 2 KE / (3 N),
    sampled every `every` steps after `nequil` steps."""
    import torch
    ctx = rbe.Context(s.L, 0.03, s.r_c, s.r_s, p, P, seed, k_e=s.k_e, eps=s.eps, sigma=s.sigma, shift_lj=True,
                      precision=rbe.MIXED)
    ctx.set_lj_cutoff(WCA)
    ctx.set_langevin(kT, tau)
    d = _dev(s)
    ctx.forces(0, d["pos"], d["q"], d["typ"], None, d["F"])
    ctx.step(0, nequil, s.dt, s.accel, d["pos"], d["vel"], d["mass"], d["q"], d["typ"], None, d["F"])
    tr = torch.zeros((nsteps, 2), dtype=torch.float64, device="cuda")
    ctx.step(nequil, nsteps, s.dt, s.accel, d["pos"], d["vel"], d["mass"], d["q"], d["typ"], None, d["F"], tr)
    assert ctx.sync_status() == 0
    t = tr.cpu().numpy()[every - 1::every]
    return t[:, 0] / s.n, t[:, 1] / (1.5 * s.n)


def _mean_se(x, block=10):
    nb = len(x) // block
    bm = x[:nb * block].reshape(nb, block).mean(1)
    return float(x.mean()), float(bm.std(ddof=1) / math.sqrt(nb))


def test_equipartition_paper_electrolyte():
    """Kinetic energy per degree of freedom relaxes to kT/2 under the
    thermostat, with the IRBE forces (p = 10, P = 100) and their noise."""
    s = _paper_electrolyte()
    _, t_kin = _langevin_run(s, 10, 100, nsteps=6000, nequil=4000, seed=3, every=20)
    m, se = _mean_se(t_kin)
    assert abs(m - 1.0) < max(4 * se, 0.01), (m, se)


@pytest.mark.slow
def test_energy_per_atom_irbe_against_large_batches():
    """The comparison of Table 1: mean potential energy per atom of the 1:1
    electrolyte under Langevin dynamics with the IRBE batches (10, 100) equals
    that with batches large enough to be nearly exact (every shell atom,
    2,000 k vectors) within the statistical error."""
    s = _paper_electrolyte()
    e_irbe, _ = _langevin_run(s, 10, 100, nsteps=60000, nequil=20000, seed=5)
    e_ref, _ = _langevin_run(s, 512, 2000, nsteps=60000, nequil=20000, seed=6)   # p >= N_S (~136)
    mi, si = _mean_se(e_irbe)
    mr, sr = _mean_se(e_ref)
    print(f"\nU/N IRBE {mi:.5f} +- {si:.5f} (std {e_irbe.std():.5f}); "
          f"large batches {mr:.5f} +- {sr:.5f} (std {e_ref.std():.5f})")
    assert abs(mi - mr) < 4 * math.hypot(si, sr) + 1e-3 * abs(mr)
    assert mi < 0 and mr < 0


def test_equipartition_paper_electrolyte_2to1():
    """The same relaxation of the kinetic temperature for the 2:1 system."""
    s = _paper_electrolyte_2to1()
    _, t_kin = _langevin_run(s, 10, 100, nsteps=6000, nequil=4000, seed=4, every=20)
    m, se = _mean_se(t_kin)
    assert abs(m - 1.0) < max(4 * se, 0.01), (m, se)


@pytest.mark.slow
def test_energy_per_atom_2to1_irbe_against_large_batches():
    """Table 1's 2:1 row: mean potential energy per atom under Langevin
    dynamics with the IRBE batches (10, 100) against batches large enough to
    be nearly exact (every shell atom, 2,000 k vectors)."""
    s = _paper_electrolyte_2to1()
    e_irbe, _ = _langevin_run(s, 10, 100, nsteps=60000, nequil=20000, seed=7)
    e_ref, _ = _langevin_run(s, 512, 2000, nsteps=60000, nequil=20000, seed=8)
    mi, si = _mean_se(e_irbe)
    mr, sr = _mean_se(e_ref)
    print(f"\n2:1 U/N IRBE {mi:.5f} +- {si:.5f} (std {e_irbe.std():.5f}); "
          f"large batches {mr:.5f} +- {sr:.5f} (std {e_ref.std():.5f})")
    assert abs(mi - mr) < 4 * math.hypot(si, sr) + 1e-3 * abs(mr)
    assert mi < 0 and mr < 0
