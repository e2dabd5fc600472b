"""Pins of the oracle's bonded water terms and velocity-Verlet driver
(Algorithm 1, integration step), CPU only."""
import math

import numpy as np
import pytest

from paper_2204_13595_gb300 import systems


def test_water_bonded_forces_are_minus_gradient(orc):
    w = systems.water(5, seed=3)
    rng = np.random.default_rng(0)
    pos = w.pos + rng.normal(0, 0.05, w.pos.shape)     # off the equilibrium geometry
    kb, r0, kth, th0 = w.bonds
    U, F = orc.water_bonded(pos, w.L, 5, kb, r0, kth, th0)
    h = 1e-6
    for i in range(15):
        for a in range(3):
            pp, pm = pos.copy(), pos.copy()
            pp[i, a] += h
            pm[i, a] -= h
            g = (orc.water_bonded(pp, w.L, 5, kb, r0, kth, th0)[0] - orc.water_bonded(pm, w.L, 5, kb, r0, kth, th0)[0]) / (2 * h)
            assert -g == pytest.approx(F[i, a], rel=1e-6, abs=1e-6 * np.abs(F).max())
    assert np.abs(F.sum(0)).max() < 1e-10 * np.abs(F).max()
    # equilibrium geometry has zero bonded energy and force
    U0, F0 = orc.water_bonded(w.pos, w.L, 5, kb, r0, kth, th0)
    assert U0 < 1e-20 and np.abs(F0).max() < 1e-9


def test_velocity_verlet_energy_and_reversibility(orc):
    """A neutral-free (q = 0, eps = 0) flexible molecule: velocity Verlet keeps
    the energy to O(dt^2) and retraces its path when velocities are reversed."""
    w = systems.water(1, seed=2)
    n, L = 3, 24.0
    rng = np.random.default_rng(4)
    pos = w.pos - w.pos[0] + L / 2 + rng.normal(0, 0.03, (3, 3))
    vel = rng.normal(0, 0.01, (3, 3))
    q = np.zeros(n)
    pr = orc.make_params(L, w.alpha, w.r_c, w.r_s, 20, 4, 1, k_e=w.k_e, eps=(0.0, 0.0), sigma=w.sigma)
    kb, r0, kth, th0 = w.bonds
    U, F0 = orc.water_bonded(pos, L, 1, kb, r0, kth, th0)
    out = orc.vv_run(pos, vel, w.mass, q, w.type, w.mol, pr, 0, 400, 0.2, w.accel, F0, water=(1, kb, r0, kth, th0))
    e = out["trace"].sum(1)
    e0 = U + 0.5 * (w.mass[:, None] * vel * vel).sum() / w.accel
    assert np.abs(e - e0).max() < 2e-3 * abs(e0)
    back = orc.vv_run(out["pos"], -out["vel"], w.mass, q, w.type, w.mol, pr, 0, 400, 0.2, w.accel, out["F"],
                      water=(1, kb, r0, kth, th0))
    assert np.abs(back["pos"] - pos).max() < 1e-9
    assert np.abs(back["vel"] + vel).max() < 1e-9


def _free_particles(n, L, m, seed):
    rng = np.random.default_rng(seed)
    pos = rng.random((n, 3)) * L
    return pos, np.zeros(n), np.zeros(n, dtype=np.int32), np.full(n, m)


def test_langevin_zero_temperature_decay(orc):
    """kT = 0, no interactions: the scheme of R14 gives w_0 = (1 - a) v_0 and
    w_k = (1 - 2a) w_{k-1} for the half-step velocities, so
    v_n = (1 - a)^2 (1 - 2a)^(n - 1) v_0 with a = dt / (2 tau)."""
    n, L, dt, tau, accel = 64, 40.0, 0.01, 0.25, 0.7
    pos, q, typ, mass = _free_particles(n, L, 2.5, 1)
    vel = np.random.default_rng(2).normal(size=(n, 3))
    pr = orc.make_params(L, 0.05, 3.0, 6.0, 10, 1, 5, eps=(0.0,), sigma=(1.0,), lang_kT=0.0, lang_tau=tau)
    F0 = np.zeros((n, 3))
    a = dt / (2 * tau)
    for nsteps in (1, 5, 30):
        out = orc.vv_run(pos, vel, mass, q, typ, None, pr, 0, nsteps, dt, accel, F0)
        pred = (1 - a) ** 2 * (1 - 2 * a) ** (nsteps - 1) * vel
        assert np.allclose(out["vel"], pred, rtol=1e-12, atol=0)


def test_langevin_velocity_variance_closed_form(orc):
    """Free particles from rest under R14: with eta of variance
    s2 = 2 accel kT / (m tau dt), Var w_0 = dt^2 s2 / 4,
    Var w_k = (1 - 2a)^2 Var w_{k-1} + dt^2 s2, and
    Var v_n = (1 - a)^2 Var w_{n-1} + dt^2 s2 / 4, which tends to accel kT / m
    (equipartition).  Checked per mass class at a transient and a late step."""
    n, L, dt, tau, accel, kT = 20000, 400.0, 0.01, 0.05, 1.0, 1.7
    pos, q, typ, _ = _free_particles(n, L, 1.0, 3)
    mass = np.where(np.arange(n) % 2 == 0, 1.0, 4.0)
    vel = np.zeros((n, 3))
    pr = orc.make_params(L, 0.05, 3.0, 6.0, 10, 1, 9, eps=(0.0,), sigma=(1.0,), lang_kT=kT, lang_tau=tau)
    a = dt / (2 * tau)
    for nsteps in (3, 40):
        out = orc.vv_run(pos, vel, mass, q, typ, None, pr, 0, nsteps, dt, accel, np.zeros((n, 3)))
        for m in (1.0, 4.0):
            s2 = 2 * accel * kT / (m * tau * dt)
            vw = dt * dt * s2 / 4
            for _ in range(nsteps - 1):
                vw = (1 - 2 * a) ** 2 * vw + dt * dt * s2
            pred = (1 - a) ** 2 * vw + dt * dt * s2 / 4
            v = out["vel"][mass == m]
            emp = float((v * v).mean())
            rel_sd = math.sqrt(2.0 / v.size)
            assert abs(emp / pred - 1) < 5 * rel_sd, (nsteps, m, emp, pred)
            assert abs(float(v.mean())) < 5 * math.sqrt(pred / v.size)
        if nsteps == 40:
            for m in (1.0, 4.0):
                v = out["vel"][mass == m]
                assert float((v * v).mean()) == pytest.approx(accel * kT / m, rel=5 * math.sqrt(2.0 / v.size))
