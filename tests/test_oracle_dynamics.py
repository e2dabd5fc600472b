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
