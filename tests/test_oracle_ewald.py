"""Pins of the oracle's exact Ewald / LJ reference (Eqs. (2.1)-(2.5)), CPU only."""
import json
import math
import os

import numpy as np
import pytest

from paper_2204_13595_gb300 import systems

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "pins.json")))


def _kmax(alpha, L, tail=46.0):
    return int(math.ceil(math.sqrt(tail * alpha * L * L) / math.pi)) + 1


def _coul(E):
    return E[0] + E[1] + E[2] + E[4]


def test_madelung_nacl(orc):
    """Rock salt: U = -N M q^2 / (2 r0) with M = 1.747564594633 (Eq. (2.1) lattice sum)."""
    pos, q, L = systems.nacl_crystal(2, 1.0)
    n = len(q)
    pr = orc.make_params(L, 1.2, 0.5, 1.9, 10, 10, 1, k_e=1.0)
    r = orc.ewald_exact(pos, q, np.zeros(n, np.int32), None, pr, 4.5, _kmax(1.2, L))
    M = -2.0 * _coul(r["E"]) / n
    assert M == pytest.approx(GOLD["madelung_nacl"]["value"], rel=1e-10)
    assert np.abs(r["F"]).max() < 1e-12          # every ion sits at an inversion centre


def _random_neutral(rng, n, L, dmin=0.8):
    pos = systems._rsa(rng, n, L, dmin)
    q = np.where(np.arange(n) % 2 == 0, 1.0, -1.0) * rng.uniform(0.5, 1.5, n)
    q -= q.mean()
    return pos, q


def _small_water(n_mol, seed):
    w = systems.water(n_mol, seed=seed)
    return w


@pytest.mark.parametrize("kind", ["ions", "water"])
def test_alpha_invariance(orc, kind):
    """The converged Ewald total does not depend on alpha (Eq. (2.2) is an identity)."""
    if kind == "ions":
        rng = np.random.default_rng(3)
        L = 8.0
        pos, q = _random_neutral(rng, 24, L)
        typ, mol = np.zeros(24, np.int32), None
    else:
        w = _small_water(8, 4)
        L, pos, q, typ, mol = w.L, w.pos, w.q, w.type, w.mol
    out = []
    for a_scale, rcut in [(1.0, 1.2 * L), (2.0, 0.9 * L)]:
        alpha = a_scale * (5.2 / (1.2 * L)) ** 2
        pr = orc.make_params(L, alpha, 0.2 * L, 0.45 * L, 4, 4, 1, k_e=1.0)
        r = orc.ewald_exact(pos, q, typ, mol, pr, rcut, _kmax(alpha, L))
        out.append(r)
    assert _coul(out[0]["E"]) == pytest.approx(_coul(out[1]["E"]), rel=1e-10, abs=1e-10)
    F0, F1 = out[0]["F"], out[1]["F"]
    assert np.abs(F0 - F1).max() < 1e-8 * np.abs(F0).max()


def test_direct_lattice_sum(orc):
    """Eq. (2.1) summed directly over cubic shells of images converges to the
    Ewald value for a neutral, dipole-free cell."""
    rng = np.random.default_rng(9)
    L = 6.0
    d = rng.uniform(-1.6, 1.6, (3, 3))
    qs = np.array([1.0, -0.6, -0.4])
    # inversion-symmetric about the centre: zero net dipole
    pos = np.concatenate([L / 2 + d, L / 2 - d])
    q = np.concatenate([qs, qs])
    alpha = (5.0 / (0.9 * L)) ** 2
    pr = orc.make_params(L, alpha, 0.5, 2.9, 4, 4, 1, k_e=1.0)
    r = orc.ewald_exact(pos, q, np.zeros(6, np.int32), None, pr, 1.5 * L, _kmax(alpha, L))
    ew = _coul(r["E"])
    errs = [abs(orc.direct_coulomb(pos, q, L, 1.0, ns) - ew) for ns in (4, 8, 16)]
    assert errs[2] < 2e-4 * abs(ew)
    assert errs[2] < errs[1] < errs[0]          # converging, not merely close


def _energy_total(orc, pos, q, typ, mol, pr, rcut, kmax):
    return orc.ewald_exact(pos, q, typ, mol, pr, rcut, kmax)["E"].sum()


@pytest.mark.parametrize("kind", ["ions", "water"])
def test_exact_forces_are_minus_gradient(orc, kind):
    """F_i = -dU/dr_i by central differences (Eq. (2.5) vs Eq. (2.3))."""
    if kind == "ions":
        rng = np.random.default_rng(21)
        L = 7.0
        pos, q = _random_neutral(rng, 16, L, dmin=0.9)
        typ, mol = np.zeros(16, np.int32), None
        eps, sig = (1.0,), (0.8,)
    else:
        w = _small_water(6, 8)
        L, pos, q, typ, mol = w.L, w.pos, w.q, w.type, w.mol
        eps, sig = w.eps, w.sigma
    alpha = (4.5 / (0.45 * L)) ** 2
    pr = orc.make_params(L, alpha, 0.2 * L, 0.45 * L, 4, 4, 1, k_e=1.0, eps=eps, sigma=sig)
    rcut, km = 0.45 * L, _kmax(alpha, L)
    F = orc.ewald_exact(pos, q, typ, mol, pr, rcut, km)["F"]
    h = 1e-5
    rng = np.random.default_rng(1)
    for i in rng.choice(len(q), 4, replace=False):
        for a in range(3):
            pp, pm = pos.copy(), pos.copy()
            pp[i, a] += h
            pm[i, a] -= h
            g = (_energy_total(orc, pp, q, typ, mol, pr, rcut, km) - _energy_total(orc, pm, q, typ, mol, pr, rcut, km)) / (2 * h)
            assert -g == pytest.approx(F[i, a], rel=1e-6, abs=1e-6 * np.abs(F).max())


def test_virial_trace_is_scaling_derivative(orc):
    """tr W = -dU/dlambda for r -> lambda r, L -> lambda L (cutoffs scaled too),
    and for pure Coulomb tr W = U (Euler's relation for a degree -1 potential)."""
    rng = np.random.default_rng(5)
    L = 8.0
    pos, q = _random_neutral(rng, 20, L, dmin=0.9)
    typ = np.zeros(20, np.int32)
    alpha = (5.2 / (0.49 * L)) ** 2

    def U(lam, eps):
        pr = orc.make_params(lam * L, alpha / lam**2, 0.2 * lam * L, 0.49 * lam * L, 4, 4, 1,
                             k_e=1.0, eps=(eps,), sigma=(0.9,))
        return orc.ewald_exact(lam * pos, q, typ, None, pr, 0.49 * lam * L, _kmax(alpha, L))

    for eps in (0.0, 1.0):
        r = U(1.0, eps)
        h = 1e-6
        dU = (U(1 + h, eps)["E"].sum() - U(1 - h, eps)["E"].sum()) / (2 * h)
        assert r["W"][:3].sum() == pytest.approx(-dU, rel=1e-7)
        if eps == 0.0:
            assert r["W"][:3].sum() == pytest.approx(_coul(r["E"]), rel=1e-8)


def test_two_particle_closed_forms(orc):
    """Isolated pair: LJ 4 eps[(s/r)^12-(s/r)^6] and its force; real-space
    Ewald u = q1 q2 erfc(sqrt(a) r)/r with the force of Eq. (2.10)."""
    L, r = 30.0, 1.13
    pos = np.array([[10.0, 10.0, 10.0], [10.0 + r / math.sqrt(3), 10.0 + r / math.sqrt(3), 10.0 + r / math.sqrt(3)]])
    typ = np.zeros(2, np.int32)
    pr = orc.make_params(L, 1.0, 2.0, 4.0, 1, 1, 1, k_e=1.0, eps=(0.7,), sigma=(1.05,))
    # a pair closer than r_c is in the core: p >= N_S makes the estimator exact
    out = orc.rbe_forces(pos, np.zeros(2), typ, None, pr, 0)
    sr6 = (1.05 / r) ** 6
    assert out["E"][3] == pytest.approx(4 * 0.7 * (sr6 * sr6 - sr6), rel=1e-14)
    fmag = 24 * 0.7 * (2 * sr6 * sr6 - sr6) / r       # along r_1 - r_2 on atom 1
    unit = (pos[0] - pos[1]) / r
    assert np.allclose(out["F_real"][0], fmag * unit, rtol=1e-13, atol=0)
    q = np.array([0.7, -1.3])
    out = orc.rbe_forces(pos, q, typ, None, orc.make_params(L, 1.0, 2.0, 4.0, 1, 1, 1, k_e=1.0), 0)
    sa = 1.0
    u = 0.7 * -1.3 * math.erfc(sa * r) / r
    dudr = 0.7 * -1.3 * (-math.erfc(sa * r) / r**2 - 2 * sa / math.sqrt(math.pi) * math.exp(-r * r) / r)
    assert out["E"][0] == pytest.approx(u, rel=1e-14)
    assert np.allclose(out["F_real"][0], -dudr * unit, rtol=1e-13, atol=0)
