"""Pins of the oracle's IRBE estimator (Eqs. (2.9)-(2.14), Algorithm 1), CPU only.

Special cases that reduce to the exact sums, invariants, finite differences
with frozen draws, and unbiasedness / variance over seeds.
"""
import json
import math
import os

import numpy as np
import pytest

from paper_2204_13595_gb300 import systems

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "pins.json")))


def _params(orc, s, p=None, P=None, seed=1, **kw):
    return orc.make_params(s.L, kw.get("alpha", s.alpha), kw.get("r_c", s.r_c), kw.get("r_s", s.r_s),
                           s.p if p is None else p, s.P if P is None else P, seed,
                           k_e=s.k_e, eps=s.eps, sigma=s.sigma)


@pytest.fixture(scope="module")
def elec():
    return systems.electrolyte()


@pytest.fixture(scope="module")
def wat():
    return systems.water(334, seed=6)       # 1002 atoms, L = 21.5 A: the stencil wraps


def test_cell_stencil_equals_brute_force(orc, elec, wat):
    """Canonical-order lists from the Sec. 2.3 stencil equal the all-pairs scan."""
    for s, cap in ((elec, 64), (wat, 160)):
        pr = _params(orc, s)
        a = orc.lists(s.pos, pr, 3, brute=True, cap_core=cap, cap_shell=600)
        b = orc.lists(s.pos, pr, 3, brute=False, cap_core=cap, cap_shell=600)
        assert a["status"] == 0 and b["status"] == 0
        for k in ("n_core", "n_shell", "n_batch", "core", "batch", "shell"):
            assert (a[k] == b[k]).all(), k


def test_lists_membership_and_batches(orc, elec):
    """C(i) = {r <= r_c}, S(i) = {r_c < r <= r_s} (Sec. 2.3) checked against
    plain FP64 distances away from the boundaries; B(i) is a subset of S(i)
    of size min(p, N_S) without repeats (Algorithm 1, shell step)."""
    s = elec
    pr = _params(orc, s)
    out = orc.lists(s.pos, pr, 0, cap_core=64, cap_shell=400)
    d = s.pos[None, :, :] - s.pos[:, None, :]
    d -= s.L * np.round(d / s.L)
    r = np.sqrt((d * d).sum(-1))
    np.fill_diagonal(r, np.inf)
    margin = 1e-7
    for i in range(0, s.n, 37):
        core = set(out["core"][i, :out["n_core"][i]].tolist())
        shell = set(out["shell"][i, :out["n_shell"][i]].tolist())
        clear_core = set(np.nonzero(r[i] <= s.r_c - margin)[0].tolist())
        clear_shell = set(np.nonzero((r[i] > s.r_c + margin) & (r[i] <= s.r_s - margin))[0].tolist())
        assert clear_core <= core and clear_shell <= shell
        assert core.isdisjoint(shell) and i not in core and i not in shell
        assert all(r[i, j] <= s.r_c + margin for j in core)
        assert all(s.r_c - margin < r[i, j] <= s.r_s + margin for j in shell)
        b = out["batch"][i, :out["n_batch"][i]].tolist()
        assert len(b) == min(s.p, len(shell)) and len(set(b)) == len(b) and set(b) <= shell


def test_neighbour_counts_match_density_and_paper(orc):
    """Mean |C|+|S| = 4/3 pi r_s^3 rho: ~140 for the paper's electrolyte at
    15 sigma (Sec. 3.1), ~700 for water at 1.2 nm (Sec. 2.1)."""
    g = GOLD
    e = systems.electrolyte(n=g["electrolyte_paper"]["n_ions"], L=g["electrolyte_paper"]["L"], seed=12,
                            r_c=5.0, r_s=15.0)
    pr = _params(orc, e)
    out = orc.lists(e.pos, pr, 0, cap_core=0)
    tot = (out["n_core"] + out["n_shell"]).mean()
    rho = e.n / e.L**3
    assert tot == pytest.approx(4 / 3 * math.pi * 15.0**3 * rho, rel=0.02)
    assert tot == pytest.approx(g["neighbours_electrolyte_15sigma"]["value"], rel=0.05)
    assert out["n_core"].mean() == pytest.approx(4 / 3 * math.pi * 5.0**3 * rho, rel=0.05)
    w = systems.water(1000, seed=13, r_c=6.0, r_s=12.0)
    pr = _params(orc, w)
    out = orc.lists(w.pos, pr, 0, cap_core=0)
    tot = (out["n_core"] + out["n_shell"]).mean()
    assert tot == pytest.approx(4 / 3 * math.pi * 12.0**3 * w.n / w.L**3, rel=0.02)
    assert tot == pytest.approx(g["neighbours_water_12A"]["value"], rel=0.05)


def test_rbl_reduces_to_truncated_sum_when_p_covers_shell(orc, elec, wat):
    """p >= max N_S: B(i) = S(i) with weight 1, so the real-space estimate is
    the plain truncated erfc + LJ sum (Eq. (2.11) with N_S/p -> 1)."""
    for s in (elec, wat):
        pr = _params(orc, s, p=2000)
        est = orc.rbe_forces(s.pos, s.q, s.type, s.mol, pr, 5)
        ex = orc.ewald_exact(s.pos, s.q, s.type, s.mol, pr, s.r_s, 0)   # kmax 0: real space only
        scale = np.abs(ex["F"]).max()
        assert np.abs(est["F_real"] - ex["F"]).max() < 1e-12 * scale
        for k in (0, 3, 4):
            assert est["E"][k] == pytest.approx(ex["E"][k], rel=1e-12, abs=1e-12 * np.abs(ex["E"]).max())
        # virial: the estimator's W less its reweighted reciprocal part (the
        # textbook Ewald reciprocal virial of each drawn k, weight S/P) is the
        # real-space virial -1/2 sum r_ij (x) f_ij, which must equal the
        # exact truncated real-space virial of the separate Ewald code
        k = 2 * np.pi * est["m"] / s.L
        k2 = (k * k).sum(1)
        e = 0.5 * (orc.S(s.alpha, s.L) / s.P) * 4 * np.pi * s.k_e / (s.L**3 * k2) * np.abs(est["rho"]) ** 2
        b = 2 * (1 / k2 + 1 / (4 * s.alpha))
        Wk = [np.sum(e * ((a == c) - b * k[:, a] * k[:, c])) for a, c in ((0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2))]
        assert np.sum(e) == pytest.approx(est["E"][1], rel=1e-12)
        assert np.abs(est["W"] - np.array(Wk) - ex["W"]).max() < 1e-12 * np.abs(ex["W"]).max()
        assert np.abs(est["corr"]).max() < 1e-12 * scale      # Newton's third law


def test_momentum_invariants(orc, wat):
    """sum_i F_i = 0 after Eq. (2.13); sum_i F_i^{long,*} = 0 exactly in
    exact arithmetic (sum_i q_i e^{-ik.r_i} rho(k) = |rho|^2 is real)."""
    s = wat
    out = orc.rbe_forces(s.pos, s.q, s.type, s.mol, _params(orc, s), 9)
    scale = np.abs(out["F"]).max() * s.n
    assert np.abs(out["F"].sum(0)).max() < 1e-13 * scale
    assert np.abs(out["F_long"].sum(0)).max() < 1e-13 * np.abs(out["F_long"]).max() * s.n
    assert np.allclose(out["corr"], out["F_real"].mean(0), rtol=0, atol=1e-14 * scale)


def test_rbe_force_is_gradient_of_rbe_energy(orc, wat):
    """With the k samples frozen by (seed, step), F^{long,*} = -grad E_k^*
    (Eq. (2.9) differentiates the reweighted U^long of Eq. (2.3))."""
    s = wat
    pr = _params(orc, s, P=50)
    base = orc.rbe_forces(s.pos, s.q, s.type, s.mol, pr, 4)
    h = 1e-5
    for i in (0, 1, 500, 1001):
        for a in range(3):
            pp, pm = s.pos.copy(), s.pos.copy()
            pp[i, a] += h
            pm[i, a] -= h
            ep = orc.rbe_forces(pp, s.q, s.type, s.mol, pr, 4)["E"][1]
            em = orc.rbe_forces(pm, s.q, s.type, s.mol, pr, 4)["E"][1]
            assert -(ep - em) / (2 * h) == pytest.approx(base["F_long"][i, a], rel=1e-6,
                                                          abs=1e-7 * np.abs(base["F_long"]).max())


def test_rho_is_structure_factor(orc, elec):
    """rho(k) of Eq. (2.4) against a direct complex sum written with numpy."""
    s = elec
    m = orc.sample_k(1, 0, 16, s.alpha, s.L)
    r = orc.rho(s.pos, s.q, s.L, m)
    k = 2 * np.pi * m / s.L
    ref = (s.q[None, :] * np.exp(1j * (k @ s.pos.T))).sum(1)
    assert np.allclose(r, ref, rtol=0, atol=1e-11 * np.abs(s.q).sum())


def _exact_target(orc, s):
    """Expectation of the estimator: real space truncated at r_s, full k space."""
    pr = _params(orc, s)
    kmax = int(math.ceil(math.sqrt(46.0 * s.alpha * s.L**2) / math.pi)) + 1
    return orc.ewald_exact(s.pos, s.q, s.type, s.mol, pr, s.r_s, kmax)


def _z_stats(samples, target):
    mean = samples.mean(0)
    se = samples.std(0, ddof=1) / math.sqrt(samples.shape[0])
    z = ((mean - target) / se).ravel()
    return z


def _unbiased(orc, s, nseeds):
    tgt = _exact_target(orc, s)
    real_tgt = orc.ewald_exact(s.pos, s.q, s.type, s.mol, _params(orc, s), s.r_s, 0)["F"]
    Fs = np.empty((nseeds, s.n, 3))
    Fr = np.empty((nseeds, s.n, 3))
    Es = np.empty(nseeds)
    Ws = np.empty((nseeds, 6))
    for k in range(nseeds):
        out = orc.rbe_forces(s.pos, s.q, s.type, s.mol, _params(orc, s, seed=1000 + k), 0)
        Fs[k] = out["F"]
        Fr[k] = out["F_real"] - out["corr"]
        Es[k] = out["E"].sum()
        Ws[k] = out["W"]
    # Total force.  The Fourier part of every atom is driven by the same P
    # k samples, so the components' z-scores are strongly correlated: only
    # per-component bounds (Bonferroni max, |z|>3 fraction) are tested here.
    z = _z_stats(Fs, tgt["F"])
    assert np.abs(z).max() < 5.5
    assert np.mean(np.abs(z) > 3) < 0.01
    assert 0.5 < np.mean(z * z) < 1.5
    # Real-space part (Eqs. (2.11)-(2.13)): shell batches are independent per
    # atom, so the mean of z^2 is also held to its sampling band.
    z = _z_stats(Fr, real_tgt)
    m = z.size
    assert abs(np.mean(z * z) - 1.0) < 4 * math.sqrt(2.0 / m) + 0.02
    assert np.abs(z).max() < 5.5
    assert np.mean(np.abs(z) > 3) < 0.006
    ze = (Es.mean() - tgt["E"].sum()) / (Es.std(ddof=1) / math.sqrt(nseeds))
    assert abs(ze) < 4.0
    # the reweighted virial is unbiased for the exact (truncated real + full
    # reciprocal) Ewald virial, whose trace is pinned by the scaling test
    zw = (Ws.mean(0) - tgt["W"]) / (Ws.std(0, ddof=1) / math.sqrt(nseeds))
    assert np.abs(zw).max() < 4.5


def test_unbiased_electrolyte_2000_seeds(orc, elec):
    """E[F^{tot,*}] = F^tot (Sec. 2.4): 2,000 seeds on the 2,000-ion electrolyte."""
    _unbiased(orc, elec, 2000)


@pytest.mark.slow
def test_unbiased_electrolyte_10k_seeds(orc, elec):
    _unbiased(orc, elec, 10000)


def test_shell_variance_closed_form(orc, elec):
    """Var of the shell estimator (N_S/p) sum_B f_ij for sampling without
    replacement: N_S^2 sigma^2 / p * (N_S - p)/(N_S - 1), sigma^2 the population
    variance of f_ij over S(i); this is the (N_S - p)/p factor of Eq. (2.16)."""
    s = elec
    pr = _params(orc, s, P=1)
    atoms = [3, 400, 1234]
    lists = orc.lists(s.pos, pr, 0, cap_core=64, cap_shell=400)
    samples = np.array([orc.rbe_forces(s.pos, s.q, s.type, None, _params(orc, s, P=1, seed=5000 + k), 0)["F_real"][atoms]
                        for k in range(3000)])
    # population of pair forces over S(i), from the p >= N_S estimator with only j present
    for n_a, i in enumerate(atoms):
        ns = lists["n_shell"][i]
        shell = lists["shell"][i, :ns]
        core = lists["core"][i, :lists["n_core"][i]]
        d = s.pos[shell] - s.pos[i]
        d -= s.L * np.round(d / s.L)
        r = np.sqrt((d * d).sum(1))
        sa = math.sqrt(s.alpha)
        qq = s.k_e * s.q[i] * s.q[shell]
        from scipy.special import erfc
        sr6 = (1.0 / r) ** 6
        scal = -qq * (erfc(sa * r) / r**2 + 2 * sa / math.sqrt(math.pi) * np.exp(-s.alpha * r * r) / r) / r \
            - (48 * sr6 * sr6 - 24 * sr6) / r**2
        f = scal[:, None] * d
        var_pop = f.var(0)
        p = s.p
        pred = ns**2 * var_pop / p * (ns - p) / (ns - 1)
        emp = samples[:, n_a, :].var(0, ddof=1)
        # chi^2 with 2999 dof: relative sd of a variance estimate ~ sqrt(2/3000)=2.6%
        assert np.allclose(emp, pred, rtol=0.15), (emp, pred)
        assert ns > p and len(core) > 0


def test_fourier_variance_scales_as_one_over_P(orc, wat):
    """Var F^{long,*} is proportional to 1/P (Eq. (2.15))."""
    s = wat
    v = []
    for P in (20, 80):
        F = np.array([orc.rbe_forces(s.pos, s.q, s.type, s.mol, _params(orc, s, P=P, seed=70 + k), 0)["F_long"]
                      for k in range(300)])
        v.append(F.var(0, ddof=1).mean())
    assert v[0] / v[1] == pytest.approx(4.0, rel=0.12)


def test_fourier_variance_closed_form(orc):
    """Exact finite-sample variance of the RBE force (Sec. 2.2, Eq. (2.15)):
    F^{long,*}_i = (1/P) sum_l X_l with X = S g(k), k ~ e^{-k^2/4 alpha}/S and
    g(k) = -(4 pi k_e q_i k / (V k^2)) Im(e^{-i k.r_i} rho(k)); hence
    Var = (S sum_k e^{-k^2/4 alpha} g(k)^2 - (F^long_i)^2) / P with
    F^long_i = sum_k e^{-k^2/4 alpha} g(k).  The sums run over every k of the
    box in numpy (independent of the oracle's sampler and Fourier code) and
    the prediction is compared with the oracle's variance over 2,000 seeds."""
    s = systems.water(334, seed=6)          # 1,002 atoms, L = 21.5 A
    P, nseeds = 20, 2000
    atoms = [0, 1, 517]
    M = orc.k_table(s.alpha, s.L)[0]
    ax = np.arange(-M, M + 1)
    m = np.stack(np.meshgrid(ax, ax, ax, indexing="ij"), -1).reshape(-1, 3)
    m = m[np.any(m != 0, axis=1)]
    k = 2 * np.pi * m / s.L
    k2 = (k * k).sum(1)
    w = np.exp(-k2 / (4 * s.alpha))
    keep = w > 1e-30 * w.max()
    k, k2, w = k[keep], k2[keep], w[keep]
    S = w.sum()                                       # = H^3 - 1 (Eq. (2.6))
    assert S == pytest.approx(orc.S(s.alpha, s.L), rel=1e-12)
    rho = (s.q[None, :] * np.exp(1j * (k @ s.pos.T))).sum(1)
    V = s.L**3
    pred, mean = [], []
    for i in atoms:
        im = np.imag(np.exp(-1j * (k @ s.pos[i])) * rho)
        g = -(4 * np.pi * s.k_e * s.q[i] / (V * k2) * im)[:, None] * k
        F = (w[:, None] * g).sum(0)
        mean.append(F)
        pred.append((S * (w[:, None] * g * g).sum(0) - F * F) / P)
    pred, mean = np.array(pred), np.array(mean)
    samples = np.array([orc.rbe_forces(s.pos, s.q, s.type, s.mol,
                                       _params(orc, s, P=P, seed=9000 + t), 0)["F_long"][atoms]
                        for t in range(nseeds)])
    emp = samples.var(0, ddof=1)
    # relative sampling error of a variance from 2,000 draws of a 20-sample
    # mean is a few percent; 15% is several standard errors
    assert np.allclose(emp, pred, rtol=0.15), (emp / pred)
    # the mean agrees with the exact k-space force within its standard error
    z = (samples.mean(0) - mean) / np.sqrt(pred / nseeds)
    assert np.abs(z).max() < 4.5


def test_nve_heating_rate_equals_force_variance(orc, wat):
    """An unbiased stochastic force F = F_true + xi, with xi drawn afresh at
    each evaluation (variance sigma^2 per component), heats velocity-Verlet
    NVE dynamics by 1/2 dt^2 accel sum_i sum_c sigma_ic^2 / m_i per step: the
    velocity picks up dt accel xi / m per step (the two half kicks that use
    one evaluation add coherently), the cross terms vanish because xi has zero
    mean given the state (Sec. 2.2's unbiasedness), and the kinetic energy is
    m v^2 / (2 accel).  The variance comes from 300 seeds of the estimator at
    the start configuration; the heating is the mean slope of the total
    energy over 14 seeded NVE runs of 50 steps (flexible water, bonded terms
    deterministic).  Re-drawing the force for the first half kick of a step
    (instead of reusing the last one) would halve the heating; dropping the
    Fourier or the real-space noise would lower it by that part's share."""
    s = wat
    nvar, nrun, nsteps = 300, 14, 50
    F = np.array([orc.rbe_forces(s.pos, s.q, s.type, s.mol, _params(orc, s, seed=500 + k), 0)["F"]
                  for k in range(nvar)])
    var = F.var(0, ddof=1)
    pred = 0.5 * s.dt**2 * s.accel * (var / s.mass[:, None]).sum()
    bonded = orc.water_bonded(s.pos, s.L, s.n_water_mol, *s.bonds)[1]
    t = np.arange(nsteps, dtype=np.float64)
    slopes = []
    for k in range(nrun):
        pr = _params(orc, s, seed=2000 + k)
        F0 = orc.rbe_forces(s.pos, s.q, s.type, s.mol, pr, 0)["F"] + bonded
        out = orc.vv_run(s.pos, s.vel, s.mass, s.q, s.type, s.mol, pr, 0, nsteps, s.dt, s.accel, F0,
                         water=(s.n_water_mol, *s.bonds))
        assert out["status"] == 0
        slopes.append(np.polyfit(t, out["trace"].sum(1), 1)[0])
    slopes = np.array(slopes)
    se = slopes.std(ddof=1) / math.sqrt(nrun)
    assert abs(slopes.mean() - pred) < 4 * se + 0.06 * pred, (slopes.mean(), se, pred)
