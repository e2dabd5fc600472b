"""Pins of the oracle's method variants (reading R13): shell batches drawn with
replacement, the LJ term truncated per pair type (the WCA soft sphere of the
paper's electrolytes, Sec. 3.1) and the Metropolis-Hastings pool of k samples
(Algorithm 1, pool step; Sec. 2.2).  CPU only."""
import math

import numpy as np
import pytest

from paper_2204_13595_gb300 import systems

WCA = 2.0 ** (1.0 / 6.0)


def _params(orc, s, p=None, P=None, seed=1, **kw):
    return orc.make_params(s.L, s.alpha, s.r_c, s.r_s, s.p if p is None else p, s.P if P is None else P, seed,
                           k_e=s.k_e, eps=kw.pop("eps", s.eps), sigma=kw.pop("sigma", s.sigma), **kw)


@pytest.fixture(scope="module")
def elec():
    return systems.electrolyte()


# ---------------------------------------------------------------------------
# shell batches with replacement
# ---------------------------------------------------------------------------
def test_with_replacement_slots_are_independent_uniform(orc, elec):
    """Each slot is uniform over S(i) and the slots are independent: the
    fraction of batches holding a repeated atom is the birthday probability
    1 - prod_{k<p} (1 - k/N_S); Floyd's batches never repeat."""
    s = elec
    atoms = [5, 77, 901]
    nsteps = 600
    dup = {i: 0 for i in atoms}
    counts = {}
    ns = None
    for step in range(nsteps):
        out = orc.lists(s.pos, _params(orc, s, shell_mode=1), step, cap_core=64, cap_shell=400)
        if ns is None:
            ns = {i: int(out["n_shell"][i]) for i in atoms}
            counts = {i: np.zeros(ns[i]) for i in atoms}
            shell = {i: out["shell"][i, :ns[i]].tolist() for i in atoms}
        for i in atoms:
            b = out["batch"][i, :out["n_batch"][i]].tolist()
            assert len(b) == s.p and set(b) <= set(shell[i])
            dup[i] += len(set(b)) < len(b)
            for j in b:
                counts[i][shell[i].index(j)] += 1
    out0 = orc.lists(s.pos, _params(orc, s), 0, cap_core=64, cap_shell=400)
    for i in atoms:
        b = out0["batch"][i, :out0["n_batch"][i]].tolist()
        assert len(set(b)) == len(b)
        n = ns[i]
        p_dup = 1.0 - np.prod([1.0 - k / n for k in range(s.p)])
        sd = math.sqrt(p_dup * (1 - p_dup) / nsteps)
        assert abs(dup[i] / nsteps - p_dup) < 4.5 * sd, (i, dup[i] / nsteps, p_dup)
        # uniform marginal: chi^2 over the N_S ordinals
        c = counts[i]
        e = c.sum() / n
        chi2 = float(((c - e) ** 2 / e).sum())
        assert chi2 < n - 1 + 5 * math.sqrt(2 * (n - 1)), (i, chi2, n)


def _shell_pair_forces(s, i, shell):
    from scipy.special import erfc
    d = s.pos[shell] - s.pos[i]
    d -= s.L * np.round(d / s.L)
    r = np.sqrt((d * d).sum(1))
    sa = math.sqrt(s.alpha)
    qq = s.k_e * s.q[i] * s.q[shell]
    sr6 = (1.0 / r) ** 6
    scal = -qq * (erfc(sa * r) / r**2 + 2 * sa / math.sqrt(math.pi) * np.exp(-s.alpha * r * r) / r) / r \
        - (48 * sr6 * sr6 - 24 * sr6) / r**2
    return scal[:, None] * d


def test_with_replacement_variance_closed_form(orc, elec):
    """Var of (N_S/p) sum of p independent uniform draws of f_ij over S(i) is
    N_S^2 sigma^2 / p, sigma^2 the population variance (no finite-population
    factor (N_S - p)/(N_S - 1) as without replacement); the mean is the full
    shell sum."""
    s = elec
    atoms = [3, 400, 1234]
    lists = orc.lists(s.pos, _params(orc, s, P=1), 0, cap_core=64, cap_shell=400)
    samples = np.array([orc.rbe_forces(s.pos, s.q, s.type, None,
                                       _params(orc, s, P=1, seed=7000 + k, shell_mode=1), 0)["F_real"][atoms]
                        for k in range(3000)])
    for n_a, i in enumerate(atoms):
        ns = int(lists["n_shell"][i])
        f = _shell_pair_forces(s, i, lists["shell"][i, :ns])
        pred = ns**2 * f.var(0) / s.p
        emp = samples[:, n_a, :].var(0, ddof=1)
        assert np.allclose(emp, pred, rtol=0.15), (emp, pred)
        # the mean: core sum + full shell sum (the sampled part is unbiased)
        core = lists["core"][i, :lists["n_core"][i]]
        target = _shell_pair_forces(s, i, core).sum(0) + f.sum(0)
        se = samples[:, n_a, :].std(0, ddof=1) / math.sqrt(samples.shape[0])
        assert np.all(np.abs(samples[:, n_a, :].mean(0) - target) < 4.5 * se)


# ---------------------------------------------------------------------------
# LJ truncated per pair type (WCA)
# ---------------------------------------------------------------------------
def _pair_system(r, sig=(1.0, 1.0), types=(0, 0), L=12.0):
    pos = np.array([[1.0, 2.0, 3.0], [1.0 + r, 2.0, 3.0]])
    return pos, np.zeros(2), np.array(types, dtype=np.int32)


@pytest.mark.parametrize("r", [0.9, 1.0, 1.05, 1.1, 1.12, 1.1225, 1.2, 2.0])
def test_wca_two_particle_closed_form(orc, r):
    """WCA: U = 4 eps ((s/r)^12 - (s/r)^6) + eps for r < 2^(1/6) s, else 0;
    F = 24 eps (2 (s/r)^12 - (s/r)^6) / r along the separation."""
    L, eps, sig = 12.0, 1.3, 1.0
    pos, q, typ = _pair_system(r, L=L)
    pr = orc.make_params(L, 0.3, 2.5, 5.0, 10, 4, 1, k_e=1.0, eps=(eps,), sigma=(sig,), shift_lj=1,
                         lj_rc_factor=WCA)
    out = orc.rbe_forces(pos, q, typ, None, pr, 0)
    x = sig / r
    inside = r < WCA * sig
    U = (4 * eps * (x**12 - x**6) + eps) if inside else 0.0
    Fm = (24 * eps * (2 * x**12 - x**6) / r) if inside else 0.0
    assert out["E"][3] == pytest.approx(U, rel=1e-13, abs=1e-14)
    # momentum correction removes the mean, which is zero for a pair
    assert out["F"][1, 0] == pytest.approx(Fm, rel=1e-13, abs=1e-13)
    assert out["F"][0, 0] == pytest.approx(-Fm, rel=1e-13, abs=1e-13)
    assert abs(out["F"][1, 1]) < 1e-14 and abs(out["F"][1, 2]) < 1e-14


def test_wca_mixed_types_cut_at_mixed_sigma(orc):
    """The cutoff of pair (a, b) is 2^(1/6) sigma_ab with sigma_ab the
    Lorentz mean; at sigma_ab the shifted energy is eps_ab."""
    L = 12.0
    sa, sb, ea, eb = 1.0, 2.0, 1.0, 4.0
    sab, eab = 0.5 * (sa + sb), math.sqrt(ea * eb)
    for r, inside in ((sab, True), (WCA * sab * 0.999, True), (WCA * sab * 1.001, False)):
        pos, q, typ = _pair_system(r, types=(0, 1), L=L)
        pr = orc.make_params(L, 0.3, 4.0, 5.0, 10, 4, 1, eps=(ea, eb), sigma=(sa, sb), shift_lj=1,
                             lj_rc_factor=WCA)
        E = orc.rbe_forces(pos, q, typ, None, pr, 0)["E"][3]
        x = sab / r
        U = 4 * eab * (x**12 - x**6) + eab if inside else 0.0
        assert E == pytest.approx(U, rel=1e-12, abs=1e-14), r
    pos, q, typ = _pair_system(sab, types=(0, 1), L=L)
    pr = orc.make_params(L, 0.3, 4.0, 5.0, 10, 4, 1, eps=(ea, eb), sigma=(sa, sb), shift_lj=1, lj_rc_factor=WCA)
    assert orc.rbe_forces(pos, q, typ, None, pr, 0)["E"][3] == pytest.approx(eab, rel=1e-13)


def test_wca_electrolyte_force_is_energy_gradient(orc):
    """Central differences of the total energy at frozen draws (the WCA cut is
    continuous with zero force at the cutoff) for a small WCA electrolyte."""
    s = systems.electrolyte(n=200, L=10.0, seed=4)
    pr = orc.make_params(s.L, s.alpha, s.r_c, s.r_s, 10**6, 64, 3, k_e=s.k_e, eps=s.eps, sigma=s.sigma,
                         shift_lj=1, lj_rc_factor=WCA)
    F = orc.rbe_forces(s.pos, s.q, s.type, None, pr, 0)["F"]
    h = 1e-6
    for i in (0, 17, 111):
        for a in range(3):
            pp, pm = s.pos.copy(), s.pos.copy()
            pp[i, a] += h
            pm[i, a] -= h
            Ep = orc.rbe_forces(pp, s.q, s.type, None, pr, 0)["E"][:5].sum()
            Em = orc.rbe_forces(pm, s.q, s.type, None, pr, 0)["E"][:5].sum()
            # the momentum correction of a full (p >= N_S) real space is the
            # mean of forces that already sum to zero: F = -grad E
            assert F[i, a] == pytest.approx(-(Ep - Em) / (2 * h), rel=2e-6, abs=2e-6)


def test_wca_adjoint_matches_finite_differences(orc):
    """dE/deps and dE/dsigma through the truncated-shifted LJ (the shift at
    f sigma does not depend on sigma)."""
    s = systems.electrolyte(n=200, L=10.0, seed=4)
    kw = dict(k_e=s.k_e, shift_lj=1, lj_rc_factor=WCA)
    pr = orc.make_params(s.L, s.alpha, s.r_c, s.r_s, s.p, 16, 3, eps=(1.2,), sigma=(1.0,), **kw)
    g = orc.rbe_adjoint(s.pos, s.q, s.type, None, pr, 1, None)
    dEde, dEds = g["dEde"][0, 0], g["dEds"][0, 0]
    h = 1e-6
    E = lambda e, sg: orc.rbe_forces(s.pos, s.q, s.type, None,
                                     orc.make_params(s.L, s.alpha, s.r_c, s.r_s, s.p, 16, 3, eps=(e,), sigma=(sg,),
                                                     **kw), 1)["E"][3]
    assert dEde == pytest.approx((E(1.2 + h, 1.0) - E(1.2 - h, 1.0)) / (2 * h), rel=1e-6)
    assert dEds == pytest.approx((E(1.2, 1.0 + h) - E(1.2, 1.0 - h)) / (2 * h), rel=1e-6)
    # WCA energy is linear in eps: E_LJ = eps dE/deps
    assert 1.2 * dEde == pytest.approx(E(1.2, 1.0), rel=1e-12)


# ---------------------------------------------------------------------------
# Metropolis-Hastings pool of k samples
# ---------------------------------------------------------------------------
def test_mh_proposal_is_rounded_gaussian(orc):
    """q_m = P(round(X) = m), X ~ N(0, alpha L^2 / (2 pi^2)) (Sec. 2.2), against
    the normal CDF of scipy; w_m is the discrete Gaussian of Eq. (2.8)."""
    from scipy.stats import norm
    for alpha, L in ((0.302734, 20.0), (0.075684, 49.291)):
        M, w, q, Tq = orc.mh_tables(alpha, L)
        s = math.sqrt(alpha * L * L / (2 * math.pi**2))
        m = np.arange(-M, M + 1)
        ref = norm.sf((np.abs(m) - 0.5) / s) - norm.sf((np.abs(m) + 0.5) / s)
        ref[M] = 1 - 2 * norm.sf(0.5 / s)
        assert np.allclose(q, ref, rtol=1e-12, atol=1e-300)
        assert np.allclose(w, np.exp(-(math.pi * m) ** 2 / (alpha * L * L)), rtol=1e-14)
        assert Tq[-1] == np.iinfo(np.uint64).max and np.all(np.diff(Tq.astype(np.float64)) >= 0)


def test_mh_pool_samples_the_target(orc):
    """The chains' stationary law is P_k of Eq. (2.8): each axis's marginal over
    the pool matches w_m / H conditioned on k != 0 (chi^2 with the chain's
    near-1 acceptance making draws nearly independent); k = 0 never appears;
    the acceptance rate is high (Sec. 2.2)."""
    alpha, L = 0.302734, 20.0
    K = 200000
    pool, acc = orc.kpool(11, alpha, L, K, 100)
    assert acc > 0.9
    assert not np.any(np.all(pool == 0, axis=1))
    M, T, H = None, None, None
    M, w, q, Tq = orc.mh_tables(alpha, L)
    H = w.sum()
    p0 = w[M] / H
    for a in range(3):
        c = np.bincount(pool[:, a] + M, minlength=2 * M + 1).astype(float)
        # marginal of one axis given (m_x, m_y, m_z) != 0
        pm = (w / H) / (1 - p0**3)
        pm[M] = p0 * (1 - p0**2) / (1 - p0**3)
        e = K * pm
        keep = e > 20
        chi2 = float((((c - e) ** 2 / e)[keep]).sum()) + float((c[~keep].sum() - e[~keep].sum()) ** 2 / max(e[~keep].sum(), 1e-9))
        dof = int(keep.sum())
        # MH draws are positively correlated at a small lag: allow 1.5x
        assert chi2 < 1.5 * (dof + 5 * math.sqrt(2 * dof)), (a, chi2, dof)


def test_pool_sampler_draws_pool_entries(orc, elec):
    """With kpool = K the step's samples are pool entries; with kpool = 0 the
    variant fields leave the fresh draws of R4 unchanged."""
    s = elec
    K = 512
    pr = _params(orc, s, kpool=K, kpool_burn=50)
    pool, _ = orc.kpool(pr.seed, s.alpha, s.L, K, 50)
    rows = {tuple(r) for r in pool.tolist()}
    seen = set()
    for step in range(40):
        m = orc.sample_k_params(pr, step)
        assert all(tuple(r) in rows for r in m.tolist())
        seen |= {tuple(r) for r in m.tolist()}
    # 40 x 100 uniform draws over 512 entries leave few distinct vectors unseen
    assert len(seen) > 0.9 * len(rows)
    assert np.array_equal(orc.sample_k_params(_params(orc, s), 7), orc.sample_k(1, 7, s.P, s.alpha, s.L))
