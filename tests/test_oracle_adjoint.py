"""Pins of the oracle's gradients (derivatives of the estimator at frozen
draws) against central finite differences of the oracle estimator itself."""
import numpy as np
import pytest

from paper_2204_13595_gb300 import systems


def _pr(orc, s, eps=None, sigma=None, shift=0):
    return orc.make_params(s.L, s.alpha, s.r_c, s.r_s, s.p, s.P, 7, k_e=s.k_e, eps=eps or s.eps,
                           sigma=sigma or s.sigma, shift_lj=shift)


def _EL(orc, s, q, pr, step, v):
    out = orc.rbe_forces(s.pos, q, s.type, s.mol, pr, step)
    return out["E"][:5].sum(), float((v * out["F"]).sum())


def _type_grads(g, eps, sigma):
    """Chain rule of the Lorentz-Berthelot pair table to per-type parameters."""
    T = len(eps)
    ge, gs = np.zeros(T), np.zeros(T)
    for a in range(T):
        for b in range(T):
            ee = np.sqrt(eps[a] * eps[b])
            if a == b:
                de = 1.0
            else:
                de = 0.0 if eps[b] == 0.0 else (np.inf if eps[a] == 0.0 else eps[b] / (2 * ee))
            ge[a] += (g["e"][a, b] + g["e"][b, a]) * de if a != b else g["e"][a, a] * de
            gs[a] += (g["s"][a, b] + g["s"][b, a]) * 0.5 if a != b else g["s"][a, a]
    return ge, gs


@pytest.mark.parametrize("shift", [0, 1])
def test_adjoint_matches_finite_differences(orc, shift):
    s = systems.water(334, seed=6)
    rng = np.random.default_rng(2)
    v = rng.normal(size=s.pos.shape)
    step = 3
    pr = _pr(orc, s, shift=shift)
    g = orc.rbe_adjoint(s.pos, s.q, s.type, s.mol, pr, step, v)
    assert g["status"] == 0
    h = 1e-6
    for m in (0, 1, 2, 500, 1001):
        qp, qm = s.q.copy(), s.q.copy()
        qp[m] += h
        qm[m] -= h
        Ep, Lp = _EL(orc, s, qp, pr, step, v)
        Em, Lm = _EL(orc, s, qm, pr, step, v)
        assert g["dEdq"][m] == pytest.approx((Ep - Em) / (2 * h), rel=1e-6, abs=1e-4)
        assert g["dLdq"][m] == pytest.approx((Lp - Lm) / (2 * h), rel=1e-6, abs=1e-3)
    ge_E, gs_E = _type_grads({"e": g["dEde"], "s": g["dEds"]}, s.eps, s.sigma)
    ge_L, gs_L = _type_grads({"e": g["dLde"], "s": g["dLds"]}, s.eps, s.sigma)
    for which, grads in (("eps", (ge_E, ge_L)), ("sigma", (gs_E, gs_L))):
        hp = 1e-6 * (s.eps[0] if which == "eps" else s.sigma[0])
        par_p = list(s.eps if which == "eps" else s.sigma)
        par_m = list(par_p)
        par_p[0] += hp
        par_m[0] -= hp
        kw_p = {"eps": tuple(par_p)} if which == "eps" else {"sigma": tuple(par_p)}
        kw_m = {"eps": tuple(par_m)} if which == "eps" else {"sigma": tuple(par_m)}
        Ep, Lp = _EL(orc, s, s.q, _pr(orc, s, shift=shift, **kw_p), step, v)
        Em, Lm = _EL(orc, s, s.q, _pr(orc, s, shift=shift, **kw_m), step, v)
        assert grads[0][0] == pytest.approx((Ep - Em) / (2 * hp), rel=1e-6), which
        assert grads[1][0] == pytest.approx((Lp - Lm) / (2 * hp), rel=1e-5), which


def test_adjoint_electrolyte_all_charges(orc):
    """Every charge of a small electrolyte, including the shell batches and the
    momentum correction, against finite differences."""
    s = systems.electrolyte(n=200, L=10.0, seed=4)
    rng = np.random.default_rng(8)
    v = rng.normal(size=s.pos.shape)
    pr = _pr(orc, s)
    g = orc.rbe_adjoint(s.pos, s.q, s.type, s.mol, pr, 1, v)
    h = 1e-6
    fdE, fdL = np.zeros(s.n), np.zeros(s.n)
    for m in range(s.n):
        qp, qm = s.q.copy(), s.q.copy()
        qp[m] += h
        qm[m] -= h
        Ep, Lp = _EL(orc, s, qp, pr, 1, v)
        Em, Lm = _EL(orc, s, qm, pr, 1, v)
        fdE[m], fdL[m] = (Ep - Em) / (2 * h), (Lp - Lm) / (2 * h)
    assert np.allclose(g["dEdq"], fdE, rtol=1e-6, atol=1e-6 * np.abs(fdE).max())
    assert np.allclose(g["dLdq"], fdL, rtol=1e-5, atol=1e-5 * np.abs(fdL).max())


@pytest.mark.parametrize("shift", [0, 1])
def test_adjoint_euler_homogeneity(orc, shift):
    """At frozen draws the Coulomb energy and forces are homogeneous of degree 2
    in the charges and the LJ energy and forces of degree 1 in the pair
    well depths eps_ab (the shift of Eq. (2.10) scales with eps_ab too), so by
    Euler's theorem q.dE/dq = 2 E_coul and sum_ab eps_ab dE/deps_ab = E_LJ, and
    the same for L = sum_i gF_i . F_i (the momentum correction is linear in F)."""
    s = systems.water(334, seed=9)
    rng = np.random.default_rng(5)
    v = rng.normal(size=s.pos.shape)
    pr = _pr(orc, s, shift=shift)
    g = orc.rbe_adjoint(s.pos, s.q, s.type, s.mol, pr, 2, v)
    out = orc.rbe_forces(s.pos, s.q, s.type, s.mol, pr, 2)
    E = out["E"]
    e_coul = E[0] + E[1] + E[2] + E[4]
    T = len(s.eps)
    eps_ab = np.sqrt(np.outer(s.eps, s.eps))
    lj_E = float((eps_ab * g["dEde"][:T, :T]).sum())
    lj_L = float((eps_ab * g["dLde"][:T, :T]).sum())
    L = float((v * out["F"]).sum())
    assert float(s.q @ g["dEdq"]) == pytest.approx(2 * e_coul, rel=1e-11)
    assert lj_E == pytest.approx(E[3], rel=1e-11)
    # L has no separate Coulomb/LJ split in the output; the two Euler sums add up to L.
    scale = float(np.abs(s.q * g["dLdq"]).sum()) + float(np.abs(eps_ab * g["dLde"][:T, :T]).sum())
    assert abs(0.5 * float(s.q @ g["dLdq"]) + lj_L - L) <= 1e-11 * scale
