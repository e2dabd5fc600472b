"""Pins of the oracle's random-number layer (CPU only).

Philox4x64-10 (Salmon et al., SC'11) is pinned to numpy's independent
implementation; the k sampler to the exact law P_k of Eq. (2.8) and the
Poisson form of H in Eq. (2.7); Floyd's sampler to the uniform law over
subsets that the shell estimator of Eq. (2.11) assumes.
"""
import itertools
import math

import numpy as np
import pytest

from paper_2204_13595_gb300 import systems


def _numpy_philox_block(ctr, key):
    """Block at counter ctr from numpy.random.Philox (which increments first)."""
    g = np.random.Philox(key=np.array(key, dtype=np.uint64))
    st = g.state
    c = [int(x) for x in ctr]
    for i in range(4):  # ctr - 1 with borrow
        if c[i] > 0:
            c[i] -= 1
            break
        c[i] = 2**64 - 1
    st["state"]["counter"] = np.array(c, dtype=np.uint64)
    st["buffer_pos"] = 4
    g.state = st
    return g.random_raw(4)


@pytest.mark.parametrize("ctr,key", [
    ([0, 0, 0, 0], [0, 0]),
    ([5, 1, 77, 1], [2024, 0]),
    ([2**64 - 1, 3, 2**40, 2], [2**63 + 5, 0]),
    ([123, 0, 0, 0], [1, 2]),
])
def test_philox_matches_numpy(orc, ctr, key):
    assert (orc.philox4x64_10(ctr, key) == _numpy_philox_block(ctr, key)).all()


def test_philox_known_answer(orc):
    # Random123 known-answer vector for philox4x64-10 at zero counter and key
    out = orc.philox4x64_10([0, 0, 0, 0], [0, 0])
    assert [int(x) for x in out] == [0x16554D9ECA36314C, 0xDB20FE9D672D0FDC,
                                      0xD7E772CEE186176B, 0x7E68B68AEC7BA23B]


@pytest.mark.parametrize("alpha,L", [(systems.alpha_for(5.0), 20.0), (systems.alpha_for(10.0), 49.291),
                                     (0.03, 80.0), (systems.alpha_for(10.0), 21.53)])
def test_H_direct_sum_matches_poisson_form(orc, alpha, L):
    """Eq. (2.7): sum_m e^{-pi^2 m^2/(alpha L^2)} = sqrt(alpha L^2/pi) sum_m e^{-alpha m^2 L^2}."""
    M, H, T = orc.k_table(alpha, L)
    m = np.arange(-6, 7)
    poisson = math.sqrt(alpha * L * L / math.pi) * np.exp(-alpha * m * m * L * L).sum()
    assert H == pytest.approx(poisson, rel=1e-14)
    assert orc.S(alpha, L) == pytest.approx(H**3 - 1.0, rel=1e-15)
    # truncation: the first dropped weight is below 2^-64 of H
    assert math.exp(-math.pi**2 * (M + 1) ** 2 / (alpha * L * L)) / H < 2.0**-64
    assert (np.diff(T.astype(object)) >= 0).all()
    assert int(T[-1]) == 2**64 - 1


def test_k_sampler_law(orc):
    """chi^2 of the m_x marginal and of |m|^2 against P_k (Eq. (2.8)); k = 0 never drawn."""
    L, alpha, P = 20.0, systems.alpha_for(5.0), 500
    steps = 200
    m = np.concatenate([orc.sample_k(7, s, P, alpha, L) for s in range(steps)])
    assert not ((m == 0).all(axis=1)).any()
    c = math.pi**2 / (alpha * L * L)
    ms = np.arange(-40, 41)
    w = np.exp(-c * ms * ms)
    p1 = w / w.sum()
    p0 = p1[40]
    Z = 1 - p0**3
    # marginal of m_x conditioned on m != 0
    marg = p1 * (1 - np.where(ms == 0, p0 * p0, 0.0)) / Z
    bins = np.arange(-6, 7)
    obs = np.array([(m[:, 0] == b).sum() for b in bins] + [(np.abs(m[:, 0]) > 6).sum()])
    exp = np.array([marg[40 + b] for b in bins] + [marg[np.abs(ms) > 6].sum()]) * len(m)
    chi2 = ((obs - exp) ** 2 / exp).sum()
    dof = len(obs) - 1
    assert chi2 < dof + 5 * math.sqrt(2 * dof)
    # joint law through |m|^2 classes (checks independence of the axes)
    r2 = (m.astype(np.int64) ** 2).sum(1)
    classes = [1, 2, 3, 4, 5, 6, 8, 9]
    grid = np.stack(np.meshgrid(ms, ms, ms, indexing="ij"), -1).reshape(-1, 3)
    pj = (p1[grid[:, 0] + 40] * p1[grid[:, 1] + 40] * p1[grid[:, 2] + 40])
    g2 = (grid.astype(np.int64) ** 2).sum(1)
    pj = np.where(g2 == 0, 0.0, pj) / Z
    obs = np.array([(r2 == k).sum() for k in classes])
    exp = np.array([pj[g2 == k].sum() for k in classes]) * len(m)
    chi2 = ((obs - exp) ** 2 / exp).sum()
    assert chi2 < len(classes) + 5 * math.sqrt(2 * len(classes))


def test_k_sampler_depends_on_seed_and_step(orc):
    L, alpha = 49.291, systems.alpha_for(10.0)
    a = orc.sample_k(1, 3, 64, alpha, L)
    assert (a == orc.sample_k(1, 3, 64, alpha, L)).all()
    assert not (a == orc.sample_k(1, 4, 64, alpha, L)).all()
    assert not (a == orc.sample_k(2, 3, 64, alpha, L)).all()


def test_floyd_uniform_over_subsets(orc):
    """Every 3-subset of 6 ordinals equally likely; slots distinct and in range."""
    rng = np.random.default_rng(11)
    n, p, trials = 6, 3, 60000
    counts = {}
    words = rng.integers(0, 2**64, size=(trials, p), dtype=np.uint64)
    for t in range(trials):
        out = orc.floyd(n, p, words[t])
        s = tuple(sorted(int(x) for x in out))
        assert len(set(s)) == p and all(0 <= x < n for x in s)
        counts[s] = counts.get(s, 0) + 1
    subsets = list(itertools.combinations(range(n), p))
    assert set(counts) == set(subsets)
    e = trials / len(subsets)
    chi2 = sum((counts[s] - e) ** 2 / e for s in subsets)
    dof = len(subsets) - 1
    assert chi2 < dof + 5 * math.sqrt(2 * dof)


def test_floyd_large_n_inclusion(orc):
    """Inclusion probability p/n for each ordinal (n=50, p=20)."""
    rng = np.random.default_rng(5)
    n, p, trials = 50, 20, 20000
    hits = np.zeros(n)
    words = rng.integers(0, 2**64, size=(trials, p), dtype=np.uint64)
    for t in range(trials):
        out = orc.floyd(n, p, words[t])
        assert len(set(out.tolist())) == p
        hits[out.astype(np.int64)] += 1
    pi = p / n
    z = (hits - trials * pi) / math.sqrt(trials * pi * (1 - pi))
    assert np.abs(z).max() < 4.5
