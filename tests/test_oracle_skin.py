"""Pins of the oracle's Verlet-skin variant (reading R15; Sec. 2.3's remark
that lists need not be rebuilt every step), CPU only.

The stored list V(i) holds every j within r_s + d at the rebuild positions,
in the canonical order of that step; a later step classifies V(i) at its own
positions.  Pinned here: V(i) by the stencil equals V(i) by brute force;
while no atom has moved more than d/2, the core and shell sets from V(i)
equal those of the stencil walk at the same positions (the order of S(i) is
V(i)'s); the rebuild test switches exactly at d/2; with p >= N_S the forces
reduce to the plain estimator's; and the skin estimator is unbiased for the
truncated exact real-space force over seeds.
"""
import math

import numpy as np
import pytest

from paper_2204_13595_gb300 import systems


def _params(orc, s, skin, p=None, seed=1):
    return orc.make_params(s.L, s.alpha, s.r_c, s.r_s, s.p if p is None else p, s.P, seed,
                           k_e=s.k_e, eps=s.eps, sigma=s.sigma, skin=skin)


@pytest.fixture(scope="module")
def elec():
    return systems.electrolyte()


@pytest.fixture(scope="module")
def wat():
    return systems.water(334, seed=6)       # 1002 atoms, L = 21.5 A: the stencil wraps


def _jiggle(s, amp, seed):
    """Positions moved by uniform displacements of at most amp per component
    (seeded, synthetic: a stand-in for a few MD steps)."""
    rng = np.random.default_rng(seed)
    return s.pos + rng.uniform(-amp, amp, size=s.pos.shape)


def test_stored_lists_stencil_equals_brute_force(orc, elec, wat):
    for s, skin in ((elec, 0.5), (wat, 1.0)):
        pr = _params(orc, s, skin)
        c1, v1, st1 = orc.skin_lists(s.pos, pr, brute=False, cap=1500)
        c2, v2, st2 = orc.skin_lists(s.pos, pr, brute=True, cap=1500)
        assert st1 == 0 and st2 == 0
        assert (c1 == c2).all() and (v1 == v2).all()
        # |V(i)| = 4/3 pi (r_s + d)^3 rho on average
        rho = s.n / s.L**3
        assert c1.mean() == pytest.approx(4 / 3 * math.pi * (s.r_s + skin) ** 3 * rho, rel=0.03)


def test_stored_list_is_canonical_order_of_rebuild_step(orc, elec):
    """V(i) is in ascending canonical position at the rebuild step: the same
    order as the default method's lists built at those positions."""
    s = elec
    skin = 0.5
    big = orc.make_params(s.L, s.alpha, s.r_c, s.r_s + skin, 4000, s.P, 1, k_e=s.k_e, eps=s.eps, sigma=s.sigma)
    ref = orc.lists(s.pos, big, 0, cap_core=300, cap_shell=1500)   # C and S of radii r_c, r_s + d
    c, v, st = orc.skin_lists(s.pos, _params(orc, s, skin), cap=1500)
    assert st == 0
    assert (c == ref["n_core"] + ref["n_shell"]).all()
    # canonical rank: ascending (cell, s_x, id) on the grid of floor(L/r_c) cells
    sfix, cell = orc.quantize(s.pos, s.L, s.r_c)
    rank = np.empty(s.n, dtype=np.int64)
    rank[np.lexsort((np.arange(s.n), sfix[:, 0], cell))] = np.arange(s.n)
    for i in range(s.n):
        want = np.concatenate([ref["core"][i, :ref["n_core"][i]], ref["shell"][i, :ref["n_shell"][i]]])
        want = want[np.argsort(rank[want], kind="stable")]
        assert (v[i, :c[i]] == want).all(), i


@pytest.mark.parametrize("which", ["elec", "wat"])
def test_sets_between_rebuilds_equal_stencil_sets(orc, elec, wat, which):
    s, skin = (elec, 0.6) if which == "elec" else (wat, 1.0)
    pr = _params(orc, s, skin)
    for frame, amp in enumerate((0.05, 0.15, 0.25 * skin / math.sqrt(3.0) * 1.9)):
        pos = _jiggle(s, amp, 100 + frame)
        assert not orc.skin_displaced(pos, s.pos, s.L, skin)
        a = orc.lists(pos, pr, 7, cap_core=300, cap_shell=1500, pos_b=s.pos)
        b = orc.lists(pos, pr, 7, cap_core=300, cap_shell=1500)
        assert a["status"] == 0 and b["status"] == 0
        assert (a["n_core"] == b["n_core"]).all() and (a["n_shell"] == b["n_shell"]).all()
        for i in range(0, s.n, 17):
            nc, ns = a["n_core"][i], a["n_shell"][i]
            assert set(a["core"][i, :nc]) == set(b["core"][i, :nc])
            assert set(a["shell"][i, :ns]) == set(b["shell"][i, :ns])
        # the order of S(i) is V(i)'s: ascending canonical position at the rebuild
        _, v, _ = orc.skin_lists(s.pos, pr, cap=1500)
        for i in range(0, s.n, 53):
            pos_in_v = {j: t for t, j in enumerate(v[i]) if j >= 0}
            order = [pos_in_v[j] for j in a["shell"][i, :a["n_shell"][i]]]
            assert order == sorted(order)


def test_rebuild_test_switches_at_half_the_skin(orc, elec):
    s = elec
    skin = 0.6
    for frac, expect in ((0.49, False), (0.51, True)):
        pos = s.pos.copy()
        pos[123] += frac * skin * np.array([0.6, 0.0, 0.8])     # |displacement| = frac * skin
        assert orc.skin_displaced(pos, s.pos, s.L, skin) is expect
    # a displacement across the periodic boundary counts by its minimum image
    pos = s.pos.copy()
    pos[5, 0] += s.L + 0.2 * skin
    assert not orc.skin_displaced(pos, s.pos, s.L, skin)


def test_without_rebuild_past_half_skin_sets_can_be_wrong(orc):
    """The rebuild test is needed: two atoms start just outside r_s + d and
    approach by 2 x 0.6 d without a rebuild, ending inside r_s; the stored
    list misses the pair while the stencil finds it."""
    L, rs, rc, skin = 20.0, 5.0, 2.5, 0.5
    pos = np.array([[5.0, 5.0, 5.0], [5.0 + rs + skin + 0.05, 5.0, 5.0], [15.0, 15.0, 15.0], [15.0, 11.0, 15.0]])
    pr = orc.make_params(L, 0.3, rc, rs, 10, 10, 1, k_e=1.0, eps=(0.0,), sigma=(1.0,), skin=skin)
    moved = pos.copy()
    moved[0, 0] += 0.6 * skin
    moved[1, 0] -= 0.6 * skin
    assert orc.skin_displaced(moved, pos, L, skin)
    a = orc.lists(moved, pr, 0, cap_core=4, cap_shell=4, pos_b=pos)
    b = orc.lists(moved, pr, 0, cap_core=4, cap_shell=4)
    assert b["n_shell"][0] == 1 and a["n_shell"][0] == 0


def test_forces_reduce_to_plain_estimator_when_p_covers_shell(orc, elec, wat):
    """With p >= max N_S the batch is all of S(i): the skin estimator's real
    space is then the plain one up to summation order."""
    for s, skin in ((elec, 0.6), (wat, 1.0)):
        pr = _params(orc, s, skin, p=4000)
        pos = _jiggle(s, 0.1, 7)
        a = orc.rbe_forces(pos, s.q, s.type, s.mol, pr, 3, pos_b=s.pos)
        b = orc.rbe_forces(pos, s.q, s.type, s.mol, pr, 3)
        assert a["status"] == 0 and b["status"] == 0
        assert np.abs(a["F"] - b["F"]).max() < 1e-12 * np.abs(b["F_abs"]).max()
        assert np.allclose(a["E"], b["E"], rtol=1e-12, atol=1e-12 * np.abs(b["E"]).max())


def test_skin_estimator_is_unbiased(orc, elec):
    """E over seeds of the skin estimator's real-space force (after the
    momentum correction of Eq. (2.13)) is the truncated exact force."""
    s = elec
    skin = 0.6
    pos = _jiggle(s, 0.1, 11)
    real = orc.ewald_exact(pos, s.q, s.type, s.mol, _params(orc, s, skin), s.r_s, 0)["F"]
    N = 800
    Fr = np.empty((N, s.n, 3))
    for k in range(N):
        out = orc.rbe_forces(pos, s.q, s.type, s.mol, _params(orc, s, skin, seed=3000 + k), 0, pos_b=s.pos)
        Fr[k] = out["F_real"] - out["corr"]
    se = Fr.std(0, ddof=1) / math.sqrt(N)
    z = ((Fr.mean(0) - real) / se).ravel()
    assert abs(np.mean(z * z) - 1.0) < 4 * math.sqrt(2.0 / z.size) + 0.03
    assert np.abs(z).max() < 5.5
