"""The seeded input generators (host only): reproducible, neutral, at the
stated densities, and the edge-case ion systems place the stated fraction of
ions in the slab."""
import numpy as np

from paper_2204_13595_gb300 import systems


def test_generators_are_reproducible_and_neutral():
    for make in (lambda: systems.electrolyte(n=500, L=12.6, seed=3), lambda: systems.water(334, seed=6),
                 lambda: systems.slab_ions(n=2000, L=20.0, seed=2)):
        a, b = make(), make()
        assert np.array_equal(a.pos, b.pos) and np.array_equal(a.vel, b.vel)
        assert abs(a.q.sum()) <= 1e-12 * np.abs(a.q).sum()
        assert ((a.pos >= 0) & (a.pos < a.L)).all()


def test_water_density_and_geometry():
    s = systems.water(4000, seed=4)
    assert s.n == 12000 and abs(4000 / s.L ** 3 - systems.WATER_DENSITY) < 1e-12
    p = s.pos.reshape(-1, 3, 3)
    d = p[:, 1:, :] - p[:, :1, :]
    d -= s.L * np.round(d / s.L)
    assert np.allclose(np.linalg.norm(d, axis=2), systems.R_OH, atol=1e-9)
    cosang = (d[:, 0] * d[:, 1]).sum(1) / (np.linalg.norm(d[:, 0], axis=1) * np.linalg.norm(d[:, 1], axis=1))
    assert np.allclose(np.arccos(cosang), systems.THETA_HOH, atol=1e-9)


def test_slab_ions_fraction_and_extent():
    s = systems.slab_ions(n=8000, L=32.0, slab_frac=0.5, slab_width=3.0, seed=11)
    k = 4000
    assert (s.pos[:k, 2] < 3.0).all()
    # the rest are uniform in the box: about 3/32 of them fall in the slab
    frac = (s.pos[k:, 2] < 3.0).mean()
    assert abs(frac - 3.0 / 32.0) < 5 * np.sqrt(frac * (1 - frac) / k)
    assert s.eps == (0.0,) and s.mol is None
    u = systems.slab_ions(n=1000, L=10.0, slab_frac=0.0, seed=1)
    assert abs(u.pos[:, 2].mean() - 5.0) < 0.5


def test_electrolyte_2to1_is_neutral_and_spaced():
    from paper_2204_13595_gb300 import systems
    s = systems.electrolyte_2to1(n_cations=60, L=12.0, seed=3)
    assert s.n == 180 and abs(s.q.sum()) == 0.0
    assert (s.q == 2.0).sum() == 60 and (s.q == -1.0).sum() == 120
    d = s.pos[:, None, :] - s.pos[None, :, :]
    d -= s.L * np.round(d / s.L)
    r = np.sqrt((d * d).sum(-1)) + np.eye(s.n) * 1e9
    assert r.min() >= 1.0
    assert systems.electrolyte_2to1(n_cations=60, L=12.0, seed=3).pos.tobytes() == s.pos.tobytes()
