"""rbe_rho_noalloc: the structure-factor entry point for callers that cannot
let the library allocate device memory (their device memory belongs to
another allocator or a fixed budget, or allocating, with the device-wide
synchronisation cudaFree brings, is not allowed where they call).  Its
scratch is a static device array shared by every call, so this test calls it
through the C ABI twice in a row on each case and checks that both calls give
the rho(k) of the existing entry point (rbe_forces' structure factors, read
back with rbe_get_kspace) and of the oracle's direct sum, within the rho
tolerance of the parity tests (1e-13 of sum |q|), so that the second call is
not disturbed by what the first left in the shared array.  The cases cover
more than one pass over the k vectors (P > 256), the compiled maximum
P = RBE_NOALLOC_PMAX, more atoms than one tile per block (n > 65,536), n = 0,
and a P beyond the maximum, which is refused.  This file is collected last;
it also passes when run alone in a fresh process."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _noalloc_twice(rbe, pos, q, L, m_dev, P):
    import torch
    out = []
    for _ in range(2):
        rho = torch.full((P, 2), np.nan, dtype=torch.float64, device="cuda")
        rbe.rho_noalloc(pos, q, L, m_dev, rho)
        torch.cuda.synchronize()
        r = rho.cpu().numpy()
        assert np.isfinite(r).all()
        out.append(r[:, 0] + 1j * r[:, 1])
    return out


def test_rho_noalloc_matches_existing_entry_point_and_oracle_twice():
    import torch

    import oracle
    from paper_2204_13595_gb300 import build, rbe, systems
    assert torch.cuda.is_available()
    build.build()
    oracle.build()
    for sysf, step in ((lambda: systems.water(4000, seed=4), 7), (lambda: systems.electrolyte(), 3),
                       (lambda: systems.water(25000, seed=6), 2)):
        s = sysf()
        ctx = rbe.Context(s.L, s.alpha, s.r_c, s.r_s, s.p, s.P, 5, k_e=s.k_e, eps=s.eps, sigma=s.sigma)
        dev = lambda a, dt=torch.float64: torch.tensor(a, dtype=dt, device="cuda")
        pos, q, typ = dev(s.pos), dev(s.q), dev(s.type, torch.int32)
        mol = None if s.mol is None else dev(s.mol, torch.int32)
        F = torch.empty_like(pos)
        ctx.forces(step, pos, q, typ, mol, F)
        assert ctx.sync_status() == 0
        m, rho_ctx = ctx.get_kspace()
        rho_orc = oracle.rho(s.pos, s.q, s.L, m)
        tol = 1e-13 * np.abs(s.q).sum()
        for got in _noalloc_twice(rbe, pos, q, s.L, torch.tensor(m, dtype=torch.int32, device="cuda"), s.P):
            assert np.max(np.abs(got - rho_ctx)) < tol
            assert np.max(np.abs(got - rho_orc)) < tol
        ctx.close()


def test_rho_noalloc_large_P_and_many_atoms_against_oracle_twice():
    """P = 300 (two passes of 256 k vectors per block) and P = RBE_NOALLOC_PMAX
    on 75,000 atoms (every block walks several tiles), random m in
    [-8, 8]^3 without 0."""
    import torch

    import oracle
    from paper_2204_13595_gb300 import build, rbe, systems
    build.build()
    oracle.build()
    s = systems.water(25000, seed=6)
    pos = torch.tensor(s.pos, dtype=torch.float64, device="cuda")
    q = torch.tensor(s.q, dtype=torch.float64, device="cuda")
    rng = np.random.default_rng(11)
    tol = 1e-13 * np.abs(s.q).sum()
    for P in (300, rbe.NOALLOC_PMAX):
        m = rng.integers(-8, 9, size=(P, 3)).astype(np.int32)
        m[np.all(m == 0, axis=1)] = (1, 0, 0)
        ref = oracle.rho(s.pos, s.q, s.L, m)
        for got in _noalloc_twice(rbe, pos, q, s.L, torch.tensor(m, device="cuda"), P):
            assert np.max(np.abs(got - ref)) < tol, P


def test_rho_noalloc_no_atoms_gives_zero_twice():
    import torch

    from paper_2204_13595_gb300 import rbe
    pos = torch.zeros((0, 3), dtype=torch.float64, device="cuda")
    q = torch.zeros(0, dtype=torch.float64, device="cuda")
    m = torch.tensor([[1, 0, 0], [0, 2, -1], [3, 3, 3]], dtype=torch.int32, device="cuda")
    for got in _noalloc_twice(rbe, pos, q, 10.0, m, 3):
        assert np.all(got == 0)


def test_rho_noalloc_rejects_oversize_P():
    import torch

    from paper_2204_13595_gb300 import rbe
    pos = torch.zeros((4, 3), dtype=torch.float64, device="cuda")
    q = torch.tensor([1.0, -1.0, 1.0, -1.0], dtype=torch.float64, device="cuda")
    m = torch.ones((rbe.NOALLOC_PMAX + 1, 3), dtype=torch.int32, device="cuda")
    rho = torch.zeros((rbe.NOALLOC_PMAX + 1, 2), dtype=torch.float64, device="cuda")
    with pytest.raises(rbe.RbeError) as e:
        rbe.rho_noalloc(pos, q, 10.0, m, rho)
    assert e.value.code == rbe.ELIMIT
