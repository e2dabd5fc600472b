"""rbe_rho_noalloc: the structure-factor entry point for callers that cannot
let the library allocate device memory (their device memory belongs to
another allocator or a fixed budget, or allocating is not allowed where they
call).  Its scratch is a static device array, so this test checks, through
the C ABI, that two calls in a row give the same rho(k) as the context path
of rbe_forces (within the rho tolerance of the parity tests), that the
second call is not disturbed by what the first left in the shared array, and
that a P beyond the compiled maximum is refused.  This file is collected
last; it also passes when run alone in a fresh process."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_rho_noalloc_matches_context_path_twice():
    import torch

    import oracle  # noqa: F401  (builds the test oracle; not used by the entry point)
    from paper_2204_13595_gb300 import build, rbe, systems
    assert torch.cuda.is_available()
    build.build()
    for sysf, step in ((lambda: systems.water(4000, seed=4), 7), (lambda: systems.electrolyte(), 3)):
        s = sysf()
        ctx = rbe.Context(s.L, s.alpha, s.r_c, s.r_s, s.p, s.P, 5, k_e=s.k_e, eps=s.eps, sigma=s.sigma)
        dev = lambda a, dt=torch.float64: torch.tensor(a, dtype=dt, device="cuda")
        pos, q, typ = dev(s.pos), dev(s.q), dev(s.type, torch.int32)
        mol = None if s.mol is None else dev(s.mol, torch.int32)
        F = torch.empty_like(pos)
        ctx.forces(step, pos, q, typ, mol, F)
        assert ctx.sync_status() == 0
        m, rho_ctx = ctx.get_kspace()
        m_dev = torch.tensor(m, dtype=torch.int32, device="cuda")
        tol = 1e-13 * np.abs(s.q).sum()
        for call in range(2):
            rho = torch.full((s.P, 2), np.nan, dtype=torch.float64, device="cuda")
            rbe.rho_noalloc(pos, q, s.L, m_dev, rho)
            torch.cuda.synchronize()
            r = rho.cpu().numpy()
            got = r[:, 0] + 1j * r[:, 1]
            assert np.isfinite(r).all(), call
            assert np.max(np.abs(got - rho_ctx)) < tol, call
        ctx.close()


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
