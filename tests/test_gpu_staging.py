"""Stencil staging of the pair kernel.  A work unit whose stencil fits the
shared-memory staging capacity is classified from the staged copy (positions
moved to the unit's periodic images, candidate ranges concatenated into full
32-wide chunks); a unit that does not fit reads its ranges from global memory
one range at a time, and so does a pass of stencil rows whose concatenation
exceeds 2048 candidates.  All must give the oracle's lists bit for bit.  An
ion system with half of its atoms in a slab a tenth of the box thick makes part
of the units overflow, a uniform one at 2 ions per sigma^3 part of the passes
(both counted by the library in debug mode)."""
import numpy as np
import pytest

from gpu_util import cond_err, gpu_forces, oracle, params, rbe, rms_rel, systems

pytestmark = pytest.mark.gpu

CAP = 256


def _ctx(s, precision, debug=True, shell_cap=512):
    c = rbe.Context(s.L, s.alpha, s.r_c, s.r_s, s.p, s.P, s.seed, k_e=s.k_e, eps=s.eps, sigma=s.sigma,
                    precision=precision)
    c.set_capacity(128, shell_cap)
    if debug:
        c.set_debug(True, CAP)
    return c


@pytest.mark.parametrize("step", [0, 5])
def test_overflowing_units_match_oracle(step):
    s = systems.slab_ions()
    pr = params(s)
    ol = oracle.lists(s.pos, pr, step, cap_core=CAP)
    assert ol["n_core"].max() <= 128 and ol["n_shell"].max() <= 512
    ctx = _ctx(s, rbe.FP64)
    out = gpu_forces(s, step, ctx=ctx, debug_cap=CAP)
    assert out["status"] == 0
    info = ctx.info()
    assert info["unstaged_units"] > 0, "no unit exceeded the staging capacity"
    L = out["lists"]
    assert (L["n_core"] == ol["n_core"]).all()
    assert (L["n_shell"] == ol["n_shell"]).all()
    assert (L["core"] == ol["core"]).all()
    assert (L["batch"] == ol["batch"]).all()
    ref = oracle.rbe_forces(s.pos, s.q, s.type, s.mol, pr, step)
    assert cond_err(out["F"], ref) < 1e-11
    mixed = gpu_forces(s, step, ctx=_ctx(s, rbe.MIXED, debug=False))
    assert mixed["status"] == 0
    assert rms_rel(mixed["F"], out["F"]) < 1e-4
    # the mixed kernel with room for its two-atom path (staged units) next to
    # units read from global memory (one atom at a time): same lists
    mctx = _ctx(s, rbe.MIXED, shell_cap=640)
    mixed = gpu_forces(s, step, ctx=mctx, debug_cap=CAP)
    assert mixed["status"] == 0 and mctx.info()["unstaged_units"] > 0
    for k in ("n_core", "n_shell", "core", "batch"):
        assert (mixed["lists"][k] == ol[k]).all(), k
    assert rms_rel(mixed["F"], out["F"]) < 1e-4


def test_uniform_systems_stage_every_unit():
    """The paper's workloads never leave the staged path."""
    for s in (systems.electrolyte(), systems.water(4000, seed=4)):
        ctx = rbe.Context.for_system(s)
        ctx.set_debug(True, 8)
        out = gpu_forces(s, 1, ctx=ctx, debug_cap=8)
        assert out["status"] == 0
        assert ctx.info()["unstaged_units"] == 0, s.name
    assert np.isfinite(out["F"]).all()


def test_long_passes_walk_range_by_range():
    s = systems.slab_ions(n=12000, L=18.0, slab_frac=0.0, seed=5)
    step = 3
    pr = params(s)
    ol = oracle.lists(s.pos, pr, step, cap_core=CAP)
    c = rbe.Context(s.L, s.alpha, s.r_c, s.r_s, s.p, s.P, s.seed, k_e=s.k_e, eps=s.eps, sigma=s.sigma)
    c.set_debug(True, CAP)
    out = gpu_forces(s, step, ctx=c, debug_cap=CAP)
    assert out["status"] == 0
    info = c.info()
    assert info["unstaged_units"] == 0
    assert 0 < info["walked_passes"] < s.n, info["walked_passes"]
    L = out["lists"]
    assert (L["n_core"] == ol["n_core"]).all() and (L["n_shell"] == ol["n_shell"]).all()
    assert (L["core"] == ol["core"]).all() and (L["batch"] == ol["batch"]).all()
    ref = oracle.rbe_forces(s.pos, s.q, s.type, s.mol, pr, step)
    assert cond_err(out["F"], ref) < 1e-11
    # mixed: pairs of atoms whose joint pass exceeds the packed limit fall
    # back to one atom at a time
    cm = rbe.Context(s.L, s.alpha, s.r_c, s.r_s, s.p, s.P, s.seed, k_e=s.k_e, eps=s.eps, sigma=s.sigma,
                     precision=rbe.MIXED)
    cm.set_debug(True, CAP)
    mixed = gpu_forces(s, step, ctx=cm, debug_cap=CAP)
    assert mixed["status"] == 0 and cm.info()["walked_passes"] > 0
    for k in ("n_core", "n_shell", "core", "batch"):
        assert (mixed["lists"][k] == ol[k]).all(), k
    assert rms_rel(mixed["F"], out["F"]) < 1e-4
