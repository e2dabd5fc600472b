"""Parity of the method variants on the GPU with the oracle (reading R13):
shell batches with replacement, the per-pair LJ cutoff (WCA soft spheres)
and the Metropolis-Hastings k pool.  Same bars as the base method: lists,
batches and k samples bit-exact; FP64 forces within 1e-11 of each
component's condition scale; energies within 1e-12."""
import numpy as np
import pytest

from gpu_util import cond_err, ek_scale, gpu_forces, oracle, rbe, rms_rel, systems, to_dev

pytestmark = pytest.mark.gpu

WCA = 2.0 ** (1.0 / 6.0)


def _pr(s, **kw):
    return oracle.make_params(s.L, s.alpha, s.r_c, s.r_s, kw.pop("p", s.p), kw.pop("P", s.P), kw.pop("seed", s.seed),
                              k_e=s.k_e, eps=kw.pop("eps", s.eps), sigma=kw.pop("sigma", s.sigma), **kw)


def _ctx(s, precision=rbe.FP64, shell_mode=0, lj_rc_factor=0.0, shift=0, kpool=0, kpool_burn=0, debug_cap=0,
         eps=None, sigma=None):
    ctx = rbe.Context(s.L, s.alpha, s.r_c, s.r_s, s.p, s.P, s.seed, k_e=s.k_e, eps=eps or s.eps,
                      sigma=sigma or s.sigma, shift_lj=bool(shift), precision=precision)
    ctx.set_shell_sampling(shell_mode)
    ctx.set_lj_cutoff(lj_rc_factor)
    ctx.set_kpool(kpool, kpool_burn)
    if debug_cap:
        ctx.set_debug(True, debug_cap)
    return ctx


def _run(ctx, s, step, debug_cap=0):
    import torch
    d = to_dev(s)
    F = torch.empty_like(d["pos"])
    E = torch.zeros(rbe.NE, dtype=torch.float64, device="cuda")
    ctx.forces(step, d["pos"], d["q"], d["typ"], d["mol"], F, E)
    st = ctx.sync_status()
    out = dict(F=F.cpu().numpy(), E=E.cpu().numpy(), status=st)
    if debug_cap:
        out["lists"] = ctx.get_lists(s.n, debug_cap)
    out["m"], out["rho"] = ctx.get_kspace()
    return out


@pytest.mark.parametrize("name", ["electrolyte", "water"])
def test_with_replacement_lists_and_forces(name):
    s = systems.electrolyte() if name == "electrolyte" else systems.water(334, seed=6)
    step = 4
    pr = _pr(s, shell_mode=1)
    ol = oracle.lists(s.pos, pr, step, cap_core=256)
    ref = oracle.rbe_forces(s.pos, s.q, s.type, s.mol, pr, step)
    out = _run(_ctx(s, shell_mode=1, debug_cap=256), s, step, debug_cap=256)
    assert out["status"] == 0
    L = out["lists"]
    assert (L["n_shell"] == ol["n_shell"]).all() and (L["core"] == ol["core"]).all()
    assert (L["batch"] == ol["batch"]).all()
    # repeats occur (with replacement) and differ from the Floyd batches
    b = L["batch"]
    rows = [r[r >= 0] for r in b]
    assert any(len(set(r.tolist())) < len(r) for r in rows)
    floyd = oracle.lists(s.pos, _pr(s), step, cap_core=256)["batch"]
    assert not np.array_equal(floyd, b)
    assert cond_err(out["F"], ref) < 1e-11
    mixed = _run(_ctx(s, precision=rbe.MIXED, shell_mode=1), s, step)
    assert rms_rel(mixed["F"], out["F"]) < 1e-4


def test_wca_electrolyte_forces_energies():
    """The paper's primitive-model electrolyte with shifted-truncated LJ soft
    spheres (Sec. 3.1) against the oracle; the LJ energy differs from the
    unshifted full-range LJ."""
    s = systems.electrolyte()
    step = 2
    pr = _pr(s, shift_lj=1, lj_rc_factor=WCA)
    ref = oracle.rbe_forces(s.pos, s.q, s.type, s.mol, pr, step)
    out = _run(_ctx(s, lj_rc_factor=WCA, shift=1), s, step)
    assert out["status"] == 0
    assert cond_err(out["F"], ref) < 1e-11
    for k in (0, 2, 3, 4):
        assert out["E"][k] == pytest.approx(ref["E"][k], rel=1e-12, abs=1e-12 * abs(ref["E"]).sum())
    assert abs(out["E"][1] - ref["E"][1]) < 1e-12 * ek_scale(s, ref)
    base = oracle.rbe_forces(s.pos, s.q, s.type, s.mol, _pr(s), step)
    assert abs(base["E"][3] - ref["E"][3]) > 1e-3 * abs(base["E"][3])
    mixed = _run(_ctx(s, precision=rbe.MIXED, lj_rc_factor=WCA, shift=1), s, step)
    assert rms_rel(mixed["F"], out["F"]) < 1e-4
    assert mixed["E"][3] == pytest.approx(ref["E"][3], rel=1e-5)


def test_wca_adjoint_matches_oracle():
    import torch
    s = systems.electrolyte(n=600, L=(600 / 0.25) ** (1 / 3), seed=12)
    step = 3
    pr = _pr(s, shift_lj=1, lj_rc_factor=WCA, eps=(1.3,), sigma=(1.0,))
    rng = np.random.default_rng(1)
    v = rng.normal(size=s.pos.shape)
    g = oracle.rbe_adjoint(s.pos, s.q, s.type, s.mol, pr, step, v)
    ctx = _ctx(s, lj_rc_factor=WCA, shift=1, eps=(1.3,), sigma=(1.0,))
    d = to_dev(s)
    out = ctx.adjoint(step, d["pos"], d["q"], d["typ"], d["mol"], torch.tensor(v, device="cuda"))
    for k in ("dEdq", "dLdq"):
        a = out[k].cpu().numpy()
        assert np.max(np.abs(a - g[k])) < 1e-12 * np.max(np.abs(g[k])), k
    assert out["dEdeps"][0] == pytest.approx(g["dEde"][0, 0], rel=1e-11)
    assert out["dEdsig"][0] == pytest.approx(g["dEds"][0, 0], rel=1e-11)
    assert out["dLdeps"][0] == pytest.approx(g["dLde"][0, 0], rel=1e-10)
    assert out["dLdsig"][0] == pytest.approx(g["dLds"][0, 0], rel=1e-10)


@pytest.mark.parametrize("name", ["electrolyte", "water"])
def test_kpool_samples_bit_exact_and_forces(name):
    """The pool built on the device equals the oracle's chain bit for bit:
    every step's samples match, and so do the forces."""
    s = systems.electrolyte() if name == "electrolyte" else systems.water(4000, seed=4)
    K, burn = 4096, 64
    pr = _pr(s, kpool=K, kpool_burn=burn)
    ctx = _ctx(s, kpool=K, kpool_burn=burn)
    for step in (0, 1, 9):
        out = _run(ctx, s, step)
        assert out["status"] == 0
        assert np.array_equal(out["m"], oracle.sample_k_params(pr, step)), step
    ref = oracle.rbe_forces(s.pos, s.q, s.type, s.mol, pr, 9)
    assert cond_err(out["F"], ref) < 1e-11
    # the pool's samples differ from the fresh draws of the base method
    assert not np.array_equal(out["m"], oracle.sample_k_params(_pr(s), 9))


def test_variants_in_a_batch_equal_single_system():
    """Contexts with different variants in one batch: each replica equals its
    own single-system path bit for bit."""
    import torch
    suite = systems.batch_replicas(nrep=4, n_min=1000, n_max=4000, seed0=500)
    ctxs = []
    for r, s in enumerate(suite):
        c = rbe.Context.for_system(s, precision=rbe.MIXED)
        if r == 0:
            c.set_shell_sampling(rbe.SHELL_REPLACE)
        if r == 1:
            c.set_kpool(2048, 32)
        if r == 2 and s.name == "electrolyte":
            c.set_lj_cutoff(WCA)
        ctxs.append(c)
    dev = lambda a, dt=torch.float64: torch.tensor(a, dtype=dt, device="cuda")
    D = [dict(pos=dev(s.pos), q=dev(s.q), typ=dev(s.type, torch.int32),
              mol=None if s.mol is None else dev(s.mol, torch.int32),
              F=torch.zeros((s.n, 3), dtype=torch.float64, device="cuda")) for s in suite]
    b = rbe.Batch(ctxs)
    b.bind([d["pos"] for d in D], [d["q"] for d in D], [d["typ"] for d in D], [d["mol"] for d in D],
           [d["F"] for d in D])
    b.forces(6)
    assert b.sync_status()[0] == 0
    for c, d in zip(ctxs, D):
        F1 = torch.empty_like(d["pos"])
        c.forces(6, d["pos"], d["q"], d["typ"], d["mol"], F1)
        assert torch.equal(F1, d["F"])
