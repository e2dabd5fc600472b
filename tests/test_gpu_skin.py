"""Verlet-skin variant on the GPU (rbe_set_verlet_skin; reading R15 of the
oracle) against the oracle, frame by frame.

A sequence of frames is made on the host (seeded random displacements that
accumulate, standing in for MD steps).  The oracle decides the rebuilds by
its own exact test (some atom moved more than skin/2 since the rebuild
positions) and computes each frame's lists and forces from the stored lists
of its rebuild positions; the context, called once per frame, must rebuild
at the same frames and give the same lists and batches bit for bit, FP64
forces within the parity bar, mixed forces within 1e-4 RMS of FP64.
"""
import numpy as np
import pytest

from gpu_util import cond_err, oracle, rbe, rms_rel, systems

pytestmark = pytest.mark.gpu

CAP = 256


def _frames(s, nframes, amp, seed):
    rng = np.random.default_rng(seed)
    out, pos = [], s.pos.copy()
    for f in range(nframes):
        out.append(pos.copy())
        pos = pos + rng.uniform(-amp, amp, size=pos.shape)
    return out


def _params(s, skin):
    return oracle.make_params(s.L, s.alpha, s.r_c, s.r_s, s.p, s.P, s.seed, k_e=s.k_e, eps=s.eps, sigma=s.sigma,
                              skin=skin)


@pytest.mark.parametrize("kind", ["electrolyte", "water"])
def test_skin_frames_match_oracle(kind):
    import torch
    if kind == "electrolyte":
        s, skin, amp = systems.electrolyte(), 0.6, 0.07
    else:
        s, skin, amp = systems.water(4000, seed=4), 1.0, 0.12
    frames = _frames(s, 8, amp, 31)
    pr = _params(s, skin)
    ctxs = {}
    for prec in (rbe.FP64, rbe.MIXED):
        c = rbe.Context(s.L, s.alpha, s.r_c, s.r_s, s.p, s.P, s.seed, k_e=s.k_e, eps=s.eps, sigma=s.sigma,
                        precision=prec)
        c.set_verlet_skin(skin)
        c.set_debug(True, CAP)
        ctxs[prec] = c
    q, typ = torch.tensor(s.q, device="cuda"), torch.tensor(s.type, dtype=torch.int32, device="cuda")
    mol = None if s.mol is None else torch.tensor(s.mol, dtype=torch.int32, device="cuda")
    pos_b, rebuilds = None, 0
    for f, pf in enumerate(frames):
        if pos_b is None or oracle.skin_displaced(pf, pos_b, s.L, skin):
            pos_b, rebuilds = pf, rebuilds + 1
        ol = oracle.lists(pf, pr, f, cap_core=CAP, pos_b=pos_b)
        ref = oracle.rbe_forces(pf, s.q, s.type, s.mol, pr, f, pos_b=pos_b)
        assert ol["status"] == 0 and ref["status"] == 0
        pos = torch.tensor(pf, device="cuda")
        F = {}
        for prec, c in ctxs.items():
            Fd = torch.empty_like(pos)
            c.forces(f, pos, q, typ, mol, Fd)
            assert c.sync_status() == 0
            assert c.info()["skin_rebuilds"] == rebuilds, (prec, f)
            L = c.get_lists(s.n, CAP)
            for k in ("n_core", "n_shell", "core", "batch"):
                assert (L[k] == ol[k]).all(), (prec, f, k)
            F[prec] = Fd.cpu().numpy()
        assert cond_err(F[rbe.FP64], ref) < 1e-11, f
        assert rms_rel(F[rbe.MIXED], F[rbe.FP64]) < 1e-4, f
    assert 2 <= rebuilds < len(frames), rebuilds           # the test crosses rebuilds and reuses lists
    for c in ctxs.values():
        c.close()


def test_skin_argument_checks():
    s = systems.electrolyte()
    c = rbe.Context.for_system(s)
    with pytest.raises(rbe.RbeError):
        c.set_verlet_skin(-1.0)
    with pytest.raises(rbe.RbeError):
        c.set_verlet_skin(s.L)                  # r_s + skin beyond L/2
    c.set_verlet_skin(0.5)
    import torch
    d = {k: torch.tensor(v, device="cuda") for k, v in (("pos", s.pos), ("q", s.q))}
    typ = torch.tensor(s.type, dtype=torch.int32, device="cuda")
    with pytest.raises(rbe.RbeError):
        c.adjoint(1, d["pos"], d["q"], typ, None, torch.zeros_like(d["pos"]))
    c.set_verlet_skin(0.0)
    c.close()
