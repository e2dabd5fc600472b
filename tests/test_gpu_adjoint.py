"""Adjoint of the force step on the GPU (rbe_adjoint, autograd): parity with
the oracle's gradients at frozen draws, mixed against FP64, and the
force-matching loss of the differentiation workload against central finite
differences (h = 1e-6) of the FP64 GPU forward."""
import math

import numpy as np
import pytest

from gpu_util import gpu_forces, oracle, params, rbe, rms_rel, systems, to_dev, type_grads

pytestmark = pytest.mark.gpu

G_TOL = 1e-10


def _ctx(s, precision=rbe.FP64):
    return rbe.Context(s.L, s.alpha, s.r_c, s.r_s, s.p, s.P, s.seed, k_e=s.k_e, eps=s.eps, sigma=s.sigma,
                       precision=precision)


@pytest.mark.parametrize("name", ["electrolyte_2000", "water_1002", "water_12k"])
def test_adjoint_matches_oracle(name):
    import torch
    s = {"electrolyte_2000": lambda: systems.electrolyte(), "water_1002": lambda: systems.water(334, seed=6),
         "water_12k": lambda: systems.water(4000, seed=4)}[name]()
    rng = np.random.default_rng(3)
    v = rng.normal(size=s.pos.shape)
    step = 5
    ref = oracle.rbe_adjoint(s.pos, s.q, s.type, s.mol, params(s), step, v)
    d = to_dev(s)
    ctx = _ctx(s)
    g = ctx.adjoint(step, d["pos"], d["q"], d["typ"], d["mol"], torch.tensor(v, device="cuda"))
    assert ctx.sync_status() == 0
    for k in ("dEdq", "dLdq"):
        got = g[k].cpu().numpy()
        err = np.max(np.abs(got - ref[k])) / np.max(np.abs(ref[k]))
        print(f"{name} {k}: max err / max |g| = {err:.2e}")
        assert err < G_TOL, k
    for k_gpu, k_e, k_s in (("dEdeps", "dEde", "dEds"), ("dLdeps", "dLde", "dLds")):
        ge, gs = type_grads(ref[k_e], ref[k_s], s.eps, s.sigma)
        kk = "dEdsig" if k_gpu == "dEdeps" else "dLdsig"
        fin = np.isfinite(ge)
        assert np.allclose(g[k_gpu][fin], ge[fin], rtol=1e-10, atol=1e-10 * (np.abs(ge[fin]).max() + 1e-300))
        assert np.allclose(g[kk], gs, rtol=1e-10, atol=1e-10 * (np.abs(gs).max() + 1e-300))
    # mixed precision against FP64 on identical draws
    gm = _ctx(s, rbe.MIXED).adjoint(step, d["pos"], d["q"], d["typ"], d["mol"], torch.tensor(v, device="cuda"))
    for k in ("dEdq", "dLdq"):
        e = rms_rel(gm[k].cpu().numpy(), g[k].cpu().numpy())
        print(f"{name} {k}: mixed RMS rel err {e:.2e}")
        assert e < 1e-4


def test_force_matching_gradients_by_finite_differences():
    """L = sum |F - F_ref|^2 over a 12,000-atom water box; F_ref from the
    exact Ewald oracle at q_O + 2% (H rescaled to stay neutral) and eps + 5%.
    Autograd gradients w.r.t. charges and LJ parameters against central
    differences of the FP64 GPU forward with the draws frozen."""
    import torch
    s = systems.water(4000, seed=4)
    q_ref = s.q.copy()
    q_ref[0::3] *= 1.02
    q_ref[1::3] = -0.5 * q_ref[0::3]
    q_ref[2::3] = -0.5 * q_ref[0::3]
    eps_ref = (s.eps[0] * 1.05, s.eps[1])
    pr = oracle.make_params(s.L, s.alpha, s.r_c, s.r_s, s.p, s.P, 1, k_e=s.k_e, eps=eps_ref, sigma=s.sigma)
    kmax = int(math.ceil(math.sqrt(30.0 * s.alpha * s.L**2) / math.pi)) + 1
    F_ref = torch.tensor(oracle.ewald_exact(s.pos, q_ref, s.type, s.mol, pr, s.r_s, kmax)["F"], device="cuda")
    d = to_dev(s)
    ctx = _ctx(s)
    step = 9

    def loss(q, eps, sig):
        F, E = rbe.RbeForces.apply(ctx, step, d["pos"], q, d["typ"], d["mol"], eps, sig)
        return ((F - F_ref) ** 2).sum()

    q = d["q"].clone().requires_grad_(True)
    eps = torch.tensor(s.eps, dtype=torch.float64, requires_grad=True)
    sig = torch.tensor(s.sigma, dtype=torch.float64, requires_grad=True)
    L0 = loss(q, eps, sig)
    L0.backward()
    h = 1e-6
    with torch.no_grad():
        # charge derivatives along neutral directions (q_m + h, q_m2 - h), so
        # that every perturbed system stays neutral: the derivative is
        # dL/dq_m - dL/dq_m2
        for m, m2 in ((0, 1), (1, 2), (2, 6000), (6000, 11999), (11999, 5)):
            qp, qm = d["q"].clone(), d["q"].clone()
            qp[m] += h
            qp[m2] -= h
            qm[m] -= h
            qm[m2] += h
            fd = (loss(qp, eps.detach(), sig.detach()) - loss(qm, eps.detach(), sig.detach())).item() / (2 * h)
            ad = q.grad[m].item() - q.grad[m2].item()
            print(f"dL/dq[{m}] - dL/dq[{m2}] autograd {ad:.8e} fd {fd:.8e}")
            assert ad == pytest.approx(fd, rel=2e-5, abs=1e-6 * abs(L0.item()))
        for name, par, grad in (("eps", eps, eps.grad), ("sigma", sig, sig.grad)):
            hp = 1e-6 * par[0].item()
            pp, pm = par.detach().clone(), par.detach().clone()
            pp[0] += hp
            pm[0] -= hp
            args_p = (d["q"], pp, sig.detach()) if name == "eps" else (d["q"], eps.detach(), pp)
            args_m = (d["q"], pm, sig.detach()) if name == "eps" else (d["q"], eps.detach(), pm)
            fd = (loss(*args_p) - loss(*args_m)).item() / (2 * hp)
            print(f"dL/d{name}_O autograd {grad[0].item():.8e} fd {fd:.8e}")
            assert grad[0].item() == pytest.approx(fd, rel=2e-5)
    assert ctx.sync_status() == rbe.OK
