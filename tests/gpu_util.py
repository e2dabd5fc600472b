"""Shared helpers of the GPU parity tests: run the CUDA path through the C ABI
and the oracle on the same seeded inputs."""
from __future__ import annotations

import numpy as np

import oracle
from paper_2204_13595_gb300 import rbe, systems


def params(s, p=None, P=None, seed=None):
    return oracle.make_params(s.L, s.alpha, s.r_c, s.r_s, s.p if p is None else p, s.P if P is None else P,
                              s.seed if seed is None else seed, k_e=s.k_e, eps=s.eps, sigma=s.sigma)


def to_dev(s):
    import torch
    d = dict(pos=torch.tensor(s.pos, dtype=torch.float64, device="cuda"),
             q=torch.tensor(s.q, dtype=torch.float64, device="cuda"),
             typ=torch.tensor(s.type, dtype=torch.int32, device="cuda"),
             mol=None if s.mol is None else torch.tensor(s.mol, dtype=torch.int32, device="cuda"))
    return d


def gpu_forces(s, step, precision=rbe.FP64, p=None, P=None, seed=None, debug_cap=0, bonds=False, ctx=None,
               dev=None, with_type=True):
    import torch
    if ctx is None:
        ctx = rbe.Context(s.L, s.alpha, s.r_c, s.r_s, s.p if p is None else p, s.P if P is None else P,
                          s.seed if seed is None else seed, k_e=s.k_e, eps=s.eps, sigma=s.sigma,
                          precision=precision)
        if bonds and s.n_water_mol:
            ctx.set_water_bonds(s.n_water_mol, *s.bonds)
        if debug_cap:
            ctx.set_debug(True, debug_cap)
    d = dev or to_dev(s)
    F = torch.empty_like(d["pos"])
    E = torch.zeros(rbe.NE, dtype=torch.float64, device="cuda")
    W = torch.zeros(rbe.NW, dtype=torch.float64, device="cuda")
    ctx.forces(step, d["pos"], d["q"], d["typ"] if with_type else None, d["mol"], F, E, W)
    status = ctx.sync_status()
    out = dict(F=F.cpu().numpy(), E=E.cpu().numpy(), W=W.cpu().numpy(), status=status, ctx=ctx)
    if debug_cap:
        out["lists"] = ctx.get_lists(s.n, debug_cap)
    out["m"], out["rho"] = ctx.get_kspace()
    return out


def rel_err_components(a, ref, floor_frac=1e-3):
    """max |a - ref| / (|ref| + floor_frac * rms(ref)) over components."""
    rms = np.sqrt(np.mean(ref * ref))
    return float(np.max(np.abs(a - ref) / (np.abs(ref) + floor_frac * rms)))


def cond_err(F, ref):
    """max over components of |F - F_ref| / A, A = sum of |summands| of that
    component (pair terms, momentum correction, k terms) from the oracle: the
    componentwise error measure of a floating-point sum."""
    return float(np.max(np.abs(F - ref["F"]) / ref["F_abs"]))


def literal_stats(F, ref):
    """How the FP64 forces fare against a plain per-component relative bar:
    quantiles (50, 90, 99, 99.9 %, max) of |F - F_ref| / |F_ref| and of the
    condition number A / |F_ref| (A: the sum of |summands|), and the fraction
    of components within 1e-11 relative."""
    d = np.abs(F - ref["F"]).ravel()
    f = np.abs(ref["F"]).ravel()
    a = ref["F_abs"].ravel()
    rel = d / np.maximum(f, 1e-300)
    cond = a / np.maximum(f, 1e-300)
    qs = (50, 90, 99, 99.9, 100)
    return {"rel_q": [float(np.percentile(rel, q)) for q in qs],
            "cond_q": [float(np.percentile(cond, q)) for q in qs],
            "frac_within_1e-11": float(np.mean(rel <= 1e-11))}


def ek_scale(s, ref, P=None):
    """Condition scale of E_k = sum_l c_l/2 |rho_l|^2 under perturbations of
    rho_l bounded by the sum of |q_j|: sum_l c_l |rho_l| sum_j |q_j|."""
    P = len(ref["m"]) if P is None else P
    k = 2 * np.pi * ref["m"] / s.L
    k2 = (k * k).sum(1)
    c = oracle.S(s.alpha, s.L) / P * 4 * np.pi * s.k_e / (s.L ** 3 * k2)
    return float((c * np.abs(ref["rho"])).sum() * np.abs(s.q).sum())


def rms_rel(a, ref):
    return float(np.sqrt(np.mean((a - ref) ** 2)) / np.sqrt(np.mean(ref ** 2)))


__all__ = ["params", "to_dev", "gpu_forces", "rel_err_components", "rms_rel", "cond_err", "ek_scale", "literal_stats",
           "systems", "oracle", "rbe"]


def type_grads(g_eps, g_sig, eps, sigma):
    """Lorentz-Berthelot chain rule from the oracle's ordered pair-table
    gradients to per-type eps and sigma gradients."""
    T = len(eps)
    ge, gs = np.zeros(T), np.zeros(T)
    for a in range(T):
        for b in range(T):
            if a == b:
                ge[a] += g_eps[a, a]
                gs[a] += g_sig[a, a]
                continue
            sym_e = g_eps[a, b] + g_eps[b, a]
            sym_s = g_sig[a, b] + g_sig[b, a]
            if sym_e != 0.0:
                ge[a] += sym_e * (0.0 if eps[b] == 0.0 else (np.inf if eps[a] == 0.0 else eps[b] / (2 * np.sqrt(eps[a] * eps[b]))))
            gs[a] += 0.5 * sym_s
    return ge, gs
