"""Command-line driver: runs IRBE force evaluations on a synthetic system.

  python run.py --system water --n-mol 400000 \\
         --precision mixed --steps 3 [--warmup 1] [--profile] [--skin 1.0]

Prints the mean time per force evaluation (CUDA events on the launching
stream) and, with --profile, the per-kernel launch times the library records.
Used for profiler captures of a fixed number of launches.
"""
from __future__ import annotations

import argparse
import json
import os
import sys

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main(argv=None):
    import torch

    from paper_2204_13595_gb300 import build, rbe, systems
    ap = argparse.ArgumentParser()
    ap.add_argument("--system", default="water", choices=["water", "electrolyte"])
    ap.add_argument("--n-mol", type=int, default=400000, help="water molecules (water) or ions (electrolyte)")
    ap.add_argument("--seed", type=int, default=3)
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=1)
    ap.add_argument("--profile", action="store_true")
    ap.add_argument("--skin", type=float, default=0.0,
                    help="Verlet skin in length units (0: lists every step); the first call builds the stored lists")
    a = ap.parse_args(argv)
    build.build()
    if a.system == "water":
        s = systems.water(a.n_mol, seed=a.seed)
    else:
        L = (a.n_mol / 0.25) ** (1.0 / 3.0)
        s = systems.electrolyte(n=a.n_mol, L=L, seed=a.seed)
    ctx = rbe.Context(s.L, s.alpha, s.r_c, s.r_s, s.p, s.P, a.seed, k_e=s.k_e, eps=s.eps, sigma=s.sigma,
                      precision=rbe.MIXED if a.precision == "mixed" else rbe.FP64)
    if a.skin > 0:
        ctx.set_verlet_skin(a.skin)
    dev = lambda x, dt=torch.float64: torch.tensor(x, dtype=dt, device="cuda")
    pos, q, typ = dev(s.pos), dev(s.q), dev(s.type, torch.int32)
    mol = None if s.mol is None else dev(s.mol, torch.int32)
    F = torch.empty_like(pos)
    for w in range(a.warmup):
        ctx.forces(w, pos, q, typ, mol, F)
    if ctx.sync_status() != 0:
        raise SystemExit("device status error")
    ctx.set_profiling(a.profile)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for k in range(a.steps):
        ctx.forces(a.warmup + k, pos, q, typ, mol, F)
    e1.record()
    e1.synchronize()
    out = {"system": a.system, "n_atoms": s.n, "precision": a.precision, "steps": a.steps,
           "ms_per_step": e0.elapsed_time(e1) / max(a.steps, 1), "info": ctx.info()}
    if a.profile:
        out["kernels_ms"] = {k: v for k, v in ctx.profile().items() if v[1]}
    if ctx.sync_status() != 0:
        raise SystemExit("device status error")
    print(json.dumps(out))


if __name__ == "__main__":
    main()
