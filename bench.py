#!/usr/bin/env python3
"""Benchmark of the IRBE (RBL + RBE) force step on GB300.

Workload: the 1.2M-atom water-like system (400,000 rigid-geometry 3-site
molecules at 0.0334 / A^3, L = 228.79 A, r_c = 5 A, r_s = 10 A, p = 20,
P = 200, alpha from erfc(sqrt(alpha) r_s) = 1e-4), seeded synthetic inputs.
A step is one full force evaluation (rbe_forces: cell sort, lists and shell
batches, pair forces, k sampling, rho(k), Fourier forces, momentum
correction, energies and virial).  The headline is the mixed-precision path
(FP32 pair/phase arithmetic, FP64 positions and sums), whose force RMS error
against the FP64 path on identical draws is measured in the same run; the
FP64 path is timed beside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

The same line carries a "batch" object: 64 independent replicas of uneven
size (1,000 to 50,000 atoms, log-uniform, electrolyte and water, each its own
box, alpha and P) stepped together for 500 velocity-Verlet steps by the
batched path (one launch per stage, a persistent pair kernel over all
replicas, one CUDA graph per step, tiling autotuned), against looping the
single-system rbe_step over the replicas; aggregate atom-steps/s of both.  A
"next_rows" object times the adjoint (12,000-atom water), the method variants
(1.2M atoms) and Langevin dynamics of the paper's 5,120-ion electrolyte.

--impl reference times the plain CPU oracle (the same estimator in FP64 C)
on the host cores, one full force evaluation of the same system per step.
Under torchrun every rank runs an independent replica (the path does not
shard: replicas only); rank 0 prints the JSON line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "RBE+RBL force evals/s at 1.2M atoms (mixed precision at <=1e-4 force RMS error vs FP64)"
UNIT = "force_evals/s"
N_MOL = 400000
SEED = 3
DT_FS = 1.0
L2_FLUSH_BYTES = 512 << 20
# algorithmic work of the RBL kernel per atom: 420 pair classifications x 9
# ops + 72.5 pair evaluations x 45 ops (core 52.5 + p = 20), in lane ops
RBL_OPS_PER_ATOM = 420 * 9 + 72.5 * 45
# Eq. (2.10) terms per atom (52.5 core + p = 20 batch members) and counted
# operations per term: the part of RBL_OPS_PER_ATOM that the FP64 path
# computes in FP64 (its classification is FP32 and integer, as on the mixed path)
RBL_PAIRS_PER_ATOM, RBL_OPS_PER_PAIR = 72.5, 45
SM_COUNT = 152
LANES_PER_SM = 128
SFU_LANES_PER_SM = 16
SM_MAX_MHZ = 2070.0
HBM_FALLBACK_GBS = 6800.0


PROBES = {"ffma": 0, "dfma": 1, "sfu": 2, "alu": 3, "copy": 4}
PROBE_SRC = os.path.join(ROOT, "bench_probes.cu")
PROBE_LIB = os.path.join(ROOT, "_build", "libbench_probes.so")


def build_probes() -> str:
    """Compiles bench_probes.cu (the pipe and copy throughput probes, not part
    of librbe.so) into _build/libbench_probes.so when stale."""
    if os.path.exists(PROBE_LIB) and os.path.getmtime(PROBE_LIB) >= os.path.getmtime(PROBE_SRC):
        return PROBE_LIB
    from paper_2204_13595_gb300 import build as b
    os.makedirs(os.path.dirname(PROBE_LIB), exist_ok=True)
    tmp = PROBE_LIB + ".tmp"
    cmd = [b.nvcc()] + b.ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-shared", PROBE_SRC,
                                 "-o", tmp, "-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for bench_probes.cu:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, PROBE_LIB)
    return PROBE_LIB


_probe_lib = None


def peak_probe(kind, stream=None):
    """Measured throughput of a pipe ('ffma', 'dfma', 'sfu', 'alu': operations
    per second) or of device memory ('copy': bytes per second), from
    bench_peak_probe of libbench_probes.so."""
    import ctypes
    global _probe_lib
    if _probe_lib is None:
        _probe_lib = ctypes.CDLL(build_probes())
        _probe_lib.bench_peak_probe.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_double), ctypes.c_void_p]
    if stream is None:
        import torch
        stream = torch.cuda.current_stream().cuda_stream
    out = ctypes.c_double()
    rc = _probe_lib.bench_peak_probe(PROBES[kind], ctypes.byref(out), stream)
    if rc != 0:
        raise RuntimeError(f"bench_peak_probe({kind}) failed: {rc}")
    return out.value


def _kernel_roofline(prof, n, P, ncells, peaks_meas):
    """Roofline fraction of every kernel of the mixed step (per-launch CUDA-event
    times from the library's profiler).  Denominators: HBM from MEASURED_PEAKS.json
    if present, else the recipe's fallback; the FP32 lane and special-function
    peaks derived from the unit counts and the maximum SM clock."""
    peaks, src = _peaks()
    hbm = float(peaks.get("hbm_gbs", HBM_FALLBACK_GBS))
    lane = SM_COUNT * LANES_PER_SM * SM_MAX_MHZ * 1e6
    sfu = SM_COUNT * SFU_LANES_PER_SM * SM_MAX_MHZ * 1e6
    work = {   # algorithmic bytes or operations per launch
        "quantize": ("hbm", 48.0 * n),                       # pos, q in; cell, slot, x code out
        "scan": ("hbm", 12.0 * ncells),                      # counts read twice, starts written
        "scatter": ("hbm", 24.0 * n),                        # cell, slot, x code, start in; key out
        "sort": ("hbm", 20.0 * n + 8.0 * ncells),            # keys read and written, perm out
        "gather": ("hbm", 116.0 * n),                        # perm, pos, q, type, mol in; s4 f4 p4 tm out
        "rho": ("sfu", 2.0 * n * P),                         # one FP32 sincos per (atom, k)
        "kforce": ("sfu", 2.0 * n * P),
        "rbl": ("alu", RBL_OPS_PER_ATOM * n),
    }
    out = {}
    for k, (bound, w) in work.items():
        ms, cnt = prof.get(k, (0.0, 0))
        if not cnt:
            continue
        t = ms / cnt * 1e-3
        if bound == "hbm":
            a = w / t / 1e9
            out[k] = {"bound": "hbm", "achieved": a, "peak": hbm, "unit": "GB/s", "frac": a / hbm,
                      "peak_source": f"{src} HBM"}
        elif bound == "sfu":
            a = w / t / 1e12
            out[k] = {"bound": "sfu", "achieved": a, "peak": sfu / 1e12, "unit": "Top/s", "frac": a / (sfu / 1e12),
                      "peak_source": "derived: 152 SMs x 16 SFU lanes x 2070 MHz"}
        else:
            a = w / t / 1e12
            out[k] = {"bound": "alu", "achieved": a, "peak": lane / 1e12, "unit": "Top/s", "frac": a / (lane / 1e12),
                      "peak_source": "derived: 152 SMs x 128 lanes x 2070 MHz"}
        out[k]["avg_launch_ms"] = t * 1e3
    for k in ("rhosum", "finalize", "ksample"):
        ms, cnt = prof.get(k, (0.0, 0))
        if cnt:
            out[k] = {"bound": "latency", "avg_launch_ms": ms / cnt}
    return out


def _fp64_rbl_roofline(prof64, n, meas):
    """The FP64 path's pair kernel against the measured FP64 FMA rate of this
    GPU (bench_peak_probe 'dfma'): the counted FP64 operations of the pair
    terms per launch over its CUDA-event time.  The library erfc, exp and
    reciprocal square root take several FP64 instructions per counted
    operation, so the FP64 pipe is far busier than this fraction says."""
    ms, cnt = prof64.get("rbl", (0.0, 0)) if prof64 else (0.0, 0)
    peak = meas.get("dfma")
    if not cnt or not isinstance(peak, float):
        return None
    t = ms / cnt * 1e-3
    a = RBL_PAIRS_PER_ATOM * RBL_OPS_PER_PAIR * n / t
    return {"bound": "fp64", "achieved": a / 1e12, "peak": peak / 1e12, "unit": "Top/s", "frac": a / peak,
            "peak_source": "measured: bench_peak_probe dfma in this run", "avg_launch_ms": t * 1e3}


def _dist():
    from paper_2204_13595_gb300 import replicas
    ws, rank, _ = replicas.world()
    return ws, rank


def _workload_config(s):
    return {"workload": f"water-like {s.n} atoms ({s.n // 3} 3-site molecules), L={s.L:.3f} A, "
                        f"r_c={s.r_c} A, r_s={s.r_s} A, p={s.p}, P={s.P}, alpha={s.alpha:.6f} A^-2",
            "n_atoms": s.n, "r_c": s.r_c, "r_s": s.r_s, "p": s.p, "P": s.P,
            "l2": "flushed between timed steps (512 MB write, outside the timed region)",
            "step": "one rbe_forces call (one force evaluation)"}


def _clock_sampler():
    q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")
    try:
        return subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits", "-lms", "200"],
                                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
    except OSError:
        return None


def _clock_summary(proc, dev_index):
    if proc is None:
        return None
    proc.terminate()
    try:
        out, _ = proc.communicate(timeout=5)
    except subprocess.TimeoutExpired:
        proc.kill()
        out, _ = proc.communicate()
    sm, mx, reasons = [], [], set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for line in out.splitlines():
        f = [x.strip() for x in line.split(",")]
        if len(f) < 9 or f[0] != str(dev_index):
            continue
        try:
            sm.append(float(f[1]))
            mx.append(float(f[2]))
        except ValueError:
            continue
        for nm, v in zip(names, f[5:9]):
            if v.lower() == "active":
                reasons.add(nm)
    if not sm:
        return None
    return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
            "samples": len(sm)}


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        try:
            return json.load(open(path)), "measured"
        except (OSError, ValueError):
            pass
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def _traffic(kernel_src):
    """DRAM bytes per launch of the RBL kernel from the committed ncu summary,
    if it was taken on the current kernel source."""
    path = os.path.join(ROOT, "profiles", "rbl_traffic.json")
    if not os.path.exists(path):
        return None
    try:
        rec = json.load(open(path))
    except (OSError, ValueError):
        return None
    sha = hashlib.sha256(open(kernel_src, "rb").read()).hexdigest()
    if rec.get("source_sha256") != sha or rec.get("precision") != "mixed":
        return None
    return rec.get("dram_bytes_per_launch_full")


def run_reference(args):
    import numpy as np  # noqa: F401
    import oracle
    from paper_2204_13595_gb300 import systems
    ws, rank = _dist()
    if rank != 0:
        return 0
    oracle.build()
    s = systems.water(N_MOL, seed=SEED)
    pr = oracle.make_params(s.L, s.alpha, s.r_c, s.r_s, s.p, s.P, SEED, k_e=s.k_e, eps=s.eps, sigma=s.sigma)
    for w in range(args.warmup):
        oracle.rbe_forces(s.pos, s.q, s.type, s.mol, pr, w)
    t0 = time.perf_counter()
    for k in range(args.steps):
        oracle.rbe_forces(s.pos, s.q, s.type, s.mol, pr, args.warmup + k)
    dt = (time.perf_counter() - t0) / args.steps
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    v = 1.0 / dt
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": _workload_config(s),
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": "one full FP64 oracle force evaluation of the 1.2M-atom system per step"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


BATCH_STEPS = 500


def _batch_leg(flush):
    """64-replica batched stepping against the looped single-system path."""
    import torch

    from paper_2204_13595_gb300 import rbe, systems

    t0 = time.perf_counter()
    suite = systems.batch_replicas()
    gen_s = time.perf_counter() - t0
    dev = lambda a, dt=torch.float64: torch.tensor(a, dtype=dt, device="cuda")

    def state():
        return [dict(pos=dev(x.pos), vel=dev(x.vel), mass=dev(x.mass), q=dev(x.q), typ=dev(x.type, torch.int32),
                     mol=None if x.mol is None else dev(x.mol, torch.int32),
                     F=torch.zeros((x.n, 3), dtype=torch.float64, device="cuda")) for x in suite]

    ctxs = [rbe.Context.for_system(x, precision=rbe.MIXED) for x in suite]
    A, B = state(), state()
    bt = rbe.Batch(ctxs)
    bt.bind([d["pos"] for d in A], [d["q"] for d in A], [d["typ"] for d in A], [d["mol"] for d in A],
            [d["F"] for d in A], vel=[d["vel"] for d in A], mass=[d["mass"] for d in A],
            dt=[x.dt for x in suite], accel=[x.accel for x in suite])
    t0 = time.perf_counter()
    tune = bt.autotune(step=0)
    tune_s = time.perf_counter() - t0
    natoms = sum(x.n for x in suite)
    stream = torch.cuda.current_stream()

    # batched: warm-up, then BATCH_STEPS graph replays, each timed with events
    # on the stream, L2 flushed between replays (outside the events)
    bt.forces(0)
    bt.step(0, 3)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(BATCH_STEPS)]
    for k in range(BATCH_STEPS):
        flush.fill_(float(k))
        ev[k][0].record(stream)
        bt.step(3 + k, 1)
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    batched_ms = sum(a.elapsed_time(b) for a, b in ev) / BATCH_STEPS
    if bt.sync_status()[0] != 0:
        raise RuntimeError("device status error in the batched run")

    # looped single-system path on an identical copy: per replica rbe_step
    # over the same steps (the loop inside the library), one timed region
    for x, c, d in zip(suite, ctxs, B):
        c.forces(0, d["pos"], d["q"], d["typ"], d["mol"], d["F"])
        c.step(0, 3, x.dt, x.accel, d["pos"], d["vel"], d["mass"], d["q"], d["typ"], d["mol"], d["F"])
    torch.cuda.synchronize()
    flush.fill_(0.0)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for x, c, d in zip(suite, ctxs, B):
        c.step(3, BATCH_STEPS, x.dt, x.accel, d["pos"], d["vel"], d["mass"], d["q"], d["typ"], d["mol"], d["F"])
    e1.record(stream)
    torch.cuda.synchronize()
    looped_ms = e0.elapsed_time(e1) / BATCH_STEPS
    same = all(torch.equal(a["pos"], b["pos"]) and torch.equal(a["F"], b["F"]) for a, b in zip(A, B))
    info = bt.info()
    bt.close()
    return {
        "workload": "64 replicas, 1,000-50,000 atoms log-uniform (electrolyte P=100 / water P=200), mixed, "
                    f"{BATCH_STEPS} velocity-Verlet steps",
        "replicas": len(suite), "atoms": natoms, "steps": BATCH_STEPS,
        "atom_steps_per_s": natoms * 1e3 / batched_ms, "ms_per_step": batched_ms,
        "looped_atom_steps_per_s": natoms * 1e3 / looped_ms, "looped_ms_per_step": looped_ms,
        "speedup_vs_looped": looped_ms / batched_ms,
        "bitwise_equal_to_looped": bool(same),
        "launches_per_step": int(info["launches_per_step"]), "pair_tasks": int(info["tasks"]),
        "autotune": tune, "autotune_s": tune_s, "generate_s": gen_s,
        "timing": "batched: CUDA events per graph replay, L2 flushed between replays; looped: one event pair "
                  "around all replicas' rbe_step calls",
    }


def _configs_leg(flush):
    """The other configurations' lines (each after its own warm-up, CUDA
    events on the launching stream, L2 flushed between timed calls):
    the 2,000-ion 1:1 electrolyte in FP64 (one force evaluation, then 100
    velocity-Verlet NVE steps at dt = 0.002 tau, in tau/day) with the force
    RMS error of the estimator against a converged exact Ewald sum of the
    oracle; the 90,000-atom water box in FP64 (force evaluations and 100
    velocity-Verlet steps at 1 fs)."""
    import numpy as np
    import torch

    import oracle
    from paper_2204_13595_gb300 import rbe, systems

    stream = torch.cuda.current_stream()
    dev = lambda a, dt=torch.float64: torch.tensor(a, dtype=dt, device="cuda")

    def timed(fn, n):
        tot = 0.0
        for k in range(n):
            flush.fill_(float(k))
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn(k)
            e1.record(stream)
            e1.synchronize()
            tot += e0.elapsed_time(e1)
        return tot / n

    out = {}
    for key, s, nsteps, unit_day in (("electrolyte_2000_fp64", systems.electrolyte(), 100, "tau_per_day"),
                                     ("water_90k_fp64", systems.water(30000, seed=2), 100, "ns_per_day")):
        c = rbe.Context.for_system(s, precision=rbe.FP64)
        d = dict(pos=dev(s.pos), vel=dev(s.vel), mass=dev(s.mass), q=dev(s.q), typ=dev(s.type, torch.int32),
                 mol=None if s.mol is None else dev(s.mol, torch.int32))
        F = torch.empty_like(d["pos"])
        for k in range(3):
            c.forces(k, d["pos"], d["q"], d["typ"], d["mol"], F)
        f_ms = timed(lambda k: c.forces(3 + k, d["pos"], d["q"], d["typ"], d["mol"], F), 10)
        c.forces(0, d["pos"], d["q"], d["typ"], d["mol"], F)
        F0 = F.cpu().numpy()
        s_ms = timed(lambda k: c.step(0, nsteps, s.dt, s.accel, d["pos"], d["vel"], d["mass"], d["q"], d["typ"],
                                      d["mol"], F), 1) / nsteps
        if c.sync_status() != 0:
            raise RuntimeError(f"device status error in the {key} leg")
        steps_per_s = 1e3 / s_ms
        row = {"n_atoms": s.n, "force_evals_per_s": 1e3 / f_ms, "force_ms": f_ms, "steps": nsteps,
               "md_ms_per_step": s_ms, "md_steps_per_s": steps_per_s,
               unit_day: steps_per_s * s.dt * 86400.0 * (1e-6 if unit_day == "ns_per_day" else 1.0)}
        if key.startswith("electrolyte"):
            # the method's own (stochastic) error: the estimator at step 0
            # against real space to r_s plus the full reciprocal sum
            pr = oracle.make_params(s.L, s.alpha, s.r_c, s.r_s, s.p, s.P, s.seed, k_e=s.k_e, eps=s.eps,
                                    sigma=s.sigma)
            kmax = int(np.ceil(np.sqrt(46.0 * s.alpha * s.L ** 2) / np.pi)) + 1
            t0 = time.perf_counter()
            ex = oracle.ewald_exact(s.pos, s.q, s.type, s.mol, pr, s.r_s, kmax)["F"]
            row["exact_ewald_s"] = time.perf_counter() - t0
            row["force_rms_rel_err_vs_exact_ewald"] = float(np.sqrt(((F0 - ex) ** 2).mean() / (ex ** 2).mean()))
        out[key] = row
        c.close()
    return out


def _oracle_timings():
    """The oracle on one host core (a subprocess with OMP_NUM_THREADS=1): one
    full FP64 force evaluation of the 1.2M-atom water box; and the exact Ewald
    sum (real space to r_s, the full reciprocal sum to a 1e-20 tail) of the
    12,000-atom water box on all host cores."""
    import numpy as np

    import oracle
    from paper_2204_13595_gb300 import systems
    code = ("import sys,time; sys.path.insert(0, %r)\n"
            "import oracle\nfrom paper_2204_13595_gb300 import systems\n"
            "s = systems.water(%d, seed=%d)\n"
            "pr = oracle.make_params(s.L, s.alpha, s.r_c, s.r_s, s.p, s.P, %d, k_e=s.k_e, eps=s.eps, sigma=s.sigma)\n"
            "t0 = time.perf_counter(); oracle.rbe_forces(s.pos, s.q, s.type, s.mol, pr, 0)\n"
            "print(time.perf_counter() - t0)\n") % (ROOT, N_MOL, SEED, SEED)
    env = dict(os.environ, OMP_NUM_THREADS="1")
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=900)
    one = float(r.stdout.strip().splitlines()[-1]) if r.returncode == 0 else None
    w = systems.water(4000, seed=4)
    pr = oracle.make_params(w.L, w.alpha, w.r_c, w.r_s, w.p, w.P, 4, k_e=w.k_e, eps=w.eps, sigma=w.sigma)
    kmax = int(np.ceil(np.sqrt(46.0 * w.alpha * w.L ** 2) / np.pi)) + 1
    t0 = time.perf_counter()
    oracle.ewald_exact(w.pos, w.q, w.type, w.mol, pr, w.r_s, kmax)
    ex_s = time.perf_counter() - t0
    return {"oracle_1core_water_1p2M": {"force_evals_per_s": (1.0 / one) if one else None, "seconds": one,
                                        "cores": 1},
            "exact_ewald_water_12k": {"seconds": ex_s, "kmax": kmax,
                                      "cores": int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))}}


def _next_rows_leg(flush, big):
    """Timing of the widened rows beside the headline (each after its own
    warm-up, CUDA events on the launching stream): the adjoint at frozen draws
    (row f1) on the 12,000-atom water box of the differentiation workload
    against the forward call on the same box; the method variants (row f3) on
    the 1.2M-atom box; Langevin dynamics (row f4) on the paper's 5,120-ion 1:1
    electrolyte with WCA soft spheres (Sec. 3.1)."""
    import numpy as np
    import torch

    from paper_2204_13595_gb300 import rbe, systems

    stream = torch.cuda.current_stream()
    dev = lambda a, dt=torch.float64: torch.tensor(a, dtype=dt, device="cuda")

    def events(fn, n):
        tot = 0.0
        for k in range(n):
            flush.fill_(float(k))
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn(k)
            e1.record(stream)
            e1.synchronize()
            tot += e0.elapsed_time(e1)
        return tot / n

    out = {}
    # f1: adjoint (dE/dq, dL/dq, dL/d(eps, sigma) of L = sum gF . F) at frozen draws
    w = systems.water(4000, seed=4)
    pos, q, typ, mol = dev(w.pos), dev(w.q), dev(w.type, torch.int32), dev(w.mol, torch.int32)
    gF = dev(np.random.default_rng(4).normal(size=w.pos.shape))
    F = torch.empty_like(pos)
    adj = {"workload": "water-like 12,000 atoms (4,000 molecules, seed 4), r_c=5, r_s=10, p=20, P=200; "
                       "frozen draws (same step)"}
    for name, prec in (("mixed", rbe.MIXED), ("fp64", rbe.FP64)):
        c = rbe.Context.for_system(w, precision=prec)
        for k in range(3):
            c.forces(7, pos, q, typ, mol, F)
            c.adjoint(7, pos, q, typ, mol, gF)
        f_ms = events(lambda k: c.forces(7, pos, q, typ, mol, F), 10)
        a_ms = events(lambda k: c.adjoint(7, pos, q, typ, mol, gF), 10)
        if c.sync_status() != 0:
            raise RuntimeError("device status error in the adjoint leg")
        adj[name] = {"forces_ms": f_ms, "adjoint_ms": a_ms, "adjoint_over_forces": a_ms / f_ms}
        c.close()
    out["adjoint"] = adj

    # f3: variants of the method on the 1.2M-atom box (mixed)
    s, bpos, bq, btyp, bmol = big
    F = torch.empty_like(bpos)
    var = {"workload": "the headline's 1.2M-atom water box, mixed"}
    for name, setup in (("shell_with_replacement", lambda c: c.set_shell_sampling(rbe.SHELL_REPLACE)),
                        ("k_pool_mh_4096", lambda c: c.set_kpool(4096, 64))):
        c = rbe.Context(s.L, s.alpha, s.r_c, s.r_s, s.p, s.P, SEED, k_e=s.k_e, eps=s.eps, sigma=s.sigma,
                        precision=rbe.MIXED)
        setup(c)
        for k in range(3):
            c.forces(k, bpos, bq, btyp, bmol, F)
        ms = events(lambda k: c.forces(3 + k, bpos, bq, btyp, bmol, F), 5)
        if c.sync_status() != 0:
            raise RuntimeError("device status error in the variants leg")
        var[name] = {"force_evals_per_s": 1e3 / ms, "ms_per_step": ms}
        c.close()
    # Verlet skin (row f3): the cost of a force evaluation from valid stored
    # lists (static positions), of one that rebuilds them, and of
    # velocity-Verlet steps (bonded water, NVE, 1 fs, rebuilds as they come),
    # each against the same with lists every step
    skin = {"workload": "the headline's 1.2M-atom water box, mixed; MD: NVE velocity Verlet at 1 fs with bonds after "
                        "5 warm-up steps, stored lists rebuilt when an atom moved more than skin/2"}
    nmd = 40
    for sk in (0.0, 1.0, 2.0):
        c = rbe.Context.for_system(s, precision=rbe.MIXED)
        if sk > 0:
            c.set_verlet_skin(sk)
        for k in range(3):
            c.forces(k, bpos, bq, btyp, bmol, F)
        static_ms = events(lambda k: c.forces(3 + k, bpos, bq, btyp, bmol, F), 5)
        row = {"static_force_ms": static_ms}
        if sk > 0:
            def rebuild(k):
                c.set_verlet_skin(sk)            # the next call rebuilds
                c.forces(20 + k, bpos, bq, btyp, bmol, F)
            row["rebuild_force_ms"] = events(rebuild, 3)
        d = dict(pos=bpos.clone(), vel=dev(s.vel), mass=dev(s.mass))
        c.forces(0, d["pos"], bq, btyp, bmol, F)
        c.step(0, 5, s.dt, s.accel, d["pos"], d["vel"], d["mass"], bq, btyp, bmol, F)
        r0 = c.info()["skin_rebuilds"]
        ms = events(lambda k: c.step(5, nmd, s.dt, s.accel, d["pos"], d["vel"], d["mass"], bq, btyp, bmol, F),
                    1) / nmd
        if c.sync_status() != 0:
            raise RuntimeError("device status error in the Verlet-skin leg")
        info = c.info()
        row.update({"md_ms_per_step": ms, "md_ns_per_day": 0.0864 * 1e3 / ms * s.dt,
                    "md_rebuilds": int(info["skin_rebuilds"] - r0), "md_steps": nmd,
                    "stored_list_entries": int(info["skin_vcap"]) if sk > 0 else 0})
        skin[f"skin_{sk:g}A"] = row
        c.close()
    base = skin["skin_0A"]["static_force_ms"]
    for sk in (1.0, 2.0):
        r = skin[f"skin_{sk:g}A"]
        gain = base - r["static_force_ms"]
        r["break_even_steps_between_rebuilds"] = (r["rebuild_force_ms"] - r["static_force_ms"]) / gain if gain > 0 else None
    var["verlet_skin"] = skin
    out["variants"] = var

    # f4: Langevin dynamics of the paper's 1:1 electrolyte (WCA, kT = 1, tau = 1)
    e = systems.electrolyte(n=5120, L=80.0, seed=21, r_c=5.0, r_s=15.0, p=10, P=100, dt=0.002)
    c = rbe.Context(e.L, 0.03, e.r_c, e.r_s, e.p, e.P, 21, k_e=e.k_e, eps=e.eps, sigma=e.sigma, shift_lj=True,
                    precision=rbe.MIXED)
    c.set_lj_cutoff(2.0 ** (1.0 / 6.0))
    c.set_langevin(1.0, 1.0)
    d = dict(pos=dev(e.pos), vel=dev(e.vel), mass=dev(e.mass), q=dev(e.q), typ=dev(e.type, torch.int32),
             F=torch.zeros((e.n, 3), dtype=torch.float64, device="cuda"))
    c.forces(0, d["pos"], d["q"], d["typ"], None, d["F"])
    c.step(0, 50, e.dt, e.accel, d["pos"], d["vel"], d["mass"], d["q"], d["typ"], None, d["F"])
    nsteps = 500
    ms = events(lambda k: c.step(50, nsteps, e.dt, e.accel, d["pos"], d["vel"], d["mass"], d["q"], d["typ"], None,
                                 d["F"]), 1) / nsteps
    if c.sync_status() != 0:
        raise RuntimeError("device status error in the Langevin leg")
    out["langevin"] = {"workload": "1:1 electrolyte, 5,120 ions, L=80 sigma, WCA, r_c=5, r_s=15, p=10, P=100, "
                                   "alpha=0.03, dt=0.002, kT=1, tau=1, mixed",
                       "steps_per_s": 1e3 / ms, "ms_per_step": ms, "tau_per_day": 1e3 / ms * e.dt * 86400.0,
                       "atom_steps_per_s": e.n * 1e3 / ms}
    c.close()
    return out


def run_ours(args):
    import numpy as np
    import torch

    from paper_2204_13595_gb300 import build as b
    from paper_2204_13595_gb300 import rbe, replicas, systems

    ws, rank = _dist()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    b.build()
    s = systems.water(N_MOL, seed=replicas.rank_seed(SEED, rank))
    dev = lambda a, dt=torch.float64: torch.tensor(a, dtype=dt, device="cuda")
    pos, q, typ, mol = dev(s.pos), dev(s.q), dev(s.type, torch.int32), dev(s.mol, torch.int32)
    F = torch.empty_like(pos)
    E = torch.zeros(rbe.NE, dtype=torch.float64, device="cuda")
    W = torch.zeros(rbe.NW, dtype=torch.float64, device="cuda")
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    def make(prec):
        return rbe.Context(s.L, s.alpha, s.r_c, s.r_s, s.p, s.P, SEED, k_e=s.k_e, eps=s.eps, sigma=s.sigma,
                           precision=prec)

    def timed(ctx, steps, warmup, profile=False):
        for w in range(warmup):
            ctx.forces(w, pos, q, typ, mol, F, E, W)
        if ctx.sync_status() != 0:
            raise RuntimeError("device status error during warm-up")
        if profile:
            ctx.profile(reset=True)
            ctx.set_profiling(True)
        total = 0.0
        replicas.barrier(ws)
        torch.cuda.synchronize()
        for k in range(steps):
            flush.fill_(float(k))
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ctx.forces(warmup + k, pos, q, typ, mol, F, E, W)
            e1.record(stream)
            e1.synchronize()
            total += e0.elapsed_time(e1)
        torch.cuda.synchronize()
        replicas.barrier(ws)
        prof = None
        if profile:
            prof = ctx.profile(reset=True)
            ctx.set_profiling(False)
        launches = int(ctx.info()["launches"])
        if ctx.sync_status() != 0:
            raise RuntimeError("device status error during the timed steps")
        ms = replicas.max_over_ranks(total / steps, ws, device="cuda")
        return ms, prof, launches

    # fixed-error check: mixed vs FP64 on identical draws (outside timing)
    mixed, f64 = make(rbe.MIXED), make(rbe.FP64)
    mixed.forces(123, pos, q, typ, mol, F)
    Fm = F.clone()
    f64.forces(123, pos, q, typ, mol, F)
    err = float(torch.sqrt(((Fm - F) ** 2).mean()) / torch.sqrt((F ** 2).mean()))

    # measured pipe and memory throughput of this GPU (context for the derived peaks)
    meas = {}
    for kind in ("ffma", "dfma", "sfu", "alu", "copy"):
        try:
            meas[kind] = peak_probe(kind)
        except Exception as e:        # report, do not fail the bench
            meas[kind] = f"unavailable: {e}"
    clocks_proc = _clock_sampler() if rank == 0 else None
    # the headline steps run unprofiled (with per-kernel profiling on, the
    # library serialises the Fourier kernels with the pair kernel); a separate
    # profiled pass gives the per-kernel times
    ms_mixed, _, launches = timed(mixed, args.steps, args.warmup)
    _, prof, _ = timed(mixed, max(3, min(args.steps, 10)), 1, profile=True)
    ms_f64, _, _ = timed(f64, max(3, min(args.steps, 10)), max(3, min(args.warmup, 3)))
    _, prof64, _ = timed(f64, 3, 1, profile=True)
    batch = _batch_leg(flush) if ws == 1 else None
    next_rows = _next_rows_leg(flush, (s, pos, q, typ, mol)) if ws == 1 else None
    configs = _configs_leg(flush) if ws == 1 else None
    clocks = _clock_summary(clocks_proc, local) if rank == 0 else None

    # end to end through the same C ABI with pinned host buffers
    hp = torch.tensor(s.pos, dtype=torch.float64).pin_memory()
    hq = torch.tensor(s.q, dtype=torch.float64).pin_memory()
    ht = torch.tensor(s.type, dtype=torch.int32).pin_memory()
    hm = torch.tensor(s.mol, dtype=torch.int32).pin_memory()
    hF = torch.empty((s.n, 3), dtype=torch.float64).pin_memory()
    hE = torch.empty(rbe.NE, dtype=torch.float64).pin_memory()
    hW = torch.empty(rbe.NW, dtype=torch.float64).pin_memory()
    for w in range(args.warmup):
        mixed.forces(w, hp, hq, ht, hm, hF, hE, hW)
    replicas.barrier(ws)
    t0 = time.perf_counter()
    for k in range(args.steps):
        mixed.forces(args.warmup + k, hp, hq, ht, hm, hF, hE, hW)
    e2e_s = replicas.max_over_ranks((time.perf_counter() - t0) / args.steps, ws, device="cuda")
    h2d = hp.numel() * 8 + hq.numel() * 8 + ht.numel() * 4 + hm.numel() * 4
    d2h = hF.numel() * 8 + hE.numel() * 8 + hW.numel() * 8

    if rank != 0:
        if ws > 1:
            torch.distributed.destroy_process_group()
        return 0

    # roofline of the dominant kernel (the RBL list + pair kernel)
    rbl_ms, rbl_n = prof["rbl"]
    rbl_avg_s = rbl_ms / max(rbl_n, 1) * 1e-3
    achieved = RBL_OPS_PER_ATOM * s.n / rbl_avg_s / 1e12
    peak = SM_COUNT * LANES_PER_SM * SM_MAX_MHZ * 1e6 / 1e12
    kshare = {k: round(v[0] / max(sum(x[0] for x in prof.values()), 1e-30), 4) for k, v in prof.items() if v[1]}
    traffic = _traffic(os.path.join(ROOT, "paper_2204_13595_gb300", "csrc", "k_rbl.cu"))

    # CPU baseline: the oracle on the host cores, one full evaluation
    import oracle
    oracle.build()
    pr = oracle.make_params(s.L, s.alpha, s.r_c, s.r_s, s.p, s.P, SEED, k_e=s.k_e, eps=s.eps, sigma=s.sigma)
    t0 = time.perf_counter()
    oracle.rbe_forces(s.pos, s.q, s.type, s.mol, pr, 0)
    cpu_s = time.perf_counter() - t0
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    oracle_more = _oracle_timings()

    value = replicas.throughput(ws, 1, ms_mixed)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_mixed, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32 pair/phase + f64 positions/sums (mixed)", "data": "synthetic",
        "config": dict(_workload_config(s), precision="mixed", parallelism=f"replicas x{ws}"),
        "ns_per_day": 0.0864 * value * DT_FS, "atom_steps_per_s": value * s.n,
        "fp64": {"value": ws * 1e3 / ms_f64, "ms_per_step": ms_f64, "ns_per_day": 0.0864 * ws * 1e3 / ms_f64 * DT_FS},
        "speedup_mixed_vs_fp64": ms_f64 / ms_mixed,
        "mixed_force_rms_rel_err_vs_fp64": err,
        "roofline": {"kernel": "k_rbl (lists + shell batch + pair forces, mixed)", "bound": "alu",
                     "achieved": achieved, "peak": peak, "unit": "Top/s", "frac": achieved / peak,
                     "traffic": traffic, "peak_source": "derived: 152 SMs x 128 lanes x 2070 MHz, 1 op/lane/clk",
                     "avg_launch_ms": rbl_avg_s * 1e3},
        "kernel_share": kshare,
        "kernel_roofline": dict(_kernel_roofline(prof, s.n, s.P, mixed.info()["n_cell"] ** 3, meas),
                                rbl_fp64=_fp64_rbl_roofline(prof64, s.n, meas)),
        "measured_pipes": {
            "ffma_per_s": meas.get("ffma"), "dfma_per_s": meas.get("dfma"), "sfu_sin_per_s": meas.get("sfu"),
            "int_ops_per_s": meas.get("alu"), "copy_bytes_per_s": meas.get("copy"),
            "note": "bench_peak_probe in this run (best of 3 launches): context for the derived peaks"},
        "cpu_baseline": {"value": 1.0 / cpu_s, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": "one full FP64 oracle force evaluation of the same 1.2M-atom system"},
        "oracle_timings": oracle_more,
        "e2e": {"value": replicas.throughput(ws, 1, e2e_s * 1e3), "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "clocks": clocks, "gpu_launches": launches * args.steps,
        "batch": batch,
        "next_rows": next_rows,
        "configs": configs,
    }
    print(json.dumps(line))
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
