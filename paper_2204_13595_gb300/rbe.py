"""Thin ctypes binding of librbe.so (include/rbe.h).

Argument marshalling only: every step of the force evaluation runs in the
library's CUDA kernels.  Tensors are passed by data pointer; the current torch
CUDA stream is used unless a stream is given.  Importing this module fails
loudly when the library is missing: there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "librbe.so")

OK, EINVAL, ENONNEUTRAL, EOVERLAP, ENONFINITE, ECAPACITY, ECUDA, ENOMEM = 0, -1, -2, -3, -4, -5, -6, -7
FP64, MIXED = 0, 1
NE, NW = 6, 6
E_REAL, E_KSPACE, E_SELF, E_LJ, E_EXCL, E_BOND = range(6)
KERNELS = ["quantize", "scan", "scatter", "sort", "gather", "ksample", "rho", "rhosum", "rbl", "bonded",
           "finalize", "kforce", "vv", "misc", "skin"]
EXPORTS = ["rbe_create", "rbe_set_coulomb", "rbe_set_lj", "rbe_set_precision", "rbe_set_water_bonds",
           "rbe_set_capacity", "rbe_forces", "rbe_step", "rbe_sync_status", "rbe_set_debug", "rbe_get_lists",
           "rbe_get_kspace", "rbe_get_info", "rbe_set_profiling", "rbe_get_profile", "rbe_last_error",
           "rbe_destroy", "rbe_rho_noalloc", "rbe_adjoint", "rbe_set_rbl_tiling", "rbe_batch_create",
           "rbe_batch_bind", "rbe_batch_forces", "rbe_batch_step", "rbe_batch_autotune", "rbe_batch_info",
           "rbe_batch_sync_status", "rbe_batch_last_error", "rbe_batch_destroy", "rbe_set_shell_sampling",
           "rbe_set_lj_cutoff", "rbe_set_kpool", "rbe_set_langevin", "rbe_get_langevin_force", "rbe_set_verlet_skin",
           "rbe_set_langevin_force"]
SHELL_FLOYD, SHELL_REPLACE = 0, 1
WCA_FACTOR = 2.0 ** (1.0 / 6.0)
ELIMIT = -8
NOALLOC_BLOCKS, NOALLOC_PMAX = 256, 512


class RbeError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"rbe error {code}: {msg}")
        self.code = code


def load(path: str = LIB_PATH):
    if not os.path.exists(path):
        raise RuntimeError(f"librbe.so not found at {path}: build it with paper_2204_13595_gb300.build.build()")
    L = ctypes.CDLL(path)
    vp, d, i, u64, i32p = ctypes.c_void_p, ctypes.c_double, ctypes.c_int, ctypes.c_uint64, ctypes.c_void_p
    L.rbe_create.argtypes = [ctypes.POINTER(vp), d, d, d, d, i, i, u64]
    L.rbe_set_coulomb.argtypes = [vp, d]
    L.rbe_set_lj.argtypes = [vp, i, ctypes.POINTER(d), ctypes.POINTER(d), i]
    L.rbe_set_precision.argtypes = [vp, i]
    L.rbe_set_water_bonds.argtypes = [vp, i, d, d, d, d]
    L.rbe_set_capacity.argtypes = [vp, i, i]
    L.rbe_forces.argtypes = [vp, u64, i, vp, vp, vp, vp, vp, vp, vp, vp]
    L.rbe_step.argtypes = [vp, u64, i, d, d, i, vp, vp, vp, vp, vp, vp, vp, vp, vp]
    L.rbe_sync_status.argtypes = [vp, vp]
    L.rbe_set_debug.argtypes = [vp, i, i]
    L.rbe_get_lists.argtypes = [vp, i, vp, vp, vp, vp, vp]
    L.rbe_get_kspace.argtypes = [vp, vp, vp, vp]
    L.rbe_get_info.argtypes = [vp, ctypes.POINTER(d), i]
    L.rbe_set_profiling.argtypes = [vp, i]
    L.rbe_get_profile.argtypes = [vp, ctypes.POINTER(d), ctypes.POINTER(ctypes.c_int64), i, vp]
    L.rbe_last_error.argtypes = [vp]
    L.rbe_last_error.restype = ctypes.c_char_p
    L.rbe_destroy.argtypes = [vp]
    L.rbe_destroy.restype = None
    L.rbe_rho_noalloc.argtypes = [i, vp, vp, d, i, vp, vp, vp]
    L.rbe_adjoint.argtypes = [vp, u64, i, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp]
    L.rbe_set_rbl_tiling.argtypes = [vp, i, i]
    L.rbe_set_shell_sampling.argtypes = [vp, i]
    L.rbe_set_lj_cutoff.argtypes = [vp, d]
    L.rbe_set_kpool.argtypes = [vp, i, i]
    L.rbe_set_langevin.argtypes = [vp, d, d]
    L.rbe_set_verlet_skin.argtypes = [vp, d]
    L.rbe_get_langevin_force.argtypes = [vp, i, vp, ctypes.POINTER(u64)]
    L.rbe_set_langevin_force.argtypes = [vp, i, vp, u64]
    L.rbe_batch_create.argtypes = [ctypes.POINTER(vp), i, ctypes.POINTER(vp)]
    L.rbe_batch_bind.argtypes = [vp, ctypes.POINTER(i)] + [ctypes.POINTER(vp)] * 7 + [ctypes.POINTER(d)] * 2
    L.rbe_batch_forces.argtypes = [vp, u64, vp, vp]
    L.rbe_batch_step.argtypes = [vp, u64, i, vp, vp]
    L.rbe_batch_autotune.argtypes = [vp, u64, ctypes.POINTER(d), i, vp]
    L.rbe_batch_info.argtypes = [vp, ctypes.POINTER(d), i]
    L.rbe_batch_sync_status.argtypes = [vp, vp, vp]
    L.rbe_batch_last_error.argtypes = [vp]
    L.rbe_batch_last_error.restype = ctypes.c_char_p
    L.rbe_batch_destroy.argtypes = [vp]
    L.rbe_batch_destroy.restype = None
    return L


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = load()
    return _lib


def _ptr(x):
    """Data pointer of a torch tensor or numpy array (None -> NULL)."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    return x.data_ptr()


def _stream(stream):
    if stream is not None:
        return stream if isinstance(stream, int) else stream.cuda_stream
    import torch
    return torch.cuda.current_stream().cuda_stream


def _check_noalloc_args(pos, q, m, rho):
    """Shapes, dtypes and placement that rbe_rho_noalloc reads its raw
    pointers as: pos float64 [n,3], q float64 [n], m int32 [P,3], rho float64
    [P,2], all contiguous on the current CUDA device.  Anything else would be
    read or written as the wrong type or size, so it is refused here."""
    import torch
    dev = torch.cuda.current_device() if torch.cuda.is_available() else None
    want = (("pos", pos, torch.float64, 3), ("q", q, torch.float64, None), ("m", m, torch.int32, 3),
            ("rho", rho, torch.float64, 2))
    for name, t, dt, cols in want:
        if not isinstance(t, torch.Tensor):
            raise RbeError(EINVAL, f"rho_noalloc: {name} must be a torch tensor")
        if t.dtype != dt:
            raise RbeError(EINVAL, f"rho_noalloc: {name} must be {dt}, got {t.dtype}")
        if cols is None and t.dim() != 1:
            raise RbeError(EINVAL, f"rho_noalloc: {name} must be 1-D")
        if cols is not None and (t.dim() != 2 or t.shape[1] != cols):
            raise RbeError(EINVAL, f"rho_noalloc: {name} must have shape [*, {cols}]")
        if not t.is_contiguous():
            raise RbeError(EINVAL, f"rho_noalloc: {name} must be contiguous")
    if q.shape[0] != pos.shape[0]:
        raise RbeError(EINVAL, "rho_noalloc: q and pos hold different atom counts")
    if rho.shape[0] != m.shape[0]:
        raise RbeError(EINVAL, "rho_noalloc: rho must have one row per k vector of m")
    for name, t, _, _ in want:
        if not t.is_cuda or t.device.index != dev:
            raise RbeError(EINVAL, f"rho_noalloc: {name} must be on the current CUDA device")


def rho_noalloc(pos, q, box_L, m, rho, stream=None):
    """rbe_rho_noalloc: structure factors into rho[P,2] without any device
    allocation (scratch is a static device array; see include/rbe.h)."""
    _check_noalloc_args(pos, q, m, rho)
    rc = lib().rbe_rho_noalloc(int(pos.shape[0]), _ptr(pos), _ptr(q), float(box_L), int(m.shape[0]), _ptr(m),
                               _ptr(rho), _stream(stream))
    if rc != OK:
        raise RbeError(rc, "rbe_rho_noalloc failed" + (" (P above RBE_NOALLOC_PMAX)" if rc == ELIMIT else ""))
    return rc


class Context:
    """One IRBE context (box, alpha, r_c, r_s, p, P, seed) -- rbe_create."""

    def __init__(self, L, alpha, r_c, r_s, p, P, seed, k_e=1.0, eps=None, sigma=None, shift_lj=False,
                 precision=FP64):
        self.L = lib()
        h = ctypes.c_void_p()
        rc = self.L.rbe_create(ctypes.byref(h), L, alpha, r_c, r_s, p, P, seed)
        if rc != OK or not h.value:
            raise RbeError(rc, "rbe_create rejected the parameters")
        self.h = h
        self.p, self.P = p, P
        self.ntypes = 1
        self._check(self.L.rbe_set_coulomb(self.h, k_e))
        if eps is not None:
            self.set_lj(eps, sigma, shift_lj)
        self.set_precision(precision)

    @classmethod
    def for_system(cls, s, precision=FP64, seed=None):
        ctx = cls(s.L, s.alpha, s.r_c, s.r_s, s.p, s.P, s.seed if seed is None else seed, k_e=s.k_e,
                  eps=s.eps, sigma=s.sigma, precision=precision)
        if s.n_water_mol:
            ctx.set_water_bonds(s.n_water_mol, *s.bonds)
        return ctx

    def _check(self, rc):
        if rc != OK:
            raise RbeError(rc, self.L.rbe_last_error(self.h).decode(errors="replace"))
        return rc

    def set_precision(self, mode):
        self._check(self.L.rbe_set_precision(self.h, mode))

    def set_water_bonds(self, n_mol, kb, r0, kth, th0):
        self._check(self.L.rbe_set_water_bonds(self.h, n_mol, kb, r0, kth, th0))

    def set_capacity(self, core, shell):
        self._check(self.L.rbe_set_capacity(self.h, core, shell))

    def set_shell_sampling(self, mode):
        self._check(self.L.rbe_set_shell_sampling(self.h, int(mode)))

    def set_lj_cutoff(self, factor):
        self._check(self.L.rbe_set_lj_cutoff(self.h, float(factor)))

    def set_kpool(self, size, burn_in=0):
        self._check(self.L.rbe_set_kpool(self.h, int(size), int(burn_in)))

    def set_langevin(self, kT, tau):
        """Langevin thermostat of rbe_step (tau <= 0: off)."""
        self._check(self.L.rbe_set_langevin(self.h, float(kT), float(tau)))

    def get_langevin_force(self, n):
        """The held Langevin force [n, 3] (host array) and its step (checkpoint)."""
        FL = np.zeros((n, 3))
        st = ctypes.c_uint64()
        self._check(self.L.rbe_get_langevin_force(self.h, n, _ptr(FL), ctypes.byref(st)))
        return FL, st.value

    def set_langevin_force(self, FL, step):
        FL = np.ascontiguousarray(FL, dtype=np.float64)
        self._check(self.L.rbe_set_langevin_force(self.h, int(FL.shape[0]), _ptr(FL), int(step)))

    def set_verlet_skin(self, skin):
        """rbe_set_verlet_skin: stored lists within r_s + skin, rebuilt when an
        atom has moved more than skin/2 (0: lists every step)."""
        self._check(self.L.rbe_set_verlet_skin(self.h, float(skin)))

    def set_rbl_tiling(self, atoms_per_unit=0, units_per_slot=0):
        self._check(self.L.rbe_set_rbl_tiling(self.h, int(atoms_per_unit), int(units_per_slot)))

    def set_debug(self, on, cap_core=0):
        self._check(self.L.rbe_set_debug(self.h, int(on), cap_core))

    def set_profiling(self, on):
        self._check(self.L.rbe_set_profiling(self.h, int(on)))

    def forces(self, step, pos, q, typ, mol, F, energy=None, virial=None, stream=None):
        """rbe_forces; all of pos, q, typ, mol, F on the device or all on the host."""
        n = int(pos.shape[0])
        st = _stream(stream) if not isinstance(pos, np.ndarray) else (stream or 0)
        return self._check(self.L.rbe_forces(self.h, step, n, _ptr(pos), _ptr(q), _ptr(typ), _ptr(mol), _ptr(F),
                                             _ptr(energy), _ptr(virial), st))

    def step(self, step0, nsteps, dt, accel, pos, vel, mass, q, typ, mol, F, trace=None, stream=None):
        n = int(pos.shape[0])
        return self._check(self.L.rbe_step(self.h, step0, nsteps, dt, accel, n, _ptr(pos), _ptr(vel), _ptr(mass),
                                           _ptr(q), _ptr(typ), _ptr(mol), _ptr(F), _ptr(trace), _stream(stream)))

    def adjoint(self, step, pos, q, typ, mol, gF=None, stream=None):
        """rbe_adjoint: gradients at frozen draws.  Returns dEdq, dLdq (device
        tensors, caller order) and the per-type dEdeps, dEdsig, dLdeps, dLdsig."""
        import torch
        n = int(pos.shape[0])
        dEdq = torch.empty(n, dtype=torch.float64, device=pos.device)
        dLdq = torch.empty(n, dtype=torch.float64, device=pos.device)
        T = self.ntypes
        outs = [np.zeros(T) for _ in range(4)]
        self._check(self.L.rbe_adjoint(self.h, step, n, _ptr(pos), _ptr(q), _ptr(typ), _ptr(mol), _ptr(gF),
                                       _ptr(dEdq), _ptr(dLdq), *[_ptr(o) for o in outs], _stream(stream)))
        return dict(dEdq=dEdq, dLdq=dLdq, dEdeps=outs[0], dEdsig=outs[1], dLdeps=outs[2], dLdsig=outs[3])

    def set_lj(self, eps, sigma, shift_lj=False):
        e = (ctypes.c_double * len(eps))(*[float(x) for x in eps])
        s = (ctypes.c_double * len(sigma))(*[float(x) for x in sigma])
        self._check(self.L.rbe_set_lj(self.h, len(eps), e, s, int(shift_lj)))
        self.ntypes = len(eps)

    def sync_status(self, stream=None):
        return self.L.rbe_sync_status(self.h, _stream(stream))

    def get_lists(self, n, cap_core, stream=None):
        n_core = np.zeros(n, np.int32)
        n_shell = np.zeros(n, np.int32)
        core = np.zeros((n, max(cap_core, 1)), np.int32)
        batch = np.zeros((n, self.p), np.int32)
        self._check(self.L.rbe_get_lists(self.h, n, _ptr(n_core), _ptr(n_shell), _ptr(core) if cap_core else None,
                                         _ptr(batch), _stream(stream)))
        return dict(n_core=n_core, n_shell=n_shell, core=core[:, :cap_core], batch=batch)

    def get_kspace(self, stream=None):
        m = np.zeros((self.P, 3), np.int32)
        rho = np.zeros((self.P, 2))
        self._check(self.L.rbe_get_kspace(self.h, _ptr(m), _ptr(rho), _stream(stream)))
        return m, rho[:, 0] + 1j * rho[:, 1]

    def info(self):
        keys = ["n_cell", "reach", "M", "S", "core_cap", "shell_cap", "launches", "unstaged_units", "walked_passes",
                "halt_step", "skin_rebuilds", "skin_vcap"]
        out = (ctypes.c_double * len(keys))()
        self._check(self.L.rbe_get_info(self.h, out, len(keys)))
        return {k: out[i] for i, k in enumerate(keys)}

    def profile(self, reset=True, stream=None):
        ms = (ctypes.c_double * len(KERNELS))()
        nl = (ctypes.c_int64 * len(KERNELS))()
        self._check(self.L.rbe_get_profile(self.h, ms, nl, int(reset), _stream(stream)))
        return {k: (ms[i], nl[i]) for i, k in enumerate(KERNELS)}

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            self.L.rbe_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """rbe_batch_*: many contexts (replicas) stepped together, one launch per
    stage over all replicas, one MD step replayed as a CUDA graph.  The
    contexts must outlive the batch."""

    def __init__(self, contexts):
        self.L = lib()
        self.ctxs = list(contexts)
        arr = (ctypes.c_void_p * len(self.ctxs))(*[c.h.value for c in self.ctxs])
        h = ctypes.c_void_p()
        rc = self.L.rbe_batch_create(ctypes.byref(h), len(self.ctxs), arr)
        if rc != OK or not h.value:
            raise RbeError(rc, "rbe_batch_create rejected the contexts")
        self.h = h
        self.nrep = len(self.ctxs)
        self._keep = None

    def _check(self, rc):
        if rc != OK:
            raise RbeError(rc, self.L.rbe_batch_last_error(self.h).decode(errors="replace"))
        return rc

    def bind(self, pos, q, typ, mol, F, vel=None, mass=None, dt=None, accel=None):
        """Per-replica lists of device tensors (typ, mol, vel, mass entries may
        be None); dt and accel per-replica lists of floats (or None)."""
        R = self.nrep
        VP = ctypes.c_void_p * R

        def arr(xs):
            return VP(*[_ptr(x) if xs is not None else None for x in (xs if xs is not None else [None] * R)])
        n = (ctypes.c_int * R)(*[int(p.shape[0]) for p in pos])
        dts = (ctypes.c_double * R)(*[float(x) for x in dt]) if dt is not None else None
        acs = (ctypes.c_double * R)(*[float(x) for x in accel]) if accel is not None else None
        args = [n, arr(pos), arr(q), arr(typ), arr(mol), arr(F), arr(vel), arr(mass)]
        self._keep = (pos, q, typ, mol, F, vel, mass)
        return self._check(self.L.rbe_batch_bind(self.h, *args, dts, acs))

    def forces(self, step, energy=False, stream=None):
        """Forces of every replica at `step` into the bound F; with energy=True
        returns the [nrep, NE] energies (waits)."""
        E = np.zeros((self.nrep, NE)) if energy else None
        self._check(self.L.rbe_batch_forces(self.h, step, _ptr(E), _stream(stream)))
        return E

    def step(self, step0, nsteps, trace=None, stream=None):
        return self._check(self.L.rbe_batch_step(self.h, step0, nsteps, _ptr(trace), _stream(stream)))

    def autotune(self, step=0, stream=None):
        out = (ctypes.c_double * 64)()
        self._check(self.L.rbe_batch_autotune(self.h, step, out, 64, _stream(stream)))
        nf = int(self.info()["families"])
        fams = [dict(atoms_per_unit=int(out[3 * f]), units_per_slot=int(out[3 * f + 1]), ms=out[3 * f + 2])
                for f in range(nf)]
        return dict(families=fams, persistent=bool(out[3 * nf]), tuned_ms=out[3 * nf + 1],
                    untuned_ms=out[3 * nf + 2])

    def info(self):
        out = (ctypes.c_double * 7)()
        self._check(self.L.rbe_batch_info(self.h, out, 7))
        keys = ["replicas", "atoms", "tasks", "rbl_blocks", "rbl_smem", "launches_per_step", "families"]
        return {k: out[i] for i, k in enumerate(keys)}

    def sync_status(self, stream=None):
        st = np.zeros(self.nrep, np.int32)
        first = self.L.rbe_batch_sync_status(self.h, _ptr(st), _stream(stream))
        return first, st

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            self.L.rbe_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class RbeForces:
    """Differentiable IRBE force step (torch.autograd.Function wrapper).

    ``RbeForces.apply(ctx, step, pos, q, typ, mol, eps, sigma)`` returns
    (F [n,3], E scalar: the sum of the non-bonded energy components) for the
    charges ``q`` (device tensor) and per-type LJ parameters ``eps``,
    ``sigma`` (CPU tensors).  Gradients flow to q, eps and sigma through
    rbe_adjoint with the draws of ``step`` frozen; positions are inputs only.
    """

    @staticmethod
    def apply(ctx, step, pos, q, typ, mol, eps, sigma):
        return _rbe_function().apply(ctx, step, pos, q, typ, mol, eps, sigma)


_FN = None


def _rbe_function():
    global _FN
    if _FN is not None:
        return _FN
    import torch

    class _F(torch.autograd.Function):
        @staticmethod
        def forward(actx, ctx, step, pos, q, typ, mol, eps, sigma):
            ctx.set_lj(eps.detach().cpu().tolist(), sigma.detach().cpu().tolist())
            F = torch.empty_like(pos)
            E = torch.zeros(NE, dtype=torch.float64, device=pos.device)
            qd = q.detach().contiguous()
            ctx.forces(step, pos, qd, typ, mol, F, E)
            actx.rbe = (ctx, step, pos, qd, typ, mol)
            actx.lj_dev = eps.device
            return F, E[:E_BOND].sum()

        @staticmethod
        def backward(actx, gF, gE):
            ctx, step, pos, q, typ, mol = actx.rbe
            gFc = None if gF is None else gF.contiguous()
            g = ctx.adjoint(step, pos, q, typ, mol, gFc)
            ge = 0.0 if gE is None else float(gE)
            dq = g["dLdq"] + ge * g["dEdq"]
            de = torch.tensor(g["dLdeps"] + ge * g["dEdeps"], dtype=torch.float64, device=actx.lj_dev)
            ds = torch.tensor(g["dLdsig"] + ge * g["dEdsig"], dtype=torch.float64, device=actx.lj_dev)
            return None, None, None, dq, None, None, de, ds

    _FN = _F
    return _FN
