"""Plain FP64 CPU oracle for the IRBE (RBL + RBE) force step (arXiv 2204.13595).

TEST INFRASTRUCTURE ONLY: tests/, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may use it; the product package never imports it.
It shares no code with the CUDA library.  The arithmetic lives in
``rbe_oracle.c`` (plain C, FP64, ``-ffp-contract=off``); this module only
compiles it and marshals numpy arrays through ctypes.

Parity status of each function (what pins it; tests/test_oracle_*.py):
  philox4x64_10     numpy.random.Philox bit match
  k sampler / S     chi^2 against the exact marginals of Eq. (2.8); the
                    Poisson form of H, Eq. (2.7)
  floyd             chi^2 over all C(6,3) subsets; uniform inclusion
  lists             brute force == cell stencil; neighbour counts vs 4/3 pi r^3 rho
                    and the paper's ~140 / ~700 (Sec. 2.1, Sec. 3.1)
  skin_lists,       (reading R15) stored lists: stencil == brute force; a step's
  lists(pos_b=)     sets from them == the stencil sets at that step while no
                    atom moved more than skin/2, and the rebuild test decides
                    that boundary exactly
  ewald_exact       NaCl Madelung constant; alpha invariance; direct lattice
                    sum; central finite differences; virial trace = energy
  rbe_forces        p >= max N_S reduces to the truncated exact sum;
                    RBE energy gradient by finite differences (frozen draws);
                    sum_i F_i = 0; unbiasedness over seeds with the exact
                    finite-sample variance (Eqs. (2.11), (2.9), (2.14))
  rbe_adjoint       central finite differences of the estimator with frozen
                    draws (charges, per-type eps and sigma through the
                    Lorentz-Berthelot pair table)
  water_bonded      central finite differences
  vv_run            time reversibility and energy of a harmonic dimer
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rbe_oracle.c")
_LIB = os.path.join(_HERE, "librbe_oracle.so")
_lock = threading.Lock()
_lib = None

MAXT = 16


def build(force: bool = False) -> str:
    """Compile rbe_oracle.c into librbe_oracle.so (OpenMP when available)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    base = ["gcc", "-O2", "-ffp-contract=off", "-shared", "-fPIC", "-o", _LIB + ".tmp", _SRC, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True)
    os.replace(_LIB + ".tmp", _LIB)
    return _LIB


class Params(ctypes.Structure):
    _fields_ = [
        ("L", ctypes.c_double),
        ("alpha", ctypes.c_double),
        ("r_c", ctypes.c_double),
        ("r_s", ctypes.c_double),
        ("k_e", ctypes.c_double),
        ("p", ctypes.c_int),
        ("P", ctypes.c_int),
        ("seed", ctypes.c_uint64),
        ("ntypes", ctypes.c_int),
        ("shift_lj", ctypes.c_int),
        ("eps", ctypes.c_double * MAXT),
        ("sigma", ctypes.c_double * MAXT),
        ("shell_mode", ctypes.c_int),
        ("lj_rc_factor", ctypes.c_double),
        ("kpool", ctypes.c_int),
        ("kpool_burn", ctypes.c_int),
        ("lang_kT", ctypes.c_double),
        ("lang_tau", ctypes.c_double),
        ("skin", ctypes.c_double),
    ]


def make_params(L, alpha, r_c, r_s, p, P, seed, k_e=1.0, eps=(0.0,), sigma=(1.0,), shift_lj=0, shell_mode=0,
                lj_rc_factor=0.0, kpool=0, kpool_burn=0, lang_kT=0.0, lang_tau=0.0, skin=0.0):
    """Parameters of the estimator; shell_mode, lj_rc_factor, kpool and
    kpool_burn select the variants of reading R13, lang_kT and lang_tau the
    Langevin thermostat of R14 used by vv_run, skin the Verlet skin of R15
    (used with rebuild positions pos_b; defaults: the base method)."""
    pr = Params()
    pr.skin = float(skin)
    pr.lang_kT, pr.lang_tau = float(lang_kT), float(lang_tau)
    pr.shell_mode, pr.lj_rc_factor = int(shell_mode), float(lj_rc_factor)
    pr.kpool, pr.kpool_burn = int(kpool), int(kpool_burn)
    pr.L, pr.alpha, pr.r_c, pr.r_s, pr.k_e = float(L), float(alpha), float(r_c), float(r_s), float(k_e)
    pr.p, pr.P, pr.seed = int(p), int(P), int(seed)
    pr.ntypes = len(eps)
    pr.shift_lj = int(shift_lj)
    for t, (e, s) in enumerate(zip(eps, sigma)):
        pr.eps[t] = float(e)
        pr.sigma[t] = float(s)
    return pr


_P = ctypes.POINTER


def _ptr(a, ctype):
    if a is None:
        return None
    return a.ctypes.data_as(_P(ctype))


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB)
            d, i32, u32, u64 = ctypes.c_double, ctypes.c_int32, ctypes.c_uint32, ctypes.c_uint64
            L.orc_philox4x64_10.argtypes = [_P(u64), _P(u64), _P(u64)]
            L.orc_radius2_fixed.argtypes = [d, d]
            L.orc_radius2_fixed.restype = u64
            L.orc_n_cell.argtypes = [d, d]
            L.orc_quantize.argtypes = [ctypes.c_int, _P(d), d, d, _P(u32), _P(i32)]
            L.orc_kmax.argtypes = [d, d]
            L.orc_k_table.argtypes = [d, d, ctypes.c_int, _P(u64)]
            L.orc_k_table.restype = d
            L.orc_sample_k.argtypes = [u64, u64, ctypes.c_int, d, d, _P(i32)]
            L.orc_mh_tables.argtypes = [d, d, ctypes.c_int, _P(d), _P(d), _P(u64)]
            L.orc_kpool.argtypes = [u64, d, d, ctypes.c_int, ctypes.c_int, _P(i32)]
            L.orc_kpool.restype = d
            L.orc_sample_k_params.argtypes = [_P(Params), u64, _P(i32)]
            L.orc_S.argtypes = [d, d]
            L.orc_S.restype = d
            L.orc_floyd.argtypes = [u64, ctypes.c_int, _P(u64), _P(u64)]
            L.orc_lists.argtypes = [ctypes.c_int, _P(d), _P(Params), u64, ctypes.c_int,
                                    _P(i32), _P(i32), _P(i32), _P(i32), ctypes.c_int,
                                    _P(i32), ctypes.c_int, _P(i32), ctypes.c_int]
            L.orc_lists_skin.argtypes = [ctypes.c_int, _P(d), _P(d), _P(Params), u64, ctypes.c_int,
                                         _P(i32), _P(i32), _P(i32), _P(i32), ctypes.c_int,
                                         _P(i32), ctypes.c_int, _P(i32), ctypes.c_int]
            L.orc_skin_lists.argtypes = [ctypes.c_int, _P(d), _P(Params), ctypes.c_int, _P(i32), _P(i32),
                                         ctypes.c_int]
            L.orc_skin_displaced.argtypes = [ctypes.c_int, _P(d), _P(d), d, d]
            L.orc_rbe_forces_skin.argtypes = [ctypes.c_int, _P(d), _P(d), _P(d), _P(i32), _P(i32), _P(Params), u64,
                                              _P(d), _P(d), _P(d), _P(d), _P(d), _P(d), _P(i32), _P(d), _P(d)]
            L.orc_rho.argtypes = [ctypes.c_int, _P(d), _P(d), d, ctypes.c_int, _P(i32), _P(d)]
            L.orc_rbe_forces.argtypes = [ctypes.c_int, _P(d), _P(d), _P(i32), _P(i32), _P(Params), u64,
                                         _P(d), _P(d), _P(d), _P(d), _P(d), _P(d), _P(i32), _P(d), _P(d)]
            L.orc_rbe_adjoint.argtypes = [ctypes.c_int, _P(d), _P(d), _P(i32), _P(i32), _P(Params), u64, _P(d),
                                          _P(d), _P(d), _P(d), _P(d), _P(d), _P(d)]
            L.orc_ewald_exact.argtypes = [ctypes.c_int, _P(d), _P(d), _P(i32), _P(i32), _P(Params),
                                          d, ctypes.c_int, _P(d), _P(d), _P(d)]
            L.orc_direct_coulomb.argtypes = [ctypes.c_int, _P(d), _P(d), d, d, ctypes.c_int]
            L.orc_direct_coulomb.restype = d
            L.orc_water_bonded.argtypes = [ctypes.c_int, ctypes.c_int, _P(d), d, d, d, d, d, _P(d)]
            L.orc_water_bonded.restype = d
            L.orc_vv_run.argtypes = [ctypes.c_int, _P(d), _P(d), _P(d), _P(d), _P(i32), _P(i32), _P(Params),
                                     u64, ctypes.c_int, d, d, ctypes.c_int, d, d, d, d, _P(d), _P(d)]
            _lib = L
    return _lib


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.int32)


# --------------------------------------------------------------------------
# thin wrappers
# --------------------------------------------------------------------------
def philox4x64_10(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint64)
    k = np.ascontiguousarray(key, dtype=np.uint64)
    out = np.zeros(4, dtype=np.uint64)
    lib().orc_philox4x64_10(_ptr(c, ctypes.c_uint64), _ptr(k, ctypes.c_uint64), _ptr(out, ctypes.c_uint64))
    return out


def radius2_fixed(r, L):
    return int(lib().orc_radius2_fixed(r, L))


def n_cell(L, r_c):
    return int(lib().orc_n_cell(L, r_c))


def quantize(pos, L, r_c):
    pos = _f64(pos)
    n = pos.shape[0]
    s = np.zeros((n, 3), dtype=np.uint32)
    cell = np.zeros(n, dtype=np.int32)
    lib().orc_quantize(n, _ptr(pos, ctypes.c_double), L, r_c, _ptr(s, ctypes.c_uint32), _ptr(cell, ctypes.c_int32))
    return s, cell


def k_table(alpha, L):
    M = int(lib().orc_kmax(alpha, L))
    T = np.zeros(2 * M + 1, dtype=np.uint64)
    H = lib().orc_k_table(alpha, L, M, _ptr(T, ctypes.c_uint64))
    return M, H, T


def mh_tables(alpha, L):
    """Target w_m, proposal q_m and the proposal's inverse-CDF thresholds of the
    Metropolis-Hastings pool (reading R13), |m| <= M."""
    M = lib().orc_kmax(alpha, L)
    w, q = np.zeros(2 * M + 1), np.zeros(2 * M + 1)
    Tq = np.zeros(2 * M + 1, dtype=np.uint64)
    lib().orc_mh_tables(alpha, L, M, _ptr(w, ctypes.c_double), _ptr(q, ctypes.c_double),
                        _ptr(Tq, ctypes.c_uint64))
    return M, w, q, Tq


def kpool(seed, alpha, L, K, burn):
    """The pool [K, 3] and the chains' acceptance rate."""
    pool = np.zeros((K, 3), dtype=np.int32)
    acc = lib().orc_kpool(seed, alpha, L, K, burn, _ptr(pool, ctypes.c_int32))
    return pool, acc


def sample_k_params(pr, step):
    """The P wave-vector integers of a step under the parameters' sampling mode."""
    m = np.zeros((pr.P, 3), dtype=np.int32)
    lib().orc_sample_k_params(ctypes.byref(pr), step, _ptr(m, ctypes.c_int32))
    return m


def sample_k(seed, step, P, alpha, L):
    m = np.zeros((P, 3), dtype=np.int32)
    lib().orc_sample_k(seed, step, P, alpha, L, _ptr(m, ctypes.c_int32))
    return m


def S(alpha, L):
    return float(lib().orc_S(alpha, L))


def floyd(n, p, words):
    w = np.ascontiguousarray(words, dtype=np.uint64)
    out = np.zeros(p, dtype=np.uint64)
    lib().orc_floyd(n, p, _ptr(w, ctypes.c_uint64), _ptr(out, ctypes.c_uint64))
    return out


def lists(pos, pr, step, brute=False, cap_core=512, cap_shell=0, pos_b=None):
    """Per-atom C(i), S(i) sizes, core ids (canonical order), batch ids.
    With pos_b (and pr.skin > 0) the sets come from the stored lists of the
    rebuild positions pos_b (reading R15)."""
    pos = _f64(pos)
    pb = None if pos_b is None else _f64(pos_b)
    n = pos.shape[0]
    n_core = np.zeros(n, dtype=np.int32)
    n_shell = np.zeros(n, dtype=np.int32)
    n_batch = np.zeros(n, dtype=np.int32)
    core = np.full((n, cap_core), -1, dtype=np.int32) if cap_core else None
    cap_b = max(pr.p, 1)
    batch = np.full((n, cap_b), -1, dtype=np.int32)
    shell = np.full((n, cap_shell), -1, dtype=np.int32) if cap_shell else None
    tail = (ctypes.byref(pr), step, int(brute),
            _ptr(n_core, ctypes.c_int32), _ptr(n_shell, ctypes.c_int32), _ptr(n_batch, ctypes.c_int32),
            _ptr(core, ctypes.c_int32), cap_core, _ptr(batch, ctypes.c_int32), cap_b,
            _ptr(shell, ctypes.c_int32), cap_shell)
    if pb is None:
        st = lib().orc_lists(n, _ptr(pos, ctypes.c_double), *tail)
    else:
        st = lib().orc_lists_skin(n, _ptr(pos, ctypes.c_double), _ptr(pb, ctypes.c_double), *tail)
    return dict(status=st, n_core=n_core, n_shell=n_shell, n_batch=n_batch, core=core, batch=batch, shell=shell)


def skin_lists(pos_b, pr, brute=False, cap=2048):
    """The stored lists V(i) of reading R15 built at positions pos_b:
    (counts[n], ids[n, cap] in the order of V(i), status)."""
    pb = _f64(pos_b)
    n = pb.shape[0]
    counts = np.zeros(n, dtype=np.int32)
    ids = np.full((n, cap), -1, dtype=np.int32)
    st = lib().orc_skin_lists(n, _ptr(pb, ctypes.c_double), ctypes.byref(pr), int(brute),
                              _ptr(counts, ctypes.c_int32), _ptr(ids, ctypes.c_int32), cap)
    return counts, ids, st


def skin_displaced(pos, pos_b, L, skin):
    """Reading R15's rebuild test: True when some atom moved by more than
    skin/2 (fixed-point units) since pos_b."""
    return bool(lib().orc_skin_displaced(_f64(pos).shape[0], _ptr(_f64(pos), ctypes.c_double),
                                         _ptr(_f64(pos_b), ctypes.c_double), float(L), float(skin)))


def rho(pos, q, L, m):
    pos, q = _f64(pos), _f64(q)
    m = np.ascontiguousarray(m, dtype=np.int32)
    out = np.zeros((m.shape[0], 2))
    lib().orc_rho(pos.shape[0], _ptr(pos, ctypes.c_double), _ptr(q, ctypes.c_double), L, m.shape[0],
                  _ptr(m, ctypes.c_int32), _ptr(out, ctypes.c_double))
    return out[:, 0] + 1j * out[:, 1]


def rbe_forces(pos, q, typ, mol, pr, step, pos_b=None):
    """The IRBE estimator: dict(F, F_real, F_long, F_abs, E[6], W[6], corr, m, rho, status).

    F_abs holds, per force component, the sum of the absolute values of all
    its summands (the componentwise condition scale of the sum).  With pos_b
    (and pr.skin > 0) the sets C(i), S(i) come from the stored lists of the
    rebuild positions pos_b (reading R15)."""
    pos, q = _f64(pos), _f64(q)
    pb = None if pos_b is None else _f64(pos_b)
    typ, mol = _i32(typ), _i32(mol)
    n = pos.shape[0]
    F = np.zeros((n, 3)); Fr = np.zeros((n, 3)); Fl = np.zeros((n, 3)); Fa = np.zeros((n, 3))
    E = np.zeros(6); W = np.zeros(6); corr = np.zeros(3)
    m = np.zeros((pr.P, 3), dtype=np.int32)
    rh = np.zeros((pr.P, 2))
    c = ctypes.c_double
    tail = (_ptr(q, c), _ptr(typ, ctypes.c_int32), _ptr(mol, ctypes.c_int32),
            ctypes.byref(pr), step, _ptr(F, c), _ptr(Fr, c), _ptr(Fl, c), _ptr(E, c), _ptr(W, c),
            _ptr(corr, c), _ptr(m, ctypes.c_int32), _ptr(rh, c), _ptr(Fa, c))
    if pb is None:
        st = lib().orc_rbe_forces(n, _ptr(pos, c), *tail)
    else:
        st = lib().orc_rbe_forces_skin(n, _ptr(pos, c), _ptr(pb, c), *tail)
    return dict(F=F, F_real=Fr, F_long=Fl, F_abs=Fa, E=E, W=W, corr=corr, m=m, rho=rh[:, 0] + 1j * rh[:, 1],
                status=st)


def rbe_adjoint(pos, q, typ, mol, pr, step, gF=None):
    """Gradients of the estimator energy E and of L = sum_i gF_i . F_i with the
    draws of (seed, step) frozen: dEdq[n], dLdq[n] and, per ordered type pair
    (a, b), dEde, dEds, dLde, dLds [MAXT, MAXT] w.r.t. eps_ab and sigma_ab."""
    pos, q = _f64(pos), _f64(q)
    typ, mol = _i32(typ), _i32(mol)
    n = pos.shape[0]
    g = None if gF is None else _f64(gF)
    out = {k: np.zeros(n) for k in ("dEdq", "dLdq")}
    out.update({k: np.zeros((MAXT, MAXT)) for k in ("dEde", "dEds", "dLde", "dLds")})
    c = ctypes.c_double
    st = lib().orc_rbe_adjoint(n, _ptr(pos, c), _ptr(q, c), _ptr(typ, ctypes.c_int32), _ptr(mol, ctypes.c_int32),
                               ctypes.byref(pr), step, _ptr(g, c), _ptr(out["dEdq"], c), _ptr(out["dLdq"], c),
                               _ptr(out["dEde"], c), _ptr(out["dEds"], c), _ptr(out["dLde"], c), _ptr(out["dLds"], c))
    out["status"] = st
    return out


def ewald_exact(pos, q, typ, mol, pr, r_cut, kmax):
    pos, q = _f64(pos), _f64(q)
    typ, mol = _i32(typ), _i32(mol)
    n = pos.shape[0]
    F = np.zeros((n, 3)); E = np.zeros(6); W = np.zeros(6)
    c = ctypes.c_double
    lib().orc_ewald_exact(n, _ptr(pos, c), _ptr(q, c), _ptr(typ, ctypes.c_int32), _ptr(mol, ctypes.c_int32),
                          ctypes.byref(pr), float(r_cut), int(kmax), _ptr(F, c), _ptr(E, c), _ptr(W, c))
    return dict(F=F, E=E, W=W)


def direct_coulomb(pos, q, L, k_e, nshell):
    pos, q = _f64(pos), _f64(q)
    c = ctypes.c_double
    return float(lib().orc_direct_coulomb(pos.shape[0], _ptr(pos, c), _ptr(q, c), L, k_e, nshell))


def water_bonded(pos, L, nmol, kb, r0, kth, th0, first=0):
    pos = _f64(pos)
    F = np.zeros_like(pos)
    c = ctypes.c_double
    U = lib().orc_water_bonded(nmol, first, _ptr(pos, c), L, kb, r0, kth, th0, _ptr(F, c))
    return U, F


def vv_run(pos, vel, mass, q, typ, mol, pr, step0, nsteps, dt, accel, F0, water=None):
    """Velocity Verlet with the IRBE forces; water=(nmol, kb, r0, kth, th0) adds bonds."""
    pos, vel, mass, q = _f64(pos).copy(), _f64(vel).copy(), _f64(mass), _f64(q)
    typ, mol = _i32(typ), _i32(mol)
    F = _f64(F0).copy()
    n = pos.shape[0]
    tr = np.zeros((nsteps, 2))
    nmw, kb, r0, kth, th0 = water if water else (0, 0.0, 0.0, 0.0, 0.0)
    c = ctypes.c_double
    st = lib().orc_vv_run(n, _ptr(pos, c), _ptr(vel, c), _ptr(mass, c), _ptr(q, c), _ptr(typ, ctypes.c_int32),
                          _ptr(mol, ctypes.c_int32), ctypes.byref(pr), step0, nsteps, dt, accel,
                          nmw, kb, r0, kth, th0, _ptr(F, c), _ptr(tr, c))
    return dict(pos=pos, vel=vel, F=F, trace=tr, status=st)
