"""Seeded synthetic systems for the IRBE force step.

This module only generates inputs (positions, charges, types, molecule ids,
masses, velocities) and the run parameters of each workload; it holds none of
the method's arithmetic.  Both the CUDA path and the CPU oracle consume what
it returns.

Workloads (shapes and densities of the paper's test systems, Sec. 3):
  * ``electrolyte``: primitive 1:1 electrolyte, charged LJ spheres (sigma=eps=1)
    placed by random sequential insertion with minimum distance 1 sigma,
    Coulomb prefactor k_e = 1.4 (Bjerrum length 1.4 sigma at kT = 1), reduced
    units (Sec. 3.1 describes the same model).
  * ``water``: rigid-geometry 3-site water (O -0.8476 e, H +0.4238 e, LJ on O
    only: sigma 3.166 A, eps 0.650 kJ/mol; O-H 1.0 A, H-O-H 109.47 deg) on a
    cubic lattice at 0.0334 molecules/A^3 with uniformly random orientations,
    k_e = 1389.35458 kJ mol^-1 A e^-2, masses in g/mol, forces in kJ/mol/A
    (the SPC/E-like bulk water of Sec. 3.2).
alpha is chosen so that erfc(sqrt(alpha) r_s) = 1e-4 in both.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

WATER_DENSITY = 0.0334          # molecules per A^3
K_E_WATER = 1389.35458          # kJ mol^-1 A e^-2
K_E_REDUCED = 1.4               # Bjerrum length 1.4 sigma, kT = 1
ACCEL_WATER = 1.0e-4            # (kJ/mol/A) / (g/mol) -> A/fs^2
KT_WATER = 2.4777               # kJ/mol at 298 K
M_O, M_H = 15.9994, 1.008
Q_O, Q_H = -0.8476, 0.4238
THETA_HOH = math.radians(109.47)
R_OH = 1.0
# harmonic bond constants chosen for the flexible water used by the
# velocity-Verlet runs (U = 1/2 k (x - x0)^2)
KB_OH = 4000.0                  # kJ mol^-1 A^-2
KTH_HOH = 400.0                 # kJ mol^-1 rad^-2


def alpha_for(r_s: float, tol: float = 1e-4) -> float:
    """alpha such that erfc(sqrt(alpha) r_s) = tol (bisection on x = sqrt(alpha) r_s)."""
    lo, hi = 0.0, 10.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if math.erfc(mid) > tol:
            lo = mid
        else:
            hi = mid
    x = 0.5 * (lo + hi)
    return (x / r_s) ** 2


@dataclass
class System:
    name: str
    L: float
    pos: np.ndarray            # [N,3] float64
    q: np.ndarray              # [N] float64
    type: np.ndarray           # [N] int32
    mol: np.ndarray | None     # [N] int32 or None
    mass: np.ndarray           # [N] float64
    vel: np.ndarray            # [N,3] float64
    alpha: float
    r_c: float
    r_s: float
    p: int
    P: int
    k_e: float
    eps: tuple
    sigma: tuple
    accel: float               # force/mass -> acceleration unit factor
    dt: float
    seed: int
    n_water_mol: int = 0       # molecules with bonded terms (atoms 0..3n-1)
    bonds: tuple = field(default_factory=tuple)  # (kb, r0, kth, th0)

    @property
    def n(self) -> int:
        return int(self.pos.shape[0])


def _maxwell(rng, mass, kT, accel):
    sd = np.sqrt(kT * accel / mass)[:, None]
    v = rng.standard_normal((mass.shape[0], 3)) * sd
    p = (v * mass[:, None]).sum(0) / mass.sum()
    return v - p


def _rsa(rng, n, L, dmin):
    """Random sequential insertion of n points in a periodic cube, min distance dmin."""
    nc = max(1, int(L // dmin))
    w = L / nc
    cells: dict = {}
    out = np.zeros((n, 3))
    k = 0
    tries = 0
    while k < n:
        tries += 1
        if tries > 200 * n + 10000:
            raise RuntimeError("random sequential insertion did not converge")
        x = rng.random(3) * L
        c = (x // w).astype(int) % nc
        ok = True
        for dx in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dz in (-1, 0, 1):
                    key = ((c[0] + dx) % nc, (c[1] + dy) % nc, (c[2] + dz) % nc)
                    for j in cells.get(key, ()):
                        d = out[j] - x
                        d -= L * np.round(d / L)
                        if d @ d < dmin * dmin:
                            ok = False
                            break
                    if not ok:
                        break
                if not ok:
                    break
            if not ok:
                break
        if ok:
            out[k] = x
            cells.setdefault((c[0], c[1], c[2]), []).append(k)
            k += 1
    return out


def electrolyte(n: int = 2000, L: float = 20.0, seed: int = 1, r_c: float = 2.5, r_s: float = 5.0,
                p: int = 10, P: int = 100, dt: float = 0.002) -> System:
    """1:1 primitive electrolyte: n/2 cations (+1), n/2 anions (-1)."""
    assert n % 2 == 0
    rng = np.random.default_rng(seed)
    pos = _rsa(rng, n, L, 1.0)
    q = np.where(np.arange(n) % 2 == 0, 1.0, -1.0)
    typ = np.zeros(n, dtype=np.int32)
    mass = np.ones(n)
    vel = _maxwell(rng, mass, 1.0, 1.0)
    return System("electrolyte", L, pos, q, typ, None, mass, vel, alpha_for(r_s), r_c, r_s, p, P,
                  K_E_REDUCED, (1.0,), (1.0,), 1.0, dt, seed)


def _random_rotations(rng, n):
    """Uniform random rotation matrices from unit quaternions (Shoemake 1992)."""
    u1, u2, u3 = rng.random(n), rng.random(n), rng.random(n)
    a = np.sqrt(1 - u1) * np.sin(2 * np.pi * u2)
    b = np.sqrt(1 - u1) * np.cos(2 * np.pi * u2)
    c = np.sqrt(u1) * np.sin(2 * np.pi * u3)
    d = np.sqrt(u1) * np.cos(2 * np.pi * u3)
    w, x, y, z = d, a, b, c
    R = np.empty((n, 3, 3))
    R[:, 0, 0] = 1 - 2 * (y * y + z * z); R[:, 0, 1] = 2 * (x * y - z * w); R[:, 0, 2] = 2 * (x * z + y * w)
    R[:, 1, 0] = 2 * (x * y + z * w); R[:, 1, 1] = 1 - 2 * (x * x + z * z); R[:, 1, 2] = 2 * (y * z - x * w)
    R[:, 2, 0] = 2 * (x * z - y * w); R[:, 2, 1] = 2 * (y * z + x * w); R[:, 2, 2] = 1 - 2 * (x * x + y * y)
    return R


def water(n_mol: int = 30000, seed: int = 2, r_c: float = 5.0, r_s: float = 10.0, p: int = 20,
          P: int = 200, dt: float = 1.0) -> System:
    """n_mol 3-site water molecules on a lattice subset with random orientations."""
    rng = np.random.default_rng(seed)
    L = (n_mol / WATER_DENSITY) ** (1.0 / 3.0)
    side = int(math.ceil(n_mol ** (1.0 / 3.0) - 1e-9))
    a = L / side
    sites = rng.permutation(side ** 3)[:n_mol]
    ix, iy, iz = sites % side, (sites // side) % side, sites // (side * side)
    centre = (np.stack([ix, iy, iz], 1) + 0.5) * a
    h = 0.5 * THETA_HOH
    local = np.array([[0.0, 0.0, 0.0],
                      [R_OH * math.sin(h), R_OH * math.cos(h), 0.0],
                      [-R_OH * math.sin(h), R_OH * math.cos(h), 0.0]])
    Rm = _random_rotations(rng, n_mol)
    atoms = centre[:, None, :] + np.einsum("mab,kb->mka", Rm, local)
    pos = atoms.reshape(-1, 3) % L
    q = np.tile([Q_O, Q_H, Q_H], n_mol)
    typ = np.tile(np.array([0, 1, 1], dtype=np.int32), n_mol)
    mol = np.repeat(np.arange(n_mol, dtype=np.int32), 3)
    mass = np.tile([M_O, M_H, M_H], n_mol)
    vel = _maxwell(rng, mass, KT_WATER, ACCEL_WATER)
    return System("water", L, pos, q, typ, mol, mass, vel, alpha_for(r_s), r_c, r_s, p, P,
                  K_E_WATER, (0.650, 0.0), (3.166, 1.0), ACCEL_WATER, dt, seed,
                  n_water_mol=n_mol, bonds=(KB_OH, R_OH, KTH_HOH, THETA_HOH))


def nacl_crystal(cells: int = 2, r0: float = 1.0):
    """Rock-salt supercell of cells^3 conventional cubes (8 ions each), edge 2 r0."""
    base = np.array([[0, 0, 0], [1, 1, 0], [1, 0, 1], [0, 1, 1],
                     [1, 0, 0], [0, 1, 0], [0, 0, 1], [1, 1, 1]], dtype=float)
    qb = np.array([1, 1, 1, 1, -1, -1, -1, -1], dtype=float)
    pos, q = [], []
    for i in range(cells):
        for j in range(cells):
            for k in range(cells):
                pos.append((base + 2 * np.array([i, j, k])) * r0)
                q.append(qb)
    return np.concatenate(pos), np.concatenate(q), 2.0 * r0 * cells
