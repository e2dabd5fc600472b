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
from scipy.spatial import cKDTree

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


def _rsa(rng, n, L, dmin, chunk=2048):
    """Random sequential insertion of n points in a periodic cube, min distance dmin.

    Candidates are uniform points drawn three coordinates at a time from rng;
    each is accepted when it is at least dmin (minimum image) from every point
    accepted before it.  Candidates are drawn in chunks and tested against the
    accepted set through a grid of cells of edge < dmin/sqrt(3) (at most one
    point per cell), then in order against the chunk's earlier acceptances; on
    return rng has consumed exactly the candidates up to the n-th acceptance,
    as a one-at-a-time insertion would."""
    state = rng.bit_generator.state
    nc = int(math.floor(L * math.sqrt(3.0) / dmin)) + 1
    w = L / nc
    reach = int(math.ceil(dmin / w))
    rr = np.arange(-reach, reach + 1)
    offs = np.stack(np.meshgrid(rr, rr, rr, indexing="ij"), -1).reshape(-1, 3)
    grid = np.full(nc ** 3, -1, dtype=np.int64)
    out = np.zeros((n, 3))
    k = 0
    used = 0
    d2min = dmin * dmin
    while k < n:
        if used > 200 * n + 10000:
            raise RuntimeError("random sequential insertion did not converge")
        X = rng.random((chunk, 3)) * L
        c = np.floor(X / w).astype(np.int64) % nc
        nb = (c[:, None, :] + offs[None, :, :]) % nc
        occ = grid[nb[..., 0] + nc * (nb[..., 1] + nc * nb[..., 2])]
        ti, si = np.nonzero(occ >= 0)
        d = out[occ[ti, si]] - X[ti]
        d -= L * np.round(d / L)
        clash = np.zeros(chunk, dtype=bool)
        clash[ti[(d * d).sum(-1) < d2min]] = True
        # in order against the chunk's earlier acceptances: only candidates
        # within dmin of an earlier candidate need the sequential test
        acc = ~clash
        cand = np.nonzero(acc)[0]
        if cand.size > 1:
            pairs = cKDTree(X[cand], boxsize=L).query_pairs(dmin, output_type="ndarray")
            if pairs.size:
                i, j = cand[pairs[:, 0]], cand[pairs[:, 1]]
                e = X[i] - X[j]
                e -= L * np.round(e / L)
                near = (e * e).sum(-1) < d2min
                i, j = np.minimum(i, j)[near], np.maximum(i, j)[near]
                order = np.argsort(j, kind="stable")
                for a, b in zip(i[order], j[order]):
                    if acc[a]:
                        acc[b] = False
        take = np.nonzero(acc)[0][: n - k]
        if take.size:
            ci = c[take]
            grid[ci[:, 0] + nc * (ci[:, 1] + nc * ci[:, 2])] = np.arange(k, k + take.size)
            out[k:k + take.size] = X[take]
            k += take.size
        used += int(take[-1]) + 1 if k == n else chunk
    # leave rng where a one-candidate-at-a-time insertion would have left it
    rng.bit_generator.state = state
    rng.random((used, 3))
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


def electrolyte_2to1(n_cations: int = 1280, L: float = 80.0, seed: int = 1, r_c: float = 5.0, r_s: float = 15.0,
                     p: int = 10, P: int = 100, dt: float = 0.002) -> System:
    """2:1 primitive electrolyte (Sec. 3.1): n_cations divalent cations (+2)
    and 2 n_cations monovalent anions (-1), equal soft spheres (sigma = eps =
    1), random sequential insertion at minimum distance 1 sigma; the charges
    repeat +2, -1, -1 along the atom index."""
    n = 3 * n_cations
    rng = np.random.default_rng(seed)
    pos = _rsa(rng, n, L, 1.0)
    q = np.where(np.arange(n) % 3 == 0, 2.0, -1.0)
    typ = np.zeros(n, dtype=np.int32)
    mass = np.ones(n)
    vel = _maxwell(rng, mass, 1.0, 1.0)
    return System("electrolyte_2to1", L, pos, q, typ, None, mass, vel, alpha_for(r_s), r_c, r_s, p, P,
                  K_E_REDUCED, (1.0,), (1.0,), 1.0, dt, seed)


def slab_ions(n: int = 8000, L: float = 32.0, slab_frac: float = 0.5, slab_width: float = 3.0, seed: int = 11,
              r_c: float = 2.5, r_s: float = 5.0, p: int = 10, P: int = 100) -> System:
    """A strongly inhomogeneous charged system (an edge case, not a paper
    workload): n uniformly random point charges (+1/-1 alternating, no LJ),
    the first slab_frac of them confined to the slab 0 <= z < slab_width, so
    that the local density there is several times the mean."""
    assert n % 2 == 0
    rng = np.random.default_rng(seed)
    pos = rng.random((n, 3)) * L
    k = int(slab_frac * n)
    pos[:k, 2] = rng.random(k) * slab_width
    q = np.where(np.arange(n) % 2 == 0, 1.0, -1.0)
    typ = np.zeros(n, dtype=np.int32)
    mass = np.ones(n)
    vel = _maxwell(rng, mass, 1.0, 1.0)
    return System("slab_ions", L, pos, q, typ, None, mass, vel, alpha_for(r_s), r_c, r_s, p, P,
                  K_E_REDUCED, (0.0,), (1.0,), 1.0, 0.002, seed)


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


def batch_replicas(nrep: int = 64, n_min: int = 1000, n_max: int = 50000, seed0: int = 0) -> list:
    """A suite of independent systems of uneven size for batched stepping:
    replica r (seed seed0 + r) has about N atoms with log N uniform in
    [log n_min, log n_max] (drawn from a generator seeded with seed0); even
    seeds are 1:1 electrolytes (N even, P = 100, density 0.25 sigma^-3 as in
    the 2,000-ion box of side 20 sigma), odd seeds water boxes (N a multiple
    of 3, P = 200).  Each replica has its own box, alpha and cutoffs."""
    rng = np.random.default_rng(seed0 + 7919)
    out = []
    for r in range(nrep):
        seed = seed0 + r
        N = float(np.exp(rng.uniform(math.log(n_min), math.log(n_max))))
        if seed % 2 == 0:
            n = max(2, int(round(N / 2)) * 2)
            L = (n / 0.25) ** (1.0 / 3.0)
            out.append(electrolyte(n=n, L=L, seed=seed, P=100))
        else:
            out.append(water(n_mol=max(1, int(round(N / 3))), seed=seed, P=200))
    return out


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
