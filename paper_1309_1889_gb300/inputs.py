"""Seeded synthetic inputs: water-like point-charge boxes and random charge clouds.

This module draws inputs only.  It holds none of the method's arithmetic (no
smoothing, basis, grid or integrator code), so both the CUDA path and the
FP64 oracle can be fed from it without sharing any computation.

Water-like boxes follow the workloads used to exercise the multilevel
summation method (MSM): rigid 3-site molecules with charges O -0.834 e and
H +0.417 e, O-H 0.09572 nm, H-O-H 104.52 degrees, about 100 atoms/nm^3.

Recipe (all with numpy PCG64):
  * molecule sites: the first ``n_mol`` entries of a seeded permutation of a
    regular lattice of ceil(L_d / s) sites per axis, s = (V / n_mol)^(1/3),
    site spacing L_d / n_d so the lattice fills the water region;
  * each site jittered by U(-0.05 s, 0.05 s) per axis, the O atom on the site;
  * orientation: a uniform random rotation (Shoemake's quaternion recipe);
  * optional filler sites (charge 0, mass 22.99) on the next lattice sites,
    used to reach an exact atom count such as 100,000 or 1,000,000;
  * velocities: Maxwell-Boltzmann at T per molecule centre of mass (a second
    seed), zero angular velocity, centre-of-mass drift removed.

Atom order: molecule m owns atoms 3m (O), 3m+1 (H), 3m+2 (H); fillers follow.
Units: nm, ps, e, amu, kJ/mol.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

Q_O = -0.834
Q_H = 0.417
M_O = 15.9994
M_H = 1.008
M_FILLER = 22.99
D_OH = 0.09572
ANGLE_HOH_DEG = 104.52
KB_KJ_PER_MOL_K = 0.0083144626


def d_hh() -> float:
    """H-H distance of the rigid geometry (law of cosines on the two O-H bonds)."""
    return 2.0 * D_OH * math.sin(math.radians(ANGLE_HOH_DEG) / 2.0)


@dataclass
class System:
    """A synthetic system: positions, charges, masses and (optionally) velocities.

    ``box`` is (x0, y0, z0, Lx, Ly, Lz): the open, non-periodic domain that
    every atom must stay inside while the MSM grids cover it.
    """

    pos: np.ndarray                 # (n, 3) float64, nm
    q: np.ndarray                   # (n,) float64, e
    mass: np.ndarray                # (n,) float64, amu
    box: np.ndarray                 # (6,) float64
    vel: np.ndarray | None = None   # (n, 3) float64, nm/ps
    n_mol: int = 0                  # leading rigid (O, H, H) triples
    lj: np.ndarray | None = None    # (n,) uint8, 1 = O-O Lennard-Jones site
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.pos.shape[0])


def _shoemake_rotations(rng: np.random.Generator, k: int) -> np.ndarray:
    """k uniform random rotation matrices from uniform quaternions (Shoemake 1992)."""
    u1, u2, u3 = rng.random(k), rng.random(k), rng.random(k)
    a = np.sqrt(1.0 - u1)
    b = np.sqrt(u1)
    w = a * np.sin(2 * np.pi * u2)
    x = a * np.cos(2 * np.pi * u2)
    y = b * np.sin(2 * np.pi * u3)
    z = b * np.cos(2 * np.pi * u3)
    R = np.empty((k, 3, 3))
    R[:, 0, 0] = 1 - 2 * (y * y + z * z)
    R[:, 0, 1] = 2 * (x * y - z * w)
    R[:, 0, 2] = 2 * (x * z + y * w)
    R[:, 1, 0] = 2 * (x * y + z * w)
    R[:, 1, 1] = 1 - 2 * (x * x + z * z)
    R[:, 1, 2] = 2 * (y * z - x * w)
    R[:, 2, 0] = 2 * (x * z - y * w)
    R[:, 2, 1] = 2 * (y * z + x * w)
    R[:, 2, 2] = 1 - 2 * (x * x + y * y)
    return R


def water_box(n_atoms: int, region, *, seed: int = 0, vel_seed: int = 1,
              temperature: float = 300.0, margin: float = 0.5,
              with_velocities: bool = True) -> System:
    """Water-like box of exactly ``n_atoms`` atoms filling ``region`` (nm).

    ``region`` is a scalar cube edge or a 3-tuple of edges.  ``n_atoms // 3``
    molecules are placed; the remainder (0-2 atoms) become zero-charge filler
    sites.  The returned box extends the water region by ``margin`` on every
    side so atoms may move during dynamics without leaving the domain.
    """
    Ld = np.broadcast_to(np.asarray(region, dtype=np.float64), (3,)).copy()
    n_mol = n_atoms // 3
    n_fill = n_atoms - 3 * n_mol
    n_sites_needed = n_mol + n_fill
    vol = float(np.prod(Ld))
    s = (vol / max(n_sites_needed, 1)) ** (1.0 / 3.0)
    nd = np.maximum(np.ceil(Ld / s).astype(np.int64), 1)
    while int(np.prod(nd)) < n_sites_needed:
        nd += 1
    spacing = Ld / nd
    rng = np.random.Generator(np.random.PCG64(seed))
    order = rng.permutation(int(np.prod(nd)))[:n_sites_needed]
    iz, rem = np.divmod(order, nd[0] * nd[1])
    iy, ix = np.divmod(rem, nd[0])
    sites = (np.stack([ix, iy, iz], axis=1) + 0.5) * spacing
    sites = sites + rng.uniform(-0.05 * s, 0.05 * s, size=sites.shape)

    half = math.radians(ANGLE_HOH_DEG) / 2.0
    body = np.array([[0.0, 0.0, 0.0],
                     [D_OH * math.sin(half), D_OH * math.cos(half), 0.0],
                     [-D_OH * math.sin(half), D_OH * math.cos(half), 0.0]])
    R = _shoemake_rotations(rng, n_mol)
    mol = np.einsum("kij,sj->ksi", R, body) + sites[:n_mol, None, :]

    n = 3 * n_mol + n_fill
    pos = np.empty((n, 3))
    pos[:3 * n_mol] = mol.reshape(-1, 3)
    pos[3 * n_mol:] = sites[n_mol:]
    q = np.zeros(n)
    q[0:3 * n_mol:3] = Q_O
    q[1:3 * n_mol:3] = Q_H
    q[2:3 * n_mol:3] = Q_H
    mass = np.full(n, M_FILLER)
    mass[0:3 * n_mol:3] = M_O
    mass[1:3 * n_mol:3] = M_H
    mass[2:3 * n_mol:3] = M_H
    lj = np.zeros(n, dtype=np.uint8)
    lj[0:3 * n_mol:3] = 1
    lj[3 * n_mol:] = 1

    vel = None
    if with_velocities:
        vrng = np.random.Generator(np.random.PCG64(vel_seed))
        kT = KB_KJ_PER_MOL_K * temperature
        m_mol = M_O + 2 * M_H
        vmol = vrng.normal(0.0, math.sqrt(kT / m_mol), size=(n_mol, 3))
        vfill = vrng.normal(0.0, math.sqrt(kT / M_FILLER), size=(n_fill, 3))
        vel = np.empty((n, 3))
        vel[:3 * n_mol] = np.repeat(vmol, 3, axis=0)
        vel[3 * n_mol:] = vfill
        p = (mass[:, None] * vel).sum(axis=0) / mass.sum()
        vel -= p

    box = np.concatenate([-np.full(3, margin), Ld + 2 * margin])
    return System(pos=pos, q=q, mass=mass, box=box, vel=vel, n_mol=n_mol, lj=lj,
                  meta={"kind": "water", "region": Ld.tolist(), "seed": seed,
                        "vel_seed": vel_seed, "margin": margin})


def random_cloud(n: int, length, *, seed: int = 0, neutral: bool = True,
                 margin: float = 0.0) -> System:
    """Uniform random positions in a box with charges U(-1, 1) (optionally neutralised).

    Used for unit checks of the electrostatics alone (no molecules, no velocities).
    """
    L = np.broadcast_to(np.asarray(length, dtype=np.float64), (3,)).copy()
    rng = np.random.Generator(np.random.PCG64(seed))
    pos = rng.random((n, 3)) * L
    q = rng.uniform(-1.0, 1.0, n)
    if neutral and n > 1:
        q -= q.mean()
    box = np.concatenate([-np.full(3, margin), L + 2 * margin])
    return System(pos=pos, q=q, mass=np.ones(n), box=box,
                  meta={"kind": "cloud", "seed": seed})


# Workload table: sizes of the water-like systems the method is exercised on.
WORKLOADS = {
    # 1000 molecules in a 3.1 nm cube, 3 levels, direct-sum check + 100 steps.
    "water3k": dict(n_atoms=3000, region=3.1, a=1.2, h=0.25, levels=3),
    # 100,000 atoms in a 10 nm cube, 4 levels (autograd / finite differences).
    "water100k": dict(n_atoms=100_000, region=10.0, a=1.2, h=0.25, levels=4),
    # 10,000 atoms in a 4.65 nm cube (parareal fine propagator: 3 levels).
    "water10k": dict(n_atoms=10_000, region=4.65, a=1.2, h=0.25, levels=3),
    # 1,000,000 atoms in a 21.5 nm cube, 5 levels (throughput workload).
    "water1M": dict(n_atoms=1_000_000, region=21.5, a=1.2, h=0.25, levels=5),
    # 12.7 M atoms in a 30 x 65 x 65 nm slab, 6 levels.
    "water12.7M": dict(n_atoms=12_700_000, region=(30.0, 65.0, 65.0), a=1.2, h=0.25, levels=6),
}
