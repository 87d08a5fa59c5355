"""Seeded periodic boxes of the paper's system types (Sec. 2.3, Sec. 4.1).

The paper benchmarks liquid water and fcc metals (Ag there; Cu here, same
lattice type).  Its DFT datasets are not available, so these generators stand
in for them with the same shapes, densities and sizes:

* water: ``n`` rigid-geometry molecules at 1.0 g/cm^3, oxygens on a jittered
  cubic grid, hydrogens at 0.96 A and 104.5 degrees with a random orientation;
* fcc: ``k^3`` conventional cells of a lattice constant ``a`` with Gaussian
  displacements;
* high-entropy alloy (the paper's third system type, Sec. 4.1): an fcc random
  solid solution of five species in equal shares (Co, Cr, Fe, Mn, Ni, the
  Cantor alloy's elements), lattice constant 3.59 A.

Everything is drawn from ``numpy.random.Generator(PCG64(seed))``.  Cells are
3x3 arrays whose rows are the lattice vectors (A).  Species indices: H=0, O=1,
Cu=2 (the default three-element model of :mod:`synth.model`) and Co=3, Cr=4,
Fe=5, Mn=6, Ni=7 (models with ``n_elem = 8``).
"""

from __future__ import annotations

import dataclasses
import math

import numpy as np

SPECIES_H = 0
SPECIES_O = 1
SPECIES_CU = 2
SPECIES_HEA = (3, 4, 5, 6, 7)  # Co, Cr, Fe, Mn, Ni

# atomic masses in amu, indexed by species
MASS_AMU = np.array([1.008, 15.999, 63.546, 58.933, 51.996, 55.845, 54.938, 58.693], dtype=np.float64)

# volume per water molecule at 1.0 g/cm^3 (A^3): 18.015 g/mol / (N_A * 1 g/cm^3)
WATER_VOLUME_A3 = 29.915
OH_BOND_A = 0.96
HOH_ANGLE_DEG = 104.5

# Boltzmann constant (eV/K) and the unit conversion 1 eV/(A*amu) -> A/fs^2
KB_EV_PER_K = 8.617333262e-5
EV_PER_A_AMU_TO_A_PER_FS2 = 9.648533212e-3


@dataclasses.dataclass
class Structure:
    """A periodic (or free, when ``cell`` is None) atomic structure."""

    pos: np.ndarray  # (N, 3) float64, A
    species: np.ndarray  # (N,) int32
    cell: np.ndarray | None  # (3, 3) float64, rows = lattice vectors, A
    name: str = ""

    @property
    def n_atoms(self) -> int:
        return int(self.pos.shape[0])


def _random_rotations(rng: np.random.Generator, n: int) -> np.ndarray:
    """Uniform random rotation matrices from unit quaternions (Shoemake)."""
    u1, u2, u3 = rng.random((3, n))
    q = np.stack(
        [
            np.sqrt(1.0 - u1) * np.sin(2 * math.pi * u2),
            np.sqrt(1.0 - u1) * np.cos(2 * math.pi * u2),
            np.sqrt(u1) * np.sin(2 * math.pi * u3),
            np.sqrt(u1) * np.cos(2 * math.pi * u3),
        ],
        axis=1,
    )
    x, y, z, w = q.T
    r = np.empty((n, 3, 3))
    r[:, 0, 0] = 1 - 2 * (y * y + z * z)
    r[:, 0, 1] = 2 * (x * y - z * w)
    r[:, 0, 2] = 2 * (x * z + y * w)
    r[:, 1, 0] = 2 * (x * y + z * w)
    r[:, 1, 1] = 1 - 2 * (x * x + z * z)
    r[:, 1, 2] = 2 * (y * z - x * w)
    r[:, 2, 0] = 2 * (x * z - y * w)
    r[:, 2, 1] = 2 * (y * z + x * w)
    r[:, 2, 2] = 1 - 2 * (x * x + y * y)
    return r


def _resolve_contacts(rng, o_pos, h_pos, h_local, edge, min_contact, max_tries):
    """Re-draw the orientation of molecules whose hydrogens come closer than
    ``min_contact`` to an atom of another molecule (minimum image), in molecule
    order, up to ``max_tries`` rounds; liquid water has no such contacts."""
    from scipy.spatial import cKDTree

    n = o_pos.shape[0]
    mol = np.concatenate([np.arange(n)] * 3)
    is_h = np.concatenate([np.zeros(n, bool), np.ones(2 * n, bool)])
    for _ in range(max_tries):
        atoms = np.concatenate([o_pos, h_pos[:, 0], h_pos[:, 1]])
        tree = cKDTree(np.mod(atoms, edge), boxsize=edge)
        pairs = tree.query_pairs(min_contact, output_type="ndarray")
        if pairs.size:
            a, b = pairs[:, 0], pairs[:, 1]
            clash = (mol[a] != mol[b]) & (is_h[a] | is_h[b])
            a, b = a[clash], b[clash]
        else:
            a = b = np.zeros(0, int)
        if a.size == 0:
            break
        # re-orient the molecule that owns a clashing hydrogen (both if both are H)
        idx = np.unique(np.concatenate([mol[a][is_h[a]], mol[b][is_h[b]]]))
        rot = _random_rotations(rng, idx.size)
        h_pos[idx] = o_pos[idx, None, :] + np.einsum("nij,hj->nhi", rot, h_local)
    return h_pos


def water_box(n_molecules: int, seed: int = 0, jitter: float = 0.1, min_contact: float = 1.5,
              max_tries: int = 60) -> Structure:
    """Periodic cubic water box at 1.0 g/cm^3 with ``3 * n_molecules`` atoms.

    Edge ``L = (n * 29.915 A^3)^(1/3)``; oxygens sit on the first ``n`` sites
    (seeded permutation) of a ``g^3`` grid, ``g = ceil(n^(1/3))``, spacing
    ``L/g``, each jittered by N(0, jitter); the two hydrogens are placed at
    0.96 A with an H-O-H angle of 104.5 degrees in a uniformly random
    orientation, re-drawn while a hydrogen lies closer than ``min_contact``
    (A) to an atom of another molecule.  Atom order is (O, H, H) per molecule.
    """
    if n_molecules < 1:
        raise ValueError("n_molecules must be >= 1")
    rng = np.random.Generator(np.random.PCG64(seed))
    edge = (n_molecules * WATER_VOLUME_A3) ** (1.0 / 3.0)
    g = int(math.ceil(n_molecules ** (1.0 / 3.0) - 1e-9))
    if g ** 3 < n_molecules:
        g += 1
    spacing = edge / g
    sites = np.stack(np.meshgrid(np.arange(g), np.arange(g), np.arange(g), indexing="ij"), -1).reshape(-1, 3)
    chosen = sites[rng.permutation(sites.shape[0])[:n_molecules]]
    o_pos = (chosen + 0.5) * spacing + rng.normal(0.0, jitter, size=(n_molecules, 3))
    half = math.radians(HOH_ANGLE_DEG) / 2.0
    h_local = np.array(
        [
            [OH_BOND_A * math.sin(half), OH_BOND_A * math.cos(half), 0.0],
            [-OH_BOND_A * math.sin(half), OH_BOND_A * math.cos(half), 0.0],
        ]
    )
    rot = _random_rotations(rng, n_molecules)
    h_pos = o_pos[:, None, :] + np.einsum("nij,hj->nhi", rot, h_local)
    if min_contact > 0:
        h_pos = _resolve_contacts(rng, o_pos, h_pos, h_local, edge, min_contact, max_tries)
    pos = np.empty((n_molecules, 3, 3))
    pos[:, 0] = o_pos
    pos[:, 1:] = h_pos
    species = np.tile(np.array([SPECIES_O, SPECIES_H, SPECIES_H], dtype=np.int32), n_molecules)
    cell = np.eye(3) * edge
    return Structure(pos.reshape(-1, 3).copy(), species, cell, name=f"water{n_molecules}")


def fcc_box(k: int, a: float = 3.615, seed: int = 0, sigma: float = 0.05, species: int = SPECIES_CU) -> Structure:
    """Periodic fcc box of ``k^3`` conventional cells (``4 k^3`` atoms).

    Lattice constant ``a`` (A), every atom displaced by N(0, sigma) per
    component.  ``sigma = 0`` gives the perfect lattice.
    """
    if k < 1:
        raise ValueError("k must be >= 1")
    rng = np.random.Generator(np.random.PCG64(seed))
    basis = np.array([[0.0, 0.0, 0.0], [0.5, 0.5, 0.0], [0.5, 0.0, 0.5], [0.0, 0.5, 0.5]])
    cells = np.stack(np.meshgrid(np.arange(k), np.arange(k), np.arange(k), indexing="ij"), -1).reshape(-1, 3)
    frac = (cells[:, None, :] + basis[None, :, :]).reshape(-1, 3)
    pos = frac * a
    if sigma > 0:
        pos = pos + rng.normal(0.0, sigma, size=pos.shape)
    n = pos.shape[0]
    return Structure(pos, np.full(n, species, dtype=np.int32), np.eye(3) * (k * a), name=f"fcc{k}")


def hea_box(k: int, a: float = 3.59, seed: int = 0, sigma: float = 0.05, species=SPECIES_HEA) -> Structure:
    """fcc random solid solution: ``4 k^3`` atoms, the species in equal shares
    (as equal as the atom count allows) on a seeded random permutation of the
    sites, N(0, sigma) displacements."""
    s = fcc_box(k, a=a, seed=seed, sigma=sigma)
    rng = np.random.Generator(np.random.PCG64([seed, 1]))
    n = s.n_atoms
    kinds = np.asarray(species, dtype=np.int32)
    labels = np.resize(kinds, n)
    rng.shuffle(labels)
    return Structure(s.pos, labels.astype(np.int32), s.cell, name=f"hea{k}")


def supercell(s: Structure, reps: tuple[int, int, int]) -> Structure:
    """Periodic repetition ``reps[0] x reps[1] x reps[2]`` of a structure."""
    if s.cell is None:
        raise ValueError("supercell needs a periodic structure")
    na, nb, nc = reps
    shifts = np.stack(np.meshgrid(np.arange(na), np.arange(nb), np.arange(nc), indexing="ij"), -1).reshape(-1, 3)
    disp = shifts.astype(np.float64) @ s.cell
    pos = (s.pos[None, :, :] + disp[:, None, :]).reshape(-1, 3)
    species = np.tile(s.species, shifts.shape[0])
    cell = s.cell * np.array([[na], [nb], [nc]], dtype=np.float64)
    return Structure(pos, species.astype(np.int32), cell, name=f"{s.name}x{na}{nb}{nc}")


def maxwell_boltzmann(masses_amu: np.ndarray, temperature_k: float, seed: int = 0) -> np.ndarray:
    """Velocities (A/fs) at exactly ``temperature_k`` with zero total momentum.

    Drawn from the Maxwell-Boltzmann distribution, the centre-of-mass
    momentum removed, then rescaled so that the kinetic energy equals
    ``(3N - 3) k_B T / 2``.
    """
    m = np.asarray(masses_amu, dtype=np.float64)
    n = m.shape[0]
    rng = np.random.Generator(np.random.PCG64(seed))
    # sigma_v^2 = k_B T / m in (eV/amu) -> (A/fs)^2 via the unit factor
    sig = np.sqrt(KB_EV_PER_K * temperature_k / m * EV_PER_A_AMU_TO_A_PER_FS2)
    v = rng.normal(size=(n, 3)) * sig[:, None]
    p = (m[:, None] * v).sum(0)
    v -= p / m.sum()
    ke = 0.5 * (m[:, None] * v * v).sum() / EV_PER_A_AMU_TO_A_PER_FS2  # eV
    target = 0.5 * (3 * n - 3) * KB_EV_PER_K * temperature_k
    if n > 1 and ke > 0:
        v *= math.sqrt(target / ke)
    return v
