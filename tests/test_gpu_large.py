"""Full-size parity on the 1,048,576-atom fcc Cu box (64^3 cells), in the launch
configuration the library uses for any size.

The oracle cannot evaluate a million atoms with its O(N^2) list, but REANN's
receptive field is T r_c (Sec. 2.2, Fig. 2): the atomic energy of atom a
depends only on atoms within T r_c of it, and its force only on atoms within
2 T r_c.  So for sampled atoms the oracle evaluates a free cluster cut from the
periodic box around the atom (radius T r_c + 1 A for the energy, 2 T r_c + 1 A
for the force) and must reproduce the GPU's full-box values.  32 atoms are
sampled: 16 anywhere, 16 whose r_c + skin shell crosses a face of the cell (4
of them near an edge or corner), whose neighbours are periodic images.
"""

from __future__ import annotations

import numpy as np
import pytest

import oracle
from synth import fcc_box, make_model

from gpu_helpers import F_TOL_MAX, potential

pytestmark = pytest.mark.gpu


def _cluster(s, a, radius):
    """Atoms within `radius` of atom a (minimum image in the cubic box), unwrapped around a."""
    L = s.cell[0, 0]
    d = s.pos - s.pos[a]
    d -= L * np.round(d / L)
    keep = np.nonzero((d * d).sum(1) < radius * radius)[0]
    order = np.concatenate([[a], keep[keep != a]])
    return d[order], s.species[order]


def test_million_atom_cu_box_sampled_against_oracle_clusters():
    import torch

    s = fcc_box(64, seed=0)
    assert s.n_atoms == 1_048_576
    T = 3
    spec = make_model(T=T)
    sy = potential(spec).system(s.pos, s.species, s.cell, skin=1.0)
    sy.evaluate()
    sy.check()
    torch.cuda.synchronize()
    eps = sy.atom_energy.double().cpu().numpy()
    forces = sy.forces.double().cpu().numpy()
    sy.close()
    rng = np.random.default_rng(64)
    # 16 atoms anywhere, and 16 whose r_c + skin shell crosses a face of the cell (their
    # neighbours include periodic images, i.e. ghost slots), 4 of them near an edge or corner
    L = s.cell[0, 0]
    frac = np.mod(s.pos / L, 1.0)
    edge = np.minimum(frac, 1.0 - frac) * L < spec.r_c + 1.0  # per axis: within r_c + skin of a face
    near_face = np.nonzero(edge.any(axis=1))[0]
    near_corner = np.nonzero(edge.sum(axis=1) >= 2)[0]
    picks = np.concatenate([
        rng.choice(s.n_atoms, size=16, replace=False),
        rng.choice(near_face, size=12, replace=False),
        rng.choice(near_corner, size=4, replace=False),
    ])
    worst_e = worst_f = 0.0
    for a in picks:
        pos_e, sp_e = _cluster(s, a, T * spec.r_c + 1.0)
        ref_e = oracle.energy_forces(spec, pos_e, sp_e, None)["atom_energy"][0]
        pos_f, sp_f = _cluster(s, a, 2 * T * spec.r_c + 1.0)
        ref_f = oracle.energy_forces(spec, pos_f, sp_f, None)["forces"][0]
        print(f"[1M] atom {a}: d_eps={abs(eps[a] - ref_e):.2e} eV  max|dF|={np.abs(forces[a] - ref_f).max():.2e} eV/A "
              f"(cluster sizes {len(sp_e)}, {len(sp_f)})")
        worst_e = max(worst_e, abs(eps[a] - ref_e))
        worst_f = max(worst_f, float(np.abs(forces[a] - ref_f).max()))
    print(f"[1M] {len(picks)} atoms: max d_eps={worst_e:.2e} eV, max|dF|={worst_f:.2e} eV/A")
    assert worst_e < 1e-5
    assert worst_f < F_TOL_MAX
