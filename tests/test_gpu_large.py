"""Full-size parity on the 1,048,576-atom fcc Cu box (64^3 cells), in the launch
configuration the library uses for any size.

The oracle cannot evaluate a million atoms with its O(N^2) list, but REANN's
receptive field is T r_c (Sec. 2.2, Fig. 2): the atomic energy of atom a
depends only on atoms within T r_c of it, and its force only on atoms within
2 T r_c.  So for sampled atoms the oracle evaluates a free cluster cut from the
periodic box around the atom (radius T r_c + 1 A for the energy, 2 T r_c + 1 A
for the force) and must reproduce the GPU's full-box values.
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
    for a in rng.choice(s.n_atoms, size=3, replace=False):
        pos_e, sp_e = _cluster(s, a, T * spec.r_c + 1.0)
        ref_e = oracle.energy_forces(spec, pos_e, sp_e, None)["atom_energy"][0]
        pos_f, sp_f = _cluster(s, a, 2 * T * spec.r_c + 1.0)
        ref_f = oracle.energy_forces(spec, pos_f, sp_f, None)["forces"][0]
        print(f"[1M] atom {a}: d_eps={abs(eps[a] - ref_e):.2e} eV  max|dF|={np.abs(forces[a] - ref_f).max():.2e} eV/A "
              f"(cluster sizes {len(sp_e)}, {len(sp_f)})")
        assert abs(eps[a] - ref_e) < 1e-5
        assert np.abs(forces[a] - ref_f).max() < F_TOL_MAX
