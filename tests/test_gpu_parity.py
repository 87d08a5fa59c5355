"""CUDA path vs the FP64 oracle on identical seeded inputs (FP32 networks).

Bar: neighbour sets bit-exact (as sets of (i, j, image shift)); energy within
1e-6 eV/atom and forces within 1e-4 eV/A max-abs of the oracle.
"""

from __future__ import annotations

import numpy as np
import pytest

import oracle
from synth import fcc_box, make_model, water_box
from synth.structures import Structure

from gpu_helpers import E_TOL_PER_ATOM, F_TOL_MAX, assert_parity, gpu_eval, potential

pytestmark = pytest.mark.gpu


def _triclinic(n=40, seed=3):
    rng = np.random.default_rng(seed)
    cell = np.array([[11.0, 0.0, 0.0], [2.5, 10.2, 0.0], [-1.7, 1.3, 10.8]])
    # jittered grid so no two atoms are too close
    g = np.stack(np.meshgrid(*[np.arange(4)] * 3, indexing="ij"), -1).reshape(-1, 3)[:n]
    frac = (g + 0.5) / 4 + rng.normal(0, 0.02, size=(n, 3))
    pos = frac @ cell + rng.integers(-2, 3, size=(n, 3)) @ cell  # some atoms in other images
    sp = rng.integers(0, 3, size=n).astype(np.int32)
    return Structure(pos, sp, cell, name="tri40")


STRUCTS = {
    "water64": lambda: water_box(64, seed=0),
    "water16_tiny": lambda: water_box(16, seed=1),
    "fcc3_tiny": lambda: fcc_box(3, seed=2),
    "triclinic40": _triclinic,
}


def _set(i, j, s):
    return set(zip(i.tolist(), j.tolist(), map(tuple, s.tolist())))


@pytest.mark.parametrize("name", list(STRUCTS))
def test_neighbor_sets_bit_exact(name):
    s = STRUCTS[name]()
    spec = make_model(T=3)
    pot = potential(spec)
    sy = pot.system(s.pos, s.species, s.cell, skin=1.0)
    gi, gj, gs = sy.neighbors()
    oi, oj, osh = oracle.neighbors(s.pos, s.cell, spec.r_c + 1.0)
    assert len(gi) == len(oi)
    assert _set(gi, gj, gs) == _set(oi, oj, osh)
    sy.close()


@pytest.mark.parametrize("name", list(STRUCTS))
def test_layers_match_oracle(name):
    s = STRUCTS[name]()
    spec = make_model(T=3)
    g = gpu_eval(spec, s)
    ref = oracle.energy_forces(spec, s.pos, s.species, s.cell, want_layers=True)
    for t in range(spec.T):
        rho, coef = g["system"].layer(t)
        rho = rho.double().cpu().numpy()
        coef = coef.double().cpu().numpy()
        scale = np.abs(ref["rho"][t]).max() + 1e-30
        np.testing.assert_allclose(rho, ref["rho"][t], rtol=2e-4, atol=2e-6 * scale)
        np.testing.assert_allclose(coef, ref["coef"][t], rtol=2e-4, atol=2e-6)
    g["system"].close()


@pytest.mark.parametrize("T", [1, 3, 5])
@pytest.mark.parametrize("name", list(STRUCTS))
def test_energy_forces_match_oracle(name, T):
    s = STRUCTS[name]()
    spec = make_model(T=T)
    g = gpu_eval(spec, s)
    ref = oracle.energy_forces(spec, s.pos, s.species, s.cell)
    assert_parity(g, ref, s.n_atoms)
    g["system"].close()


def test_cu4000_box():
    s = fcc_box(10, seed=0)
    spec = make_model(T=3)
    g = gpu_eval(spec, s)
    ref = oracle.energy_forces(spec, s.pos, s.species, s.cell)
    assert_parity(g, ref, s.n_atoms)
    g["system"].close()


def test_moved_atoms_within_skin():
    """Positions moved (< skin/2) after the build still give the oracle's E, F."""
    s = water_box(64, seed=4)
    spec = make_model(T=3)
    rng = np.random.default_rng(0)
    moved = s.pos + rng.uniform(-0.2, 0.2, size=s.pos.shape)
    g = gpu_eval(spec, s, skin=1.0, pos=moved)
    ref = oracle.energy_forces(spec, moved, s.species, s.cell)
    assert_parity(g, ref, s.n_atoms)
    g["system"].close()


def test_isolated_atom_and_ragged_species():
    # one isolated Cu atom + an odd mix of H/O: element groups of ragged sizes
    rng = np.random.default_rng(5)
    grid = np.stack(np.meshgrid(*[np.arange(5)] * 3, indexing="ij"), -1).reshape(-1, 3)[:67]
    pos = grid * 2.4 + rng.normal(0, 0.1, size=(67, 3))
    pos = np.vstack([pos, [[40.0, 40.0, 40.0]]])
    sp = np.array([0] * 45 + [1] * 22 + [2], np.int32)
    s = Structure(pos, sp, np.eye(3) * 60.0)
    spec = make_model(T=3)
    g = gpu_eval(spec, s)
    ref = oracle.energy_forces(spec, s.pos, s.species, s.cell)
    assert_parity(g, ref, s.n_atoms)
    assert g["atom_energy"][-1] == 0.0 and np.all(g["forces"][-1] == 0.0)
    g["system"].close()


def test_bitwise_deterministic():
    s = water_box(64, seed=0)
    spec = make_model(T=3)
    a = gpu_eval(spec, s)
    b = gpu_eval(spec, s)
    assert a["energy"] == b["energy"]
    assert np.array_equal(a["forces"], b["forces"])
    a["system"].close()
    b["system"].close()


def test_config1_water_24576_full_parity():
    """8192-molecule water box (24,576 atoms), T = 3: every atom against the oracle."""
    s = water_box(8192, seed=0)
    spec = make_model(T=3)
    g = gpu_eval(spec, s)
    ref = oracle.energy_forces(spec, s.pos, s.species, s.cell)
    de, df = assert_parity(g, ref, s.n_atoms)
    g["system"].close()


def _keys(i, j, sh, n):
    """(i, j, image shift) triples as sorted int64 keys (shifts within +-8)."""
    assert np.abs(sh).max() <= 8
    k = (i.astype(np.int64) * n + j.astype(np.int64)) * 17
    k = ((k + sh[:, 0] + 8) * 17 + sh[:, 1] + 8) * 17 + sh[:, 2] + 8
    return np.sort(k)


@pytest.mark.parametrize("name", ["water24576", "cu4000"])
def test_neighbor_sets_bit_exact_full_size(name):
    """The r_c + skin list at the bench's size (24,576-atom water box) and on the
    4,000-atom Cu crystal equals the oracle's brute-force list as a set, including
    the r_c .. r_c + skin shell that the FP32 pre-test with its margin decides;
    then again after a device rebuild at displaced positions."""
    import torch

    s = water_box(8192, seed=0) if name == "water24576" else fcc_box(10, seed=0)
    spec = make_model(T=3)
    pot = potential(spec)
    sy = pot.system(s.pos, s.species, s.cell, skin=1.0)
    for step in range(2):
        pos = s.pos if step == 0 else s.pos + np.random.default_rng(5).normal(0, 0.2, s.pos.shape)
        if step == 1:
            p = torch.as_tensor(pos, device="cuda").contiguous()
            sy.rebuild(p)
            sy.check()
        gi, gj, gs = sy.neighbors()
        oi, oj, osh = oracle.neighbors(pos, s.cell, spec.r_c + 1.0)
        d_skin = np.linalg.norm(pos[oj] + osh @ s.cell - pos[oi], axis=1)
        n_shell = int((d_skin >= spec.r_c).sum())
        print(f"[nbr] {name} step {step}: {len(oi)} entries, {n_shell} in the r_c .. r_c + skin shell")
        assert n_shell > 0
        assert len(gi) == len(oi)
        assert np.array_equal(_keys(gi, gj, gs, s.n_atoms), _keys(oi, oj, osh, s.n_atoms))
    sy.close()
