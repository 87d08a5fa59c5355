"""Virtual-rank spatial decomposition (Sec. 2.2, Figs. 3-5) against the undivided list.

The paper's scheme exchanges the ghost atoms' coefficients before every
message-passing layer (and their gradients in the reverse pass), so a
subdomain needs a halo of r_c (+ skin) whatever T is, and the result equals
the undivided model's.  Here the rows keep the single-domain entry order and
ghost slots hold exact copies, so with FP32 networks forces must agree bit for
bit and energies to the order of the FP64 sum.  The tensor-core networks round
each 128-row tile's deviations from its own column mean, and a rank-major
layout groups the atoms into other tiles, so there the two lists agree within
the precision's own bar (BF16: the mixed-precision bound; BF16X3: the FP32
bar).
"""

from __future__ import annotations

import numpy as np
import pytest

import oracle
from gpu_helpers import assert_parity
from synth import fcc_box, make_model, water_box

pytestmark = pytest.mark.gpu

STRUCTS = {
    "water192": lambda: water_box(64, seed=0),
    "water24576": lambda: water_box(8192, seed=0),
    "cu4000": lambda: fcc_box(10, seed=0),
}


def _eval(pot, s, ranks=None):
    import torch

    sy = pot.system(s.pos, s.species, s.cell, skin=1.0, ranks=ranks)
    sy.evaluate()
    sy.check()
    torch.cuda.synchronize()
    out = (float(sy.energy.item()), sy.forces.cpu().numpy(), sy.atom_energy.cpu().numpy(), sy.ranks())
    sy.close()
    return out


@pytest.mark.parametrize(
    "name,ranks,T,precision",
    [
        ("water192", (2, 2, 2), 3, 0),
        ("water24576", (2, 2, 2), 3, 0),
        ("water24576", (4, 1, 1), 3, 1),
        ("cu4000", (2, 2, 1), 3, 0),
        ("cu4000", (3, 1, 1), 5, 0),
        ("cu4000", (2, 1, 2), 3, 2),
    ],
)
def test_decomposed_equals_single_domain(name, ranks, T, precision):
    from paper_2505_06711_gb300 import Potential

    s = STRUCTS[name]()
    pot = Potential(make_model(T=T), precision=precision)
    try:
        e1, f1, a1, info1 = _eval(pot, s)
        ek, fk, ak, infok = _eval(pot, s, ranks)
    finally:
        pot.close()
    k = int(np.prod(ranks))
    print(f"[decomp] {name} ranks={ranks} T={T} local={infok['local'].tolist()} "
          f"ghosts={infok['ghosts'].tolist()} remote={infok['remote'].tolist()} dE={ek - e1:.3e}")
    assert len(infok["local"]) == k and int(infok["local"].sum()) == s.n_atoms
    assert (infok["remote"] > 0).all()  # every rank receives ghosts from another rank
    if precision == 0:
        assert np.array_equal(fk, f1), f"max|dF| = {np.abs(fk - f1).max():.3e}"
        assert np.array_equal(ak, a1)
        assert abs(ek - e1) <= 1e-12 * abs(e1)
    elif precision == 1:  # BF16: within the mixed-precision bound of each other
        assert abs(ek - e1) / s.n_atoms <= 1e-3
        assert float(np.sqrt(np.mean((fk - f1) ** 2))) <= 20e-3
    else:  # BF16X3: within the FP32 bar of each other
        assert abs(ek - e1) / s.n_atoms <= 1e-6
        assert float(np.abs(fk - f1).max()) <= 1e-4


def test_halo_does_not_grow_with_T():
    from paper_2505_06711_gb300 import Potential

    s = STRUCTS["water24576"]()
    ghosts = {}
    for T in (1, 3, 5):
        pot = Potential(make_model(T=T))
        try:
            sy = pot.system(s.pos, s.species, s.cell, skin=1.0, ranks=(2, 2, 2))
            ghosts[T] = sy.ranks()["ghosts"].tolist()
            sy.close()
        finally:
            pot.close()
    assert ghosts[1] == ghosts[3] == ghosts[5]


def test_one_rank_is_the_single_domain_list():
    import torch

    from paper_2505_06711_gb300 import Potential

    s = STRUCTS["cu4000"]()
    pot = Potential(make_model(T=3))
    try:
        a = pot.system(s.pos, s.species, s.cell, skin=1.0)
        b = pot.system(s.pos, s.species, s.cell, skin=1.0, ranks=(1, 1, 1))
        ia, ib = a.info(), b.info()
        rb = b.ranks()
        # one rank: no exchange between ranks; its ghost slots are the periodic images
        # some atom actually lists (the undivided list also keeps images that lie in
        # the cell's halo but within r_c + skin of no atom)
        assert rb["remote"].tolist() == [0] and 0 < rb["ghosts"][0] <= ia[1]
        assert ia[0] == ib[0] and ia[2] == ib[2]
        ea = {tuple(r) for r in np.column_stack(a.neighbors()).tolist()}
        eb = {tuple(r) for r in np.column_stack(b.neighbors()).tolist()}
        assert ea == eb
        torch.cuda.synchronize()
        a.close()
        b.close()
    finally:
        pot.close()


def test_decomposed_neighbour_sets_and_oracle():
    import torch

    from paper_2505_06711_gb300 import Potential

    s = STRUCTS["water192"]()
    spec = make_model(T=3)
    pot = Potential(spec)
    try:
        sy = pot.system(s.pos, s.species, s.cell, skin=1.0, ranks=(2, 2, 2))
        i, j, n = sy.neighbors()
        got = {(int(a), int(b), *map(int, c)) for a, b, c in zip(i, j, n)}
        ref_i, ref_j, ref_n = oracle.neighbors(s.pos, s.cell, spec.r_c + 1.0)
        want = {(int(a), int(b), *map(int, c)) for a, b, c in zip(ref_i, ref_j, ref_n)}
        assert got == want
        sy.evaluate()
        sy.check()
        torch.cuda.synchronize()
        ref = oracle.energy_forces(spec, s.pos, s.species, s.cell)
        assert_parity({"energy": float(sy.energy.item()), "forces": sy.forces.double().cpu().numpy()},
                      {"energy": ref["energy"], "forces": ref["forces"]}, s.n_atoms)
        sy.close()
    finally:
        pot.close()


def test_decomposed_list_refuses_in_place_rebuild():
    import torch

    from paper_2505_06711_gb300 import Potential, binding

    s = STRUCTS["water192"]()
    pot = Potential(make_model(T=3))
    try:
        sy = pot.system(s.pos, s.species, s.cell, skin=1.0, ranks=(2, 1, 1))
        with pytest.raises(binding.ReannError):
            sy.rebuild()
        vel = torch.zeros_like(sy.pos)
        mass = torch.ones(s.n_atoms, dtype=torch.float64, device="cuda")
        with pytest.raises(binding.ReannError):
            sy.md(vel, mass, 0.5, 1)
        e = np.zeros(1)
        f = np.zeros((s.n_atoms, 3), np.float32)
        with pytest.raises(binding.ReannError):
            sy.evaluate_host(np.ascontiguousarray(s.pos), e, f, rebuild=True)
        sy.evaluate_host(np.ascontiguousarray(s.pos), e, f, rebuild=False)  # no motion: no rebuild needed
        sy.close()
        for bad in ((0, 1, 1), (1, 65, 1)):
            with pytest.raises(binding.ReannError):
                pot.system(s.pos, s.species, s.cell, skin=1.0, ranks=bad)
    finally:
        pot.close()
