"""The hand-written adjoint exposed as a torch.autograd.Function.

* torch.autograd.grad of E(pos) equals -F from the library's reverse pass;
* central finite differences of the GPU energy (FP64 sum of FP32 atomic
  energies) on a seeded 192-atom subset of the 24,576-atom water box agree
  with those forces, and both agree with the FP64 oracle's gradient.
"""

from __future__ import annotations

import numpy as np
import pytest

import oracle
from synth import make_model, water_box

from gpu_helpers import potential

pytestmark = pytest.mark.gpu


def test_autograd_gradient_is_minus_forces():
    import torch

    from paper_2505_06711_gb300 import energy

    s = water_box(64, seed=3)
    spec = make_model(T=3)
    sy = potential(spec).system(s.pos, s.species, s.cell)
    pos = sy.pos.clone().requires_grad_(True)
    e = energy(pos, sy)
    loss = 2.0 * e + (pos**2).sum()
    (g,) = torch.autograd.grad(loss, pos)
    sy.evaluate(pos.detach().contiguous())
    torch.cuda.synchronize()
    expect = -2.0 * sy.forces.double() + 2.0 * pos.detach()
    assert torch.equal(g, expect)
    assert e.item() == sy.energy.item()
    sy.close()


def test_forces_match_finite_differences_on_192_atoms_of_the_24576_atom_box():
    import torch

    from paper_2505_06711_gb300 import energy

    s = water_box(8192, seed=0)
    spec = make_model(T=3)
    sy = potential(spec).system(s.pos, s.species, s.cell, skin=1.0)
    pos = sy.pos.clone().requires_grad_(True)
    (g,) = torch.autograd.grad(energy(pos, sy), pos)
    forces = -g.cpu().numpy()
    rng = np.random.default_rng(192)
    subset = rng.choice(s.n_atoms, size=192, replace=False)
    h = 5e-3
    fd = np.zeros((192, 3))
    p = sy.pos.clone()
    for a_i, a in enumerate(subset):
        for k in range(3):
            p[a, k] += h
            sy.evaluate(p, atom_energy=False)
            ep = sy.energy.item()
            p[a, k] -= 2 * h
            sy.evaluate(p, atom_energy=False)
            em = sy.energy.item()
            p[a, k] += h
            fd[a_i, k] = -(ep - em) / (2 * h)
    err = np.abs(fd - forces[subset])
    print(f"[fd] max|F_fd - F| = {err.max():.3e} eV/A over {len(subset)} atoms, max|F| = {np.abs(forces[subset]).max():.3f}")
    assert err.max() < 2e-3
    ref = oracle.energy_forces(spec, s.pos, s.species, s.cell)
    assert np.abs(ref["forces"][subset] - forces[subset]).max() < 1e-4
    sy.close()
