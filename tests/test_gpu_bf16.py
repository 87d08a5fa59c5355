"""Tensor-core (tcgen05, BF16 operands, FP32 accumulation) atomic networks.

Mixed-precision bar: energy within 1 meV/atom and forces within 20 meV/A RMS of
the FP64 oracle; the density and reverse-pass edge arithmetic stays FP32.

* BF16X3 (every operand a BF16 hi + lo pair, three MMAs per K step) meets the
  bar on every structure, crystals included.
* Plain BF16 meets it on water; on the near-perfect Cu crystal every atom feeds
  the networks almost the same inputs, so BF16 rounding shifts all atomic
  energies alike and the energy error exceeds 1 meV/atom.  The test records
  that error and guards it at about twice the measured value.
"""

from __future__ import annotations

import numpy as np
import pytest

import oracle
from synth import fcc_box, make_model, water_box

pytestmark = pytest.mark.gpu

E_TOL_BF16 = 1e-3  # eV/atom
F_RMS_TOL_BF16 = 20e-3  # eV/A
# plain BF16 on the Cu crystal (see module docstring): regression guards at about
# twice the errors measured on GB300 (3.6 meV/atom at T = 3, 18 meV/atom and
# 0.12 eV/A RMS at T = 5) -- these exceed the mixed-precision bar
E_TOL_BF16_CRYSTAL = {"cu4000-T3": 8e-3, "cu4000-T5": 4e-2}
F_RMS_TOL_BF16_CRYSTAL = {"cu4000-T3": 20e-3, "cu4000-T5": 0.25}

CASES = {
    "water192-T3": (lambda: water_box(64, seed=0), 3),
    "water24576-T3": (lambda: water_box(8192, seed=0), 3),
    "cu4000-T3": (lambda: fcc_box(10, seed=0), 3),
    "cu4000-T5": (lambda: fcc_box(10, seed=0), 5),
}


def _eval(spec, s, precision):
    import torch

    from paper_2505_06711_gb300 import Potential

    pot = Potential(spec, precision=precision)
    sy = pot.system(s.pos, s.species, s.cell)
    sy.evaluate()
    sy.check()
    torch.cuda.synchronize()
    out = (float(sy.energy.item()), sy.forces.double().cpu().numpy())
    sy.close()
    pot.close()
    return out


def _errors(name, precision):
    make, T = CASES[name]
    s = make()
    spec = make_model(T=T)
    e, f = _eval(spec, s, precision)
    ref = oracle.energy_forces(spec, s.pos, s.species, s.cell)
    de = abs(e - ref["energy"]) / s.n_atoms
    frms = float(np.sqrt(((f - ref["forces"]) ** 2).mean()))
    print(f"[tc p={precision}] {name} |dE|/N={de:.3e} dF_rms={frms:.3e}")
    return de, frms


@pytest.mark.parametrize("name", list(CASES))
def test_bf16x3_within_mixed_precision_bound(name):
    from paper_2505_06711_gb300 import binding

    de, frms = _errors(name, binding.REANN_MLP_BF16X3)
    assert de <= E_TOL_BF16
    assert frms <= F_RMS_TOL_BF16


@pytest.mark.parametrize("name", list(CASES))
def test_plain_bf16_error(name):
    from paper_2505_06711_gb300 import binding

    de, frms = _errors(name, binding.REANN_MLP_BF16)
    assert de <= E_TOL_BF16_CRYSTAL.get(name, E_TOL_BF16)
    assert frms <= F_RMS_TOL_BF16_CRYSTAL.get(name, F_RMS_TOL_BF16)


def test_tensor_core_and_fp32_paths_agree_on_layer0():
    """Layer-0 features involve no network: every precision gives the same rho^0."""
    from paper_2505_06711_gb300 import Potential, binding

    s = water_box(64, seed=2)
    spec = make_model(T=3)
    pots = [Potential(spec, precision=p) for p in (binding.REANN_MLP_FP32, binding.REANN_MLP_BF16,
                                                    binding.REANN_MLP_BF16X3)]
    rhos = []
    for p in pots:
        sy = p.system(s.pos, s.species, s.cell)
        sy.evaluate()
        rhos.append(sy.layer(0)[0].cpu().numpy())
        sy.close()
        p.close()
    assert np.array_equal(rhos[0], rhos[1]) and np.array_equal(rhos[0], rhos[2])
