"""Tensor-core (tcgen05, BF16 operands, FP32 accumulation) atomic networks.

Mixed-precision bar of the workload configuration: energy within 1 meV/atom and
forces within 20 meV/A RMS of the FP64 oracle; the density and reverse-pass
edge arithmetic stays FP32.  Each 128-row tile rounds only the deviations of
its activations from their column mean (the mean's product is added back in
FP32, an exact identity), so plain BF16 meets the bar on crystals too, where
every atom feeds the networks nearly the same input.  BF16X3 (every operand a
BF16 hi + lo pair) on anchored activations also meets the FP32 path's bar.
"""

from __future__ import annotations

import numpy as np
import pytest

import oracle
from synth import fcc_box, hea_box, make_model, water_box

from gpu_helpers import E_TOL_PER_ATOM, F_TOL_MAX

pytestmark = pytest.mark.gpu

E_TOL_BF16 = 1e-3  # eV/atom
F_RMS_TOL_BF16 = 20e-3  # eV/A

CASES = {
    "water192-T3": (lambda: water_box(64, seed=0), 3, 3),
    "water24576-T3": (lambda: water_box(8192, seed=0), 3, 3),
    "cu4000-T3": (lambda: fcc_box(10, seed=0), 3, 3),
    "cu4000-T5": (lambda: fcc_box(10, seed=0), 5, 3),
    "hea4000-T3": (lambda: hea_box(10, seed=0), 3, 8),
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
    make, T, n_elem = CASES[name]
    s = make()
    spec = make_model(T=T, n_elem=n_elem)
    e, f = _eval(spec, s, precision)
    ref = oracle.energy_forces(spec, s.pos, s.species, s.cell)
    de = abs(e - ref["energy"]) / s.n_atoms
    frms = float(np.sqrt(((f - ref["forces"]) ** 2).mean()))
    fmax = float(np.abs(f - ref["forces"]).max())
    print(f"[tc p={precision}] {name} |dE|/N={de:.3e} dF_rms={frms:.3e} dF_max={fmax:.3e}")
    return de, frms, fmax


@pytest.mark.parametrize("name", list(CASES))
def test_plain_bf16_within_mixed_precision_bound(name):
    from paper_2505_06711_gb300 import binding

    de, frms, _ = _errors(name, binding.REANN_MLP_BF16)
    assert de <= E_TOL_BF16
    assert frms <= F_RMS_TOL_BF16


@pytest.mark.parametrize("name", list(CASES))
def test_bf16x3_within_fp32_bar(name):
    from paper_2505_06711_gb300 import binding

    de, frms, fmax = _errors(name, binding.REANN_MLP_BF16X3)
    assert de <= E_TOL_PER_ATOM
    assert fmax <= F_TOL_MAX


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
