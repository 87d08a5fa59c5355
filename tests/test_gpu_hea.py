"""Five-element high-entropy alloy (the paper's third system type, Sec. 4.1):
an fcc random solid solution of Co, Cr, Fe, Mn, Ni on an eight-element model.

Every element has its own atomic networks, so the network tiles are cut per
element (atoms are stored element-major) and a tile never mixes weights.
"""

from __future__ import annotations

import numpy as np
import pytest

import oracle
from gpu_helpers import assert_parity, gpu_eval
from synth import hea_box, make_model

pytestmark = pytest.mark.gpu

E_TOL_BF16 = 1e-3  # eV/atom, the mixed-precision bar
F_RMS_TOL_BF16 = 20e-3  # eV/A


@pytest.mark.parametrize("k,T", [(3, 3), (10, 3), (10, 5)])
def test_hea_fp32_parity(k, T):
    spec = make_model(T=T, n_elem=8)
    s = hea_box(k, seed=0)
    assert sorted(set(s.species.tolist())) == [3, 4, 5, 6, 7]
    ref = oracle.energy_forces(spec, s.pos, s.species, s.cell)
    gpu = gpu_eval(spec, s)
    assert_parity(gpu, ref, s.n_atoms)
    gpu["system"].close()


@pytest.mark.parametrize("precision", [1, 2], ids=["bf16", "bf16x3"])
def test_hea_tensor_core_networks(precision):
    import torch

    from paper_2505_06711_gb300 import Potential

    spec = make_model(T=3, n_elem=8)
    s = hea_box(10, seed=0)
    ref = oracle.energy_forces(spec, s.pos, s.species, s.cell)
    pot = Potential(spec, precision=precision)
    try:
        sy = pot.system(s.pos, s.species, s.cell)
        sy.evaluate()
        sy.check()
        torch.cuda.synchronize()
        de = abs(float(sy.energy.item()) - ref["energy"]) / s.n_atoms
        df = float(np.sqrt(((sy.forces.double().cpu().numpy() - ref["forces"]) ** 2).mean()))
        print(f"[hea] precision={precision} |dE|/N={de:.3e} rms dF={df:.3e}")
        assert de <= E_TOL_BF16 and df <= F_RMS_TOL_BF16
        sy.close()
    finally:
        pot.close()


def test_hea_decomposed_is_bitwise_single_domain():
    import torch

    from paper_2505_06711_gb300 import Potential

    spec = make_model(T=3, n_elem=8)
    s = hea_box(10, seed=1)
    pot = Potential(spec)
    try:
        out = []
        for ranks in (None, (2, 2, 2)):
            sy = pot.system(s.pos, s.species, s.cell, ranks=ranks)
            sy.evaluate()
            sy.check()
            torch.cuda.synchronize()
            out.append(sy.forces.cpu().numpy())
            sy.close()
        assert np.array_equal(out[0], out[1])
    finally:
        pot.close()
