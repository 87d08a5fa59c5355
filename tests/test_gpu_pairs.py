"""Orbital-pair-product features: the (L+1) N (N+1)/2 features that Sec. 2.1
counts (reading 1), rho_{l,(k,k')} = sum_{a in l} w_a g_{a,k} g_{a,k'} over 8
orbitals (108 features), against the FP64 oracle, whose pair features are
pinned by the bilinear multinomial identity and force central differences."""

from __future__ import annotations

import numpy as np
import pytest

import oracle
from gpu_helpers import assert_parity, gpu_eval
from synth import fcc_box, make_model, water_box

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize(
    "name,make,T",
    [
        ("water192", lambda: water_box(64, seed=0), 3),
        ("water24576", lambda: water_box(8192, seed=0), 3),
        ("cu4000", lambda: fcc_box(10, seed=0), 3),
        ("cu4000", lambda: fcc_box(10, seed=0), 5),
    ],
)
def test_pair_features_parity(name, make, T):
    spec = make_model(T=T, pairs=True)
    s = make()
    ref = oracle.energy_forces(spec, s.pos, s.species, s.cell)
    gpu = gpu_eval(spec, s)
    assert_parity(gpu, ref, s.n_atoms)
    gpu["system"].close()


def test_pair_feature_layers_match_oracle():
    import torch

    spec = make_model(T=3, pairs=True)
    s = water_box(64, seed=0)
    ref = oracle.energy_forces(spec, s.pos, s.species, s.cell, want_layers=True)
    gpu = gpu_eval(spec, s)
    sy = gpu["system"]
    for t in range(spec.T):
        rho, coef = sy.layer(t)
        torch.cuda.synchronize()
        r = rho.double().cpu().numpy()
        assert r.shape == (s.n_atoms, 108)
        scale = np.abs(ref["rho"][t]).max()
        assert np.abs(r - ref["rho"][t]).max() <= 2e-6 * scale, t
        np.testing.assert_allclose(coef.double().cpu().numpy(), ref["coef"][t], rtol=0, atol=2e-6)
    sy.close()


def test_pair_features_decomposed_virial_and_precision_guard():
    import torch

    from paper_2505_06711_gb300 import Potential, binding

    spec = make_model(T=3, pairs=True)
    s = water_box(512, seed=1)
    pot = Potential(spec)
    try:
        out = []
        for ranks in (None, (2, 2, 1)):
            sy = pot.system(s.pos, s.species, s.cell, ranks=ranks)
            sy.evaluate(virial=True)
            sy.check()
            torch.cuda.synchronize()
            out.append((sy.forces.cpu().numpy(), sy.virial.cpu().numpy()))
            sy.close()
        assert np.array_equal(out[0][0], out[1][0])
        ref = oracle.energy_forces(spec, s.pos, s.species, s.cell)
        assert np.abs(out[0][1] - ref["virial"]).max() / s.n_atoms <= 2e-5
        with pytest.raises(binding.ReannError):
            pot.set_precision(binding.REANN_MLP_BF16)  # tensor-core networks: 48 features only
    finally:
        pot.close()
