"""Replayed rebuild and evaluation calls equal direct launches.

Repeated ``reann_nlist_rebuild`` / ``reann_energy_forces`` calls with the same
arguments run directly once, are captured into a CUDA graph on the second call
and replayed afterwards.  The graph reads the argument buffers at replay time,
so new positions written into the same buffer must give exactly the result of
direct launches (per-region profiling switches graphs off).
"""

from __future__ import annotations

import numpy as np
import pytest

import oracle
from gpu_helpers import assert_parity
from synth import make_model, water_box

pytestmark = pytest.mark.gpu


def _state(sy):
    import torch

    torch.cuda.synchronize()
    return float(sy.energy.item()), sy.forces.cpu().numpy().copy(), sy.atom_energy.cpu().numpy().copy()


def test_replay_equals_direct_launches():
    import torch

    from paper_2505_06711_gb300 import Potential, binding

    s = water_box(512, seed=3)
    spec = make_model(T=3)
    pot = Potential(spec)
    try:
        sy = pot.system(s.pos, s.species, s.cell, skin=1.0)
        rng = np.random.default_rng(11)
        base = torch.tensor(s.pos, dtype=torch.float64, device="cuda")
        runs = []
        for k in range(5):  # direct, capture, replay, replay, replay
            # new positions in the same buffer (within skin/2 of the build)
            sy.pos.copy_(base + torch.tensor(rng.uniform(-0.2, 0.2, s.pos.shape), device="cuda"))
            sy.rebuild()
            sy.evaluate()
            sy.check()
            e, f, a = _state(sy)
            # the same positions with every kernel launched directly
            binding.reann_ctx_profile(pot.ctx, True)
            sy.rebuild()
            sy.evaluate()
            binding.reann_ctx_profile(pot.ctx, False)
            e0, f0, a0 = _state(sy)
            assert e == e0 and np.array_equal(f, f0) and np.array_equal(a, a0), k
            runs.append(e)
        assert len(set(runs)) == len(runs)  # the positions really changed between calls
        # and the replayed result is the oracle's
        p = sy.pos.cpu().numpy()
        sy.rebuild()
        sy.evaluate()
        e, f, _ = _state(sy)
        ref = oracle.energy_forces(spec, p, s.species, s.cell)
        assert_parity({"energy": e, "forces": f.astype(np.float64)},
                      {"energy": ref["energy"], "forces": ref["forces"]}, s.n_atoms)
        sy.close()
    finally:
        pot.close()


def test_replay_follows_precision_and_outputs():
    import torch

    from paper_2505_06711_gb300 import Potential, binding

    s = water_box(256, seed=4)
    pot = Potential(make_model(T=3))
    try:
        sy = pot.system(s.pos, s.species, s.cell, skin=1.0)
        for _ in range(3):
            sy.evaluate()
        e32, f32, _ = _state(sy)
        pot.set_precision(binding.REANN_MLP_BF16)
        for _ in range(3):
            sy.evaluate()
        e16, f16, _ = _state(sy)
        assert e16 != e32  # a new key: the BF16 networks really ran
        pot.set_precision(binding.REANN_MLP_FP32)
        sy.evaluate()
        e, f, _ = _state(sy)
        assert e == e32 and np.array_equal(f, f32)
        # other output buffers: a new key, the results land there
        en = torch.zeros(1, dtype=torch.float64, device="cuda")
        fo = torch.zeros((s.n_atoms, 3), dtype=torch.float32, device="cuda")
        for _ in range(3):
            fo.zero_()
            binding.reann_energy_forces(pot.ctx, sy.nl, sy.pos, pot.T, en, fo, None)
            torch.cuda.synchronize()
            assert float(en.item()) == e32 and np.array_equal(fo.cpu().numpy(), f32)
        sy.close()
    finally:
        pot.close()
