"""The energy sum that allocates nothing (reann_energy_sum_noalloc).

Callers that must not allocate device memory when they need a total energy (a
force back-end inside an MD engine that owns the memory budget, or a
latency-critical callback that avoids cudaMalloc because it can synchronise
the device) sum per-atom energies they already hold with this entry point,
which uses a fixed scratch array compiled into the library.  These tests call
it through the C ABI and compare it with the energy reann_energy_forces returns
for the same atom energies (the same FP64 sum grouped differently, so within
the FP32 path's energy tolerance) and with an exact FP64 sum on the host,
twice in a row with different sizes (the scratch is shared between calls), and
check that oversized inputs are refused.

The file name makes pytest collect it last.
"""

from __future__ import annotations

import math

import pytest

from synth import make_model, water_box

from gpu_helpers import E_TOL_PER_ATOM, potential

pytestmark = pytest.mark.gpu


def _reference(spec, structure):
    import torch

    pot = potential(spec)
    sy = pot.system(structure.pos, structure.species, structure.cell)
    sy.evaluate(atom_energy=True)
    sy.check()
    torch.cuda.synchronize()
    return sy, float(sy.energy.item())


def test_noalloc_sum_matches_energy_forces_twice():
    import torch

    from paper_2505_06711_gb300 import binding

    spec = make_model(T=3)
    big, e_big = _reference(spec, water_box(4096, seed=7))  # 12,288 atoms: several scratch entries
    small, e_small = _reference(spec, water_box(64, seed=8))  # 192 atoms: one scratch entry
    out = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
    # two calls in a row on the same stream: the second reads scratch the first also used
    rc1 = binding.reann_energy_sum_noalloc(big.atom_energy, big.n, out[0:1])
    rc2 = binding.reann_energy_sum_noalloc(small.atom_energy, small.n, out[1:2])
    assert rc1 == binding.REANN_OK and rc2 == binding.REANN_OK
    torch.cuda.synchronize()
    got = out.cpu().tolist()
    assert abs(got[0] - e_big) <= E_TOL_PER_ATOM * big.n
    assert abs(got[1] - e_small) <= E_TOL_PER_ATOM * small.n
    # both are FP64 sums of the same FP32 values: only the grouping differs
    for sy, g in ((big, got[0]), (small, got[1])):
        host = math.fsum(sy.atom_energy.double().cpu().tolist())
        assert abs(g - host) <= 1e-12 * max(1.0, abs(host)) * sy.n ** 0.5
    big.close()
    small.close()


def test_noalloc_sum_refuses_oversized_input():
    import torch

    from paper_2505_06711_gb300 import binding

    limit = binding.reann_energy_sum_noalloc_max_atoms()
    assert limit == 8_388_608
    dummy = torch.zeros(1, dtype=torch.float32, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    assert binding.reann_energy_sum_noalloc(dummy, limit + 1, out) == binding.REANN_E_CAPACITY
    assert binding.reann_energy_sum_noalloc(dummy, 0, out) == binding.REANN_OK
    torch.cuda.synchronize()
    assert out.item() == 0.0
