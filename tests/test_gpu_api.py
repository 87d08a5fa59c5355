"""GPU tests of the C ABI beyond plain parity: device-side rebuild, the host-buffer
entry point, the per-region profile, and the error paths (all through ctypes)."""

from __future__ import annotations

import numpy as np
import pytest

import oracle
from synth import fcc_box, make_model, water_box
from synth.structures import Structure

from gpu_helpers import assert_parity, potential

pytestmark = pytest.mark.gpu


def _set(i, j, s):
    return set(zip(i.tolist(), j.tolist(), map(tuple, s.tolist())))


def test_device_rebuild_matches_oracle_after_motion():
    import torch

    s = water_box(64, seed=3)
    spec = make_model(T=3)
    pot = potential(spec)
    sy = pot.system(s.pos, s.species, s.cell, skin=1.0)
    rng = np.random.default_rng(1)
    moved = s.pos + rng.normal(0, 0.3, size=s.pos.shape)  # beyond skin/2: neighbours change
    p1 = torch.as_tensor(moved, device="cuda").contiguous()
    sy.rebuild(p1)
    sy.check()
    gi, gj, gs = sy.neighbors()
    oi, oj, osh = oracle.neighbors(moved, s.cell, spec.r_c + 1.0)
    assert _set(gi, gj, gs) == _set(oi, oj, osh)
    sy.evaluate(p1)
    sy.check()
    torch.cuda.synchronize()
    ref = oracle.energy_forces(spec, moved, s.species, s.cell)
    assert_parity({"energy": sy.energy.item(), "forces": sy.forces.double().cpu().numpy(),
                   "atom_energy": sy.atom_energy.double().cpu().numpy()}, ref, s.n_atoms)
    sy.close()


@pytest.mark.parametrize("shift,rebuild", [(0.1, 0), (0.8, 0), (0.1, 1)])
def test_host_entry_point(shift, rebuild):
    """Host buffers in/out; a motion beyond skin/2 triggers the rebuild on its own."""
    s = fcc_box(4, seed=5)
    spec = make_model(T=3)
    pot = potential(spec)
    sy = pot.system(s.pos, s.species, s.cell, skin=1.0)
    rng = np.random.default_rng(2)
    moved = np.ascontiguousarray(s.pos + rng.uniform(-shift, shift, size=s.pos.shape))
    e = np.zeros(1, np.float64)
    f = np.zeros((s.n_atoms, 3), np.float32)
    sy.evaluate_host(moved, e, f, rebuild=bool(rebuild))
    ref = oracle.energy_forces(spec, moved, s.species, s.cell)
    assert_parity({"energy": float(e[0]), "forces": f.astype(np.float64)}, {k: ref[k] for k in ("energy", "forces")},
                  s.n_atoms)
    sy.close()


def test_profile_regions_cover_the_step():
    import torch

    from paper_2505_06711_gb300 import binding

    s = water_box(64, seed=0)
    spec = make_model(T=3)
    pot = potential(spec)
    sy = pot.system(s.pos, s.species, s.cell)
    binding.reann_ctx_profile(pot.ctx, True)
    sy.rebuild()
    sy.evaluate()
    prof = binding.reann_ctx_profile_read(pot.ctx)
    binding.reann_ctx_profile(pot.ctx, False)
    assert prof["density_fwd"][1] == 3 and prof["density_adj"][1] == 3
    assert prof["mlp_fwd"][1] == 3 and prof["mlp_bwd"][1] == 3
    assert prof["nlist_rebuild"][1] == 1
    assert all(v[0] >= 0 for v in prof.values())
    torch.cuda.synchronize()
    sy.close()


def _expect(code, fn):
    from paper_2505_06711_gb300 import ReannError

    with pytest.raises(ReannError) as e:
        fn()
    assert e.value.code == code, e.value


def test_error_paths():
    import torch

    from paper_2505_06711_gb300 import binding

    spec = make_model(T=3)
    pot = potential(spec)
    s = water_box(16, seed=0)
    bad = s.pos.copy()
    bad[5, 1] = np.nan
    _expect(binding.REANN_E_GEOM, lambda: pot.system(bad, s.species, s.cell))
    sp = s.species.copy()
    sp[3] = 7
    _expect(binding.REANN_E_ARG, lambda: pot.system(s.pos, sp, s.cell))
    coinc = s.pos.copy()
    coinc[1] = coinc[0]
    _expect(binding.REANN_E_GEOM, lambda: pot.system(coinc, s.species, s.cell))
    _expect(binding.REANN_E_GEOM, lambda: pot.system(s.pos, s.species, np.zeros((3, 3))))
    # r_c and T must match the model
    p = torch.as_tensor(s.pos, device="cuda").contiguous()
    spc = torch.as_tensor(s.species, device="cuda").contiguous()
    _expect(binding.REANN_E_MISMATCH, lambda: binding.reann_build_nlist(pot.ctx, p, spc, s.cell, 4.0, 1.0))
    sy = pot.system(s.pos, s.species, s.cell)
    _expect(binding.REANN_E_MISMATCH,
            lambda: binding.reann_energy_forces(pot.ctx, sy.nl, p, 2, sy.energy, sy.forces, None))
    # coincident atoms appearing after the build are reported by the check
    q = s.pos.copy()
    q[1] = q[0]
    sy.evaluate(torch.as_tensor(q, device="cuda").contiguous())
    _expect(binding.REANN_E_GEOM, sy.check)
    # the context stays usable afterwards
    sy.evaluate()
    sy.check()
    sy.close()


def test_empty_and_oversized_inputs_are_refused_on_the_host():
    """N = 0 and N > 2^28 atoms: the build refuses them before any device work
    (REANN_E_ARG) and the context stays usable; an energy sum over no atoms is 0."""
    import ctypes

    import torch

    from paper_2505_06711_gb300 import binding

    spec = make_model(T=3)
    pot = potential(spec)
    s = water_box(16, seed=0)
    empty_pos = torch.zeros((0, 3), dtype=torch.float64, device="cuda")
    empty_sp = torch.zeros((0,), dtype=torch.int32, device="cuda")
    _expect(binding.REANN_E_ARG,
            lambda: binding.reann_build_nlist(pot.ctx, empty_pos, empty_sp, s.cell, spec.r_c, 1.0))
    # a count beyond the documented limit, with valid small buffers: rejected by the host check
    p = torch.as_tensor(s.pos, device="cuda").contiguous()
    spc = torch.as_tensor(s.species, device="cuda").contiguous()
    c = np.ascontiguousarray(s.cell, dtype=np.float64).reshape(9)
    out = ctypes.c_void_p()
    rc = binding.lib().reann_build_nlist(pot.ctx, (1 << 28) + 1, p.data_ptr(), spc.data_ptr(),
                                         c.ctypes.data, float(spec.r_c), 1.0, ctypes.byref(out))
    assert rc == binding.REANN_E_ARG and not out.value
    # an energy sum over no atoms
    e = torch.full((1,), 7.0, dtype=torch.float64, device="cuda")
    assert binding.reann_energy_sum_noalloc(empty_pos.new_zeros((0,), dtype=torch.float32), 0, e) == binding.REANN_OK
    torch.cuda.synchronize()
    assert float(e.item()) == 0.0
    # the context still evaluates a structure correctly
    sy = pot.system(s.pos, s.species, s.cell, skin=1.0)
    sy.evaluate()
    sy.check()
    torch.cuda.synchronize()
    ref = oracle.energy_forces(spec, s.pos, s.species, s.cell)
    assert_parity({"energy": float(sy.energy.item()), "forces": sy.forces.double().cpu().numpy()},
                  ref, s.n_atoms)
    sy.close()


def test_model_file_evaluates_like_created_model(tmp_path):
    """A model written to a file and loaded with reann_model_load evaluates bit for bit
    like the same parameters given to reann_model_create."""
    import torch

    from paper_2505_06711_gb300 import binding
    from synth import write_model_file

    spec = make_model(T=3)
    s = water_box(64, seed=11)
    path = tmp_path / "water.reann"
    write_model_file(spec, path)
    model = binding.reann_model_load(path)
    ctx = binding.reann_ctx_create(model)
    binding.reann_model_free(model)
    pos = torch.as_tensor(s.pos, device="cuda").contiguous()
    species = torch.as_tensor(s.species, dtype=torch.int32, device="cuda").contiguous()
    nl = binding.reann_build_nlist(ctx, pos, species, s.cell, spec.r_c, 1.0)
    energy = torch.zeros(1, dtype=torch.float64, device="cuda")
    forces = torch.zeros((s.n_atoms, 3), dtype=torch.float32, device="cuda")
    binding.reann_energy_forces(ctx, nl, pos, spec.T, energy, forces, None)
    binding.reann_ctx_check(ctx)
    torch.cuda.synchronize()
    e_file, f_file = float(energy.item()), forces.cpu().numpy().copy()
    binding.reann_nlist_free(nl)
    binding.reann_ctx_free(ctx)
    sy = potential(spec).system(s.pos, s.species, s.cell, skin=1.0)
    sy.evaluate()
    sy.check()
    torch.cuda.synchronize()
    assert e_file == float(sy.energy.item())
    assert np.array_equal(f_file, sy.forces.cpu().numpy())
    sy.close()


def test_bounded_wait_runs_out_and_context_recovers():
    """Failure detection without a fault: a tensor-core CTA waits on an mbarrier that
    nothing arrives on (no copy or MMA in flight), gives up after a few thousand polls,
    drains and frees its tensor memory; reann_ctx_check reports REANN_E_TIMEOUT once,
    and the same context then evaluates exactly as before."""
    import torch

    from paper_2505_06711_gb300 import Potential, ReannError, binding

    spec = make_model(T=3)
    s = water_box(64, seed=5)
    pot = Potential(spec, precision=binding.REANN_MLP_BF16)
    sy = pot.system(s.pos, s.species, s.cell, skin=1.0)
    sy.evaluate()
    sy.check()
    torch.cuda.synchronize()
    e0, f0 = float(sy.energy.item()), sy.forces.cpu().numpy().copy()
    binding.reann_ctx_wait_selftest(pot.ctx, 4096)
    with pytest.raises(ReannError) as err:
        sy.check()
    assert err.value.code == binding.REANN_E_TIMEOUT
    assert "suspect" not in str(err.value)  # the drain after the timeout completed
    sy.check()  # the flag was cleared by the previous check
    with pytest.raises(ReannError):
        binding.reann_ctx_wait_selftest(pot.ctx, 0)
    sy.forces.zero_()
    sy.evaluate()
    sy.check()
    torch.cuda.synchronize()
    assert float(sy.energy.item()) == e0
    assert np.array_equal(sy.forces.cpu().numpy(), f0)
    sy.close()
    pot.close()


def test_rebuilds_across_the_resort_period_match_oracle():
    """Device rebuilds keep the internal atom order between full sorts (every 8th
    rebuild sorts again); the list and the forces must not depend on which kind a
    rebuild was.  Ten rebuilds of a drifting box: sets equal the oracle's after each,
    forces within the FP32 bar after the last keep-order and the sort rebuild."""
    import torch

    s = water_box(256, seed=21)
    spec = make_model(T=3)
    pot = potential(spec)
    sy = pot.system(s.pos, s.species, s.cell, skin=1.0)
    rng = np.random.default_rng(22)
    pos = s.pos.copy()
    for k in range(1, 11):
        pos = pos + rng.normal(0, 0.08, pos.shape)  # drifts well beyond the skin over the ten steps
        p = torch.as_tensor(pos, device="cuda").contiguous()
        sy.rebuild(p)
        sy.check()
        gi, gj, gs = sy.neighbors()
        oi, oj, osh = oracle.neighbors(pos, s.cell, spec.r_c + 1.0)
        assert _set(gi, gj, gs) == _set(oi, oj, osh), k
        if k in (7, 8, 9):  # keep-order, sort, keep-order
            sy.evaluate(p)
            sy.check()
            torch.cuda.synchronize()
            ref = oracle.energy_forces(spec, pos, s.species, s.cell)
            assert_parity({"energy": float(sy.energy.item()), "forces": sy.forces.double().cpu().numpy()},
                          {"energy": ref["energy"], "forces": ref["forces"]}, s.n_atoms)
    sy.close()
