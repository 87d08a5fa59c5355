"""Shared helpers of the GPU tests: run the CUDA path and the oracle on the same input."""

from __future__ import annotations

import numpy as np

# Tolerances of the FP32 path against the FP64 oracle
E_TOL_PER_ATOM = 1e-6  # eV/atom
F_TOL_MAX = 1e-4  # eV/A max-abs

_POTS: dict = {}


def potential(spec, key=None):
    from paper_2505_06711_gb300 import Potential

    k = key if key is not None else (spec.T, hash(spec.params.tobytes()))
    if k not in _POTS:
        _POTS[k] = Potential(spec)
    return _POTS[k]


def gpu_eval(spec, s, skin=1.0, pos=None):
    import torch

    pot = potential(spec)
    sy = pot.system(s.pos, s.species, s.cell, skin=skin)
    p = None
    if pos is not None:
        p = torch.as_tensor(np.asarray(pos, np.float64), device=pot.device).contiguous()
    sy.evaluate(p)
    sy.check()
    torch.cuda.synchronize()
    out = {
        "energy": float(sy.energy.item()),
        "forces": sy.forces.double().cpu().numpy(),
        "atom_energy": sy.atom_energy.double().cpu().numpy(),
        "system": sy,
    }
    return out


def assert_parity(gpu, ref, n, e_tol=E_TOL_PER_ATOM, f_tol=F_TOL_MAX):
    de = abs(gpu["energy"] - ref["energy"]) / n
    df = float(np.abs(gpu["forces"] - ref["forces"]).max()) if n else 0.0
    fmax = float(np.abs(ref["forces"]).max()) if n else 0.0
    print(f"[parity] N={n} |dE|/N={de:.3e} max|dF|={df:.3e} max|F|={fmax:.3e}")
    assert de <= e_tol, f"|dE|/N = {de:.3e} > {e_tol}"
    assert df <= f_tol, f"max|dF| = {df:.3e} > {f_tol}"
    if "atom_energy" in ref and "atom_energy" in gpu:
        da = float(np.abs(gpu["atom_energy"] - ref["atom_energy"]).max()) if n else 0.0
        assert da <= 10 * e_tol, f"max|d eps| = {da:.3e}"
    return de, df
