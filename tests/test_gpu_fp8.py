"""FP8 E4M3 atomic networks on tcgen05 (REANN_MLP_FP8) against the FP64 oracle.

Every network product but the output layer runs with E4M3 operands and FP32
accumulation on anchored activations: each 128-row tile subtracts its column
mean before rounding and adds the mean's product back in FP32 (an exact
identity), activations are scaled per row and weights per output unit, each by
max |.| / 448 (rounded up to a power of two for the activations).  The bar is the mixed-precision
bound of the workload configuration: energy within 1 meV/atom and forces
within 20 meV/A RMS of the oracle on every structure, crystals included.  The
kernel arithmetic itself is pinned by the emulation test below.
"""

from __future__ import annotations

import numpy as np
import pytest

import oracle
from synth import fcc_box, hea_box, make_model, water_box

pytestmark = pytest.mark.gpu

E_TOL = 1e-3  # eV/atom
F_RMS_TOL = 20e-3  # eV/A


def _eval(spec, s, precision):
    import torch

    from paper_2505_06711_gb300 import Potential

    pot = Potential(spec, precision=precision)
    try:
        sy = pot.system(s.pos, s.species, s.cell, skin=1.0)
        sy.evaluate()
        sy.check()
        torch.cuda.synchronize()
        out = float(sy.energy.item()), sy.forces.double().cpu().numpy()
        sy.close()
    finally:
        pot.close()
    return out


@pytest.mark.parametrize(
    "name,make,T,n_elem",
    [
        ("water192", lambda: water_box(64, seed=0), 3, 3),
        ("water24576", lambda: water_box(8192, seed=0), 3, 3),
        ("cu4000", lambda: fcc_box(10, seed=0), 3, 3),
        ("cu4000", lambda: fcc_box(10, seed=0), 5, 3),
        ("hea4000", lambda: hea_box(10, seed=0), 3, 8),
    ],
)
def test_fp8_networks_against_oracle(name, make, T, n_elem):
    from paper_2505_06711_gb300 import binding

    spec = make_model(T=T, n_elem=n_elem)
    s = make()
    ref = oracle.energy_forces(spec, s.pos, s.species, s.cell)
    e8, f8 = _eval(spec, s, binding.REANN_MLP_FP8)
    e32, f32 = _eval(spec, s, binding.REANN_MLP_FP32)
    n = s.n_atoms
    de8 = abs(e8 - ref["energy"]) / n
    rms8 = float(np.sqrt(np.mean((f8 - ref["forces"]) ** 2)))
    de32 = abs(e32 - ref["energy"]) / n
    rms32 = float(np.sqrt(np.mean((f32 - ref["forces"]) ** 2)))
    print(f"[fp8] {name} T={T} |dE|/N={de8:.3e} F rms={rms8:.3e}  "
          f"(fp32: |dE|/N={de32:.3e} F rms={rms32:.3e}; |F| rms={np.sqrt(np.mean(ref['forces'] ** 2)):.3e})")
    assert np.isfinite(e8) and np.isfinite(f8).all()
    assert de8 <= E_TOL and rms8 <= F_RMS_TOL
    assert rms8 > rms32  # the FP8 path really ran (it cannot match FP32)


def test_fp8_deterministic_and_momentum_free():
    from paper_2505_06711_gb300 import binding

    spec = make_model(T=3)
    s = water_box(8192, seed=0)
    e1, f1 = _eval(spec, s, binding.REANN_MLP_FP8)
    e2, f2 = _eval(spec, s, binding.REANN_MLP_FP8)
    assert e1 == e2 and np.array_equal(f1, f2)
    # the gather-only adjoint keeps Newton's third law up to FP32 rounding of the per-atom sums
    assert np.abs(f1.sum(axis=0)).max() <= 1e-3 * np.abs(f1).sum(axis=0).max()


def e4m3(x):
    """Round to the nearest-even FP8 E4M3 value (as float64), saturating at +-448."""
    x = np.asarray(x, np.float64)
    a = np.abs(x)
    _, ex = np.frexp(np.where(a > 0, a, 1.0))  # a = m 2^ex, m in [0.5, 1)
    e = np.clip(ex - 1, -6, 8)  # below 2^-6: the subnormal spacing 2^-9
    q = np.ldexp(1.0, e - 3)
    return np.sign(x) * np.minimum(np.round(a / q) * q, 448.0)


def _pow2_scale(amax):
    """2^e with amax / 2^e in [224, 448) (1 for zero), per entry, as the kernel and the host pick them."""
    amax = np.asarray(amax, np.float32)
    _, e = np.frexp((amax * np.float32(1.0 / 448.0)).astype(np.float32))
    return np.where(amax > 0, np.ldexp(np.float32(1.0), e), np.float32(1.0)).astype(np.float32)


def _silu(z):
    z = z.astype(np.float32)
    return (z / (np.float32(1.0) + np.exp(-z))).astype(np.float32)


def test_fp8_first_network_matches_emulation():
    """The first coefficient network in FP8 against numpy doing the same roundings.

    In the 192-atom water box each element's rows form a single 128-row tile:
    the anchor is the element's column mean, the deviations of each row are
    divided by the row's power-of-two scale and rounded to E4M3, the weights by
    max |w| / 448 per output unit, and the anchors' products and the output
    layer are FP32.  The kernel accumulates in FP32 (the emulation in
    FP64) and sums the means in another order, which can flip a rounding
    decision only where an operand sits on an E4M3 rounding boundary: nearly
    every output agrees to FP32 precision."""
    import torch

    from paper_2505_06711_gb300 import Potential, binding
    from synth.model import param_layout

    spec = make_model(T=3)
    s = water_box(64, seed=0)
    lay = param_layout(spec.n_elem, spec.T, spec.n_phi, spec.l_max, spec.n_orb, spec.h1, spec.h2)
    P = spec.params.astype(np.float32)

    def blk(t, e, name):
        off, shape = lay[(t, e, name)]
        return P[off:off + int(np.prod(shape))].reshape(shape)

    pot = Potential(spec, precision=binding.REANN_MLP_FP8)
    try:
        sy = pot.system(s.pos, s.species, s.cell, skin=1.0)
        sy.evaluate()
        sy.check()
        rho0, _ = sy.layer(0)
        _, c1 = sy.layer(1)
        torch.cuda.synchronize()
        rho0, c1 = rho0.cpu().numpy(), c1.cpu().numpy()
        sy.close()
    finally:
        pot.close()
    species = np.asarray(s.species)
    worst = []

    def product(x, w):
        """(x - mean) rounded per row, w rounded per output column, the mean's product in FP32."""
        xb = x.mean(axis=0, dtype=np.float64).astype(np.float32)
        d = (x - xb).astype(np.float32)
        sr = _pow2_scale(np.abs(d).max(axis=1))
        sc = (np.abs(w).max(axis=0).astype(np.float32) / np.float32(448.0)).astype(np.float32)
        qd = e4m3(d / sr[:, None])
        qw = e4m3(w / sc[None, :])
        return ((qd @ qw) * sr[:, None] * sc[None, :]).astype(np.float32) + (xb.astype(np.float64) @ w).astype(np.float32)

    for e in np.unique(species):
        rows = species == e
        assert rows.sum() <= 128  # one tile per element
        W1, b1, W2, b2, W3, b3 = (blk(0, e, k) for k in ("W1", "b1", "W2", "b2", "W3", "b3"))
        x = rho0[rows].astype(np.float32)
        h1 = _silu(product(x, W1) + b1)
        h2 = _silu(product(h1, W2) + b2)
        y = (h2.astype(np.float64) @ W3 + b3).astype(np.float32)
        rel = np.abs(c1[rows] - y) / (np.abs(y).max() + 1e-30)
        worst.append(rel)
        print(f"[fp8 emulation] element {e}: rows {rows.sum()}, median {np.median(rel):.2e}, "
              f"99th {np.percentile(rel, 99):.2e}, max {rel.max():.2e}")
    assert len(worst) == 2  # O and H
    rel = np.concatenate([w.ravel() for w in worst])
    assert np.percentile(rel, 99) <= 1e-4  # FP32 agreement apart from rare rounding-boundary flips
    assert rel.max() <= 5e-2
