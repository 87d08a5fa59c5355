"""Seeded REANN parameter sets in the flat FP32 layout read by both sides.

The paper trains its networks on DFT data (Sec. 4.1); those weights are not
available, so seeded draws stand in for them.  The parameter set covers what
Eqs. 1-2 and the output network (Sec. 2.1) need:

* ``c0[e][m]`` -- per-element initial orbital coefficients (layer 0), N(0, 1);
* ``W[t][l][m][k]`` -- per-layer contraction of the ``N_phi`` primitive
  Gaussians of angular momentum ``l`` into ``N_orb`` orbitals, Xavier-normal;
* per layer ``t`` and element ``e`` an atomic network
  ``F -> H1 -> H2 -> out`` (SiLU between layers, zero biases, Xavier-normal
  weights), ``out = N_phi`` for the coefficient networks ``t < T-1`` (Eq. 2) and
  ``out = 1`` for the energy network ``t = T-1``.

Flat order (all float32, row-major, ``x @ W`` convention so ``W1`` is
``[F][H1]``)::

    c0        [n_elem][n_phi]
    W         [T][L+1][n_phi][n_orb]
    for t in 0..T-1, for e in 0..n_elem-1:
        W1 [F][H1], b1 [H1], W2 [H1][H2], b2 [H2], W3 [H2][out_t], b3 [out_t]

with ``F = (L+1) * n_orb`` features ordered ``f = l * n_orb + k``.

Two fixed scale factors are folded into the draws (trained models absorb
them; random ones need them so that values stay O(1)):

* every ``W1`` row of angular momentum ``l`` of layer ``t`` and element ``e``
  is multiplied by ``FEATURE_SCALE[t][e][l]`` so that the network inputs stay
  within about [0, 1] in every layer (Eq. 1 squares the coefficients, so
  without it the features grow or decay geometrically with ``t``);
* every energy-network ``W3`` is drawn Xavier-normal, made non-negative (so
  that each atomic energy is bounded from below by -0.28 sum W3: with random
  signs the model is unbounded below and MD trajectories collapse into ever
  denser clusters) and multiplied by ``ENERGY_SCALE`` so that forces
  are O(1) eV/A.

No REANN arithmetic happens here: the module only draws and lays out numbers.
"""

from __future__ import annotations

import dataclasses
import math

import numpy as np

# Input scale folded into the W1 rows of angular momentum l, per layer t and
# element e: FEATURE_SCALE[t][e][l].  Chosen once, layer by layer, so that the
# largest network input of every feature block is 1 on the 8,192-molecule
# water box (H, O; seed 0), the 32,000-atom fcc Cu box (Cu; seed 0) and the
# 4,000-atom high-entropy-alloy box (Co, Cr, Fe, Mn, Ni; seed 0, eight-element
# model) with the default model seed (two significant digits; the Cu l=1
# block, suppressed by the fcc symmetry, takes the l=0 value).  Eq. 1 squares the coefficients, so
# the layer recursion maps an outlier ratio r to about r^2 per layer; scaling
# by the maximum (not the RMS) keeps the random networks in their mildly
# non-linear range on large boxes instead of letting outliers grow without
# bound.  Layers beyond the table reuse its last row.
FEATURE_SCALE = (
    ((0.054, 0.16, 0.0017), (0.046, 0.21, 0.0019), (0.35, 0.35, 0.014),
     (0.2, 0.14, 0.021), (0.16, 0.13, 0.013), (0.21, 0.16, 0.019), (0.21, 0.14, 0.017), (0.16, 0.16, 0.013)),
    ((19.0, 46.0, 2.7), (16.0, 53.0, 3.3), (5.5, 5.5, 0.14),
     (37.0, 55.0, 2.4), (33.0, 56.0, 2.0), (33.0, 27.0, 1.8), (34.0, 48.0, 2.0), (38.0, 36.0, 1.6)),
    ((26.0, 24.0, 0.78), (17.0, 27.0, 0.87), (110.0, 110.0, 5.8),
     (56.0, 20.0, 4.0), (85.0, 31.0, 6.7), (74.0, 19.0, 5.6), (84.0, 34.0, 6.1), (84.0, 47.0, 6.5)),
    ((5.7, 12.0, 1.0), (7.9, 11.0, 1.7), (15.0, 15.0, 2.2),
     (54.0, 23.0, 5.3), (41.0, 24.0, 5.4), (24.0, 13.0, 3.5), (78.0, 38.0, 8.5), (56.0, 45.0, 7.1)),
    ((7.7, 8.7, 4.2), (4.6, 10.0, 4.3), (15.0, 15.0, 1.6),
     (210.0, 34.0, 6.3), (230.0, 49.0, 7.0), (76.0, 24.0, 7.1), (380.0, 57.0, 12.0), (210.0, 44.0, 6.4)),
)
# The same for the orbital-pair-product features (8 orbitals, 36 pairs per l,
# elements H, O, Cu), calibrated the same way, layer by layer, on the
# 2,048-molecule water box and the 4,000-atom Cu box (seed 0).
FEATURE_SCALE_PAIRS = (
    ((0.036, 0.11, 0.0025), (0.041, 0.14, 0.0028), (0.17, 0.17, 0.011)),
    ((8.3, 18.0, 1.4), (9.5, 18.0, 1.4), (21.0, 21.0, 0.66)),
    ((28.0, 65.0, 0.92), (53.0, 87.0, 1.2), (4.0, 4.0, 0.36)),
    ((12.0, 19.0, 0.78), (17.0, 24.0, 1.2), (58.0, 58.0, 1.3)),
    ((24.0, 12.0, 0.62), (58.0, 18.0, 1.0), (40.0, 40.0, 14.0)),
)
# Multiplier on the energy network's output weights (eV): gives forces of
# about 2 eV/A (99th percentile) on the water box and 0.5 eV/A (median) on
# the Cu box at T = 3.
ENERGY_SCALE = 4.0


@dataclasses.dataclass
class ModelSpec:
    n_elem: int
    T: int
    n_phi: int
    l_max: int
    n_orb: int
    h1: int
    h2: int
    r_c: float
    alpha: float
    params: np.ndarray  # float32 flat
    pairs: bool = False  # features: Eq. 1's squares (False) or orbital-pair products (True)

    @property
    def n_feat(self) -> int:
        return n_features(self.l_max, self.n_orb, self.pairs)

    def out_dim(self, t: int) -> int:
        return 1 if t == self.T - 1 else self.n_phi


def n_features(l_max: int, n_orb: int, pairs: bool = False) -> int:
    """(L+1) n_orb squares (Eq. 1), or (L+1) n_orb (n_orb+1)/2 orbital-pair products."""
    return (l_max + 1) * (n_orb * (n_orb + 1) // 2 if pairs else n_orb)


def param_layout(n_elem: int, T: int, n_phi: int, l_max: int, n_orb: int, h1: int, h2: int,
                 pairs: bool = False) -> dict:
    """Offsets (in floats) of every block of the flat parameter vector."""
    f = n_features(l_max, n_orb, pairs)
    off = 0
    lay: dict = {"c0": (off, (n_elem, n_phi))}
    off += n_elem * n_phi
    lay["W"] = (off, (T, l_max + 1, n_phi, n_orb))
    off += T * (l_max + 1) * n_phi * n_orb
    for t in range(T):
        out = 1 if t == T - 1 else n_phi
        for e in range(n_elem):
            for name, shape in (
                ("W1", (f, h1)),
                ("b1", (h1,)),
                ("W2", (h1, h2)),
                ("b2", (h2,)),
                ("W3", (h2, out)),
                ("b3", (out,)),
            ):
                lay[(t, e, name)] = (off, shape)
                off += int(np.prod(shape))
    lay["total"] = off
    return lay


def _xavier(rng: np.random.Generator, fan_in: int, fan_out: int, gain: float = 1.0) -> np.ndarray:
    std = gain * math.sqrt(2.0 / (fan_in + fan_out))
    return rng.normal(0.0, std, size=(fan_in, fan_out))


def make_model(
    T: int = 3,
    seed: int = 1234,
    n_elem: int = 3,
    n_phi: int = 8,
    l_max: int = 2,
    n_orb: int = 16,
    h1: int = 64,
    h2: int = 64,
    r_c: float = 5.0,
    alpha: float = 0.5,
    feature_scale: tuple | None = None,
    energy_scale: float | None = None,
    pairs: bool = False,
) -> ModelSpec:
    """Draw a seeded parameter set (see module docstring for the layout).

    ``pairs=True`` selects the orbital-pair-product features (with the default
    ``n_orb`` then 8, the feature count N_phi (N_phi+1) (L+1)/2 = 108 that
    Sec. 2.1 states) and their own input scales.
    """
    if T < 1:
        raise ValueError("T must be >= 1")
    if pairs and n_orb == 16:
        n_orb = 8
    fs = (FEATURE_SCALE_PAIRS if pairs else FEATURE_SCALE) if feature_scale is None else feature_scale
    if any(len(row) < l_max + 1 for per_t in fs for row in per_t):
        raise ValueError("feature_scale needs one entry per l")
    es = ENERGY_SCALE if energy_scale is None else energy_scale
    lay = param_layout(n_elem, T, n_phi, l_max, n_orb, h1, h2, pairs)
    per_l = n_orb * (n_orb + 1) // 2 if pairs else n_orb  # features per angular momentum

    def stream(*key):
        # an independent substream per block, so layer t's draws do not depend on T
        return np.random.Generator(np.random.PCG64([seed, *key]))

    p = np.zeros(lay["total"], dtype=np.float64)

    def put(key, arr):
        o, shape = lay[key]
        p[o : o + int(np.prod(shape))] = np.asarray(arr, dtype=np.float64).reshape(-1)

    put("c0", stream(0).normal(0.0, 1.0, size=(n_elem, n_phi)))
    put("W", np.stack([np.stack([_xavier(stream(1, t, l), n_phi, n_orb) for l in range(l_max + 1)]) for t in range(T)]))
    f = (l_max + 1) * per_l
    for t in range(T):
        out = 1 if t == T - 1 else n_phi
        for e in range(n_elem):
            row = np.asarray(fs[min(t, len(fs) - 1)][min(e, len(fs[0]) - 1)][: l_max + 1], dtype=np.float64)
            put((t, e, "W1"), _xavier(stream(2, t, e), f, h1) * np.repeat(row, per_l)[:, None])
            put((t, e, "b1"), np.zeros(h1))
            put((t, e, "W2"), _xavier(stream(3, t, e), h1, h2))
            put((t, e, "b2"), np.zeros(h2))
            w3 = _xavier(stream(4 if t < T - 1 else 5, t, e), h2, out)
            if t == T - 1:
                # non-negative output weights: SiLU >= -0.28 then bounds every atomic
                # energy from below, so clustering cannot release unbounded energy
                w3 = np.abs(w3) * es
            put((t, e, "W3"), w3)
            put((t, e, "b3"), np.zeros(out))
    return ModelSpec(n_elem, T, n_phi, l_max, n_orb, h1, h2, float(r_c), float(alpha), p.astype(np.float32), pairs)


MODEL_FILE_MAGIC = b"REANNMDL"
MODEL_FILE_VERSION = 1


def write_model_file(spec: ModelSpec, path) -> None:
    """Write ``spec`` in the model-file layout that ``reann_model_load`` reads.

    Little-endian: the 8-byte magic, uint32 version, int32 n_elem, T, n_phi,
    l_max, n_orb, h1, h2, feature_pairs, uint32 0, float64 r_c, alpha, int64
    n_params, then the float32 parameters.  Layout only: no REANN arithmetic.
    """
    params = np.ascontiguousarray(spec.params, dtype="<f4")
    head = np.array(
        [spec.n_elem, spec.T, spec.n_phi, spec.l_max, spec.n_orb, spec.h1, spec.h2, int(bool(spec.pairs))],
        dtype="<i4",
    )
    with open(path, "wb") as f:
        f.write(MODEL_FILE_MAGIC)
        f.write(np.array([MODEL_FILE_VERSION], dtype="<u4").tobytes())
        f.write(head.tobytes())
        f.write(np.array([0], dtype="<u4").tobytes())
        f.write(np.array([spec.r_c, spec.alpha], dtype="<f8").tobytes())
        f.write(np.array([params.size], dtype="<i8").tobytes())
        f.write(params.tobytes())
