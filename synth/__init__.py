"""Seeded synthetic inputs shared by the FP64 oracle and the CUDA path.

This package draws random numbers and lays them out; it holds none of the
REANN arithmetic (no distances, orbitals, densities or networks).  Both the
oracle (``oracle/``) and the GPU library consume what it produces:

* :mod:`synth.structures` -- periodic water boxes, fcc metal and high-entropy
  alloy boxes
  (the paper's benchmark system types, Sec. 2.3 and Sec. 4.1), Maxwell-Boltzmann
  velocities for NVE runs.
* :mod:`synth.model` -- a seeded REANN parameter set in the flat FP32 layout
  that both sides read (the paper's trained weights are not available, so
  Xavier-normal draws stand in for them).
"""

from .structures import (  # noqa: F401
    Structure,
    water_box,
    fcc_box,
    hea_box,
    supercell,
    maxwell_boltzmann,
    SPECIES_H,
    SPECIES_O,
    SPECIES_CU,
    SPECIES_HEA,
    MASS_AMU,
)
from .model import ModelSpec, make_model, param_layout, write_model_file  # noqa: F401
