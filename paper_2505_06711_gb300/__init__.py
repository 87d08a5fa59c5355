"""GB300-native REANN energy/force evaluation (arXiv 2505.06711).

The computation lives in the CUDA library ``libreann.so`` (``csrc/``, C ABI in
``include/reann.h``).  This package holds its ctypes binding
(:mod:`.binding`, same names as the C entry points) and a small convenience
layer that keeps device buffers in torch tensors.  PyTorch provides device
memory and streams only.
"""

from __future__ import annotations

import numpy as np

from . import binding
from .binding import ReannError  # noqa: F401

__all__ = ["Potential", "System", "binding", "ReannError", "ReannEnergy", "energy"]


def _energy_function():
    import torch

    class ReannEnergy(torch.autograd.Function):
        """E(pos) as a differentiable torch op over the library's hand-written adjoint.

        forward runs reann_energy_forces (T forward layers, then the reverse
        pass of Eqs. 3-5 in the same call) and keeps F = -dE/dpos; backward
        returns -F * grad_E, so no autograd graph is ever built through the
        message-passing layers.
        """

        @staticmethod
        def forward(ctx, pos, system):
            system.evaluate(pos.detach().contiguous(), atom_energy=False)
            ctx.save_for_backward(system.forces.detach().to(pos.dtype).clone())
            return system.energy.detach().clone().reshape(()).to(pos.dtype)

        @staticmethod
        def backward(ctx, grad_e):
            (forces,) = ctx.saved_tensors
            return -grad_e * forces, None

    return ReannEnergy


def energy(pos, system):
    """Differentiable total energy (0-d FP64 tensor) of ``system`` at ``pos`` (N x 3 FP64 CUDA)."""
    global ReannEnergy
    if ReannEnergy is None:
        ReannEnergy = _energy_function()
    return ReannEnergy.apply(pos, system)


ReannEnergy = None


class Potential:
    """A model uploaded to one CUDA device with its own execution context."""

    def __init__(self, spec, stream=None, precision: int = binding.REANN_MLP_FP32):
        import torch

        self.spec = spec
        self.T = spec.T
        self.r_c = float(spec.r_c)
        self.device = torch.device("cuda", torch.cuda.current_device())
        self._model = binding.reann_model_create(spec)
        try:
            self.ctx = binding.reann_ctx_create(self._model, stream)
        finally:
            binding.reann_model_free(self._model)
            self._model = None
        if precision != binding.REANN_MLP_FP32:
            binding.reann_ctx_set_mlp_precision(self.ctx, precision)

    def set_precision(self, precision: int) -> None:
        binding.reann_ctx_set_mlp_precision(self.ctx, precision)

    def system(self, pos, species, cell, skin: float = 1.0, ranks=None) -> "System":
        """One structure; ``ranks`` = (kx, ky, kz) builds the virtual-rank decomposed list."""
        return System(self, pos, species, cell, skin, ranks)

    def close(self) -> None:
        if getattr(self, "ctx", None) is not None:
            binding.reann_ctx_free(self.ctx)
            self.ctx = None

    def __del__(self):  # pragma: no cover - best effort
        try:
            self.close()
        except Exception:
            pass


class System:
    """One periodic structure with its resident neighbour list and buffers."""

    def __init__(self, pot: Potential, pos, species, cell, skin: float = 1.0, ranks=None):
        import torch

        self.pot = pot
        self.cell = np.ascontiguousarray(cell, dtype=np.float64).reshape(3, 3)
        self.skin = float(skin)
        self.pos = torch.as_tensor(np.asarray(pos, dtype=np.float64), device=pot.device).contiguous()
        self.species = torch.as_tensor(np.asarray(species, dtype=np.int32), device=pot.device).contiguous()
        self.n = int(self.pos.shape[0])
        if ranks is None:
            self.nl = binding.reann_build_nlist(pot.ctx, self.pos, self.species, self.cell, pot.r_c, self.skin)
        else:
            self.nl = binding.reann_build_nlist_decomposed(pot.ctx, self.pos, self.species, self.cell, pot.r_c,
                                                           self.skin, ranks)
        self.energy = torch.zeros(1, dtype=torch.float64, device=pot.device)
        self.forces = torch.zeros((self.n, 3), dtype=torch.float32, device=pot.device)
        self.atom_energy = torch.zeros(self.n, dtype=torch.float32, device=pot.device)

    def rebuild(self, pos=None) -> None:
        """Enqueue a device-side neighbour-list rebuild at ``pos`` (default: the build positions)."""
        binding.reann_nlist_rebuild(self.pot.ctx, self.nl, self.pos if pos is None else pos)

    def evaluate_host(self, pos, energy, forces, rebuild: bool = False) -> None:
        """Host-buffer evaluation (synchronous): copies in, rebuilds if needed, evaluates, copies out."""
        binding.reann_energy_forces_host(self.pot.ctx, self.nl, pos, self.pot.T, energy, forces, int(rebuild))

    def evaluate(self, pos=None, atom_energy: bool = True, virial: bool = False, atom_virial: bool = False) -> None:
        """Enqueue one energy + force evaluation (results in .energy/.forces/.atom_energy,
        with ``virial`` also .virial (3 x 3 FP64, W = -dE/d strain) and, with
        ``atom_virial``, .atom_virial (N x 9))."""
        import torch

        p = self.pos if pos is None else pos
        ae = self.atom_energy if atom_energy else None
        if not virial:
            binding.reann_energy_forces(self.pot.ctx, self.nl, p, self.pot.T, self.energy, self.forces, ae)
            return
        if getattr(self, "virial", None) is None:
            self.virial = torch.zeros((3, 3), dtype=torch.float64, device=self.pot.device)
        av = None
        if atom_virial:
            if getattr(self, "atom_virial", None) is None:
                self.atom_virial = torch.zeros((self.n, 9), dtype=torch.float32, device=self.pot.device)
            av = self.atom_virial
        binding.reann_energy_forces_virial(self.pot.ctx, self.nl, p, self.pot.T, self.energy, self.forces,
                                           self.virial, ae, av)

    def md(self, vel, mass, dt_fs: float, n_steps: int, record: bool = True, temperature_k: float | None = None,
           tau_fs: float = 100.0):
        """Velocity Verlet in place on self.pos / vel: NVE, or NVT (Nose-Hoover) when
        ``temperature_k`` is given.  Returns (E_pot, E_kin) per step, with NVT
        (E_pot, E_kin, E_bath), or None when not recording."""
        import torch

        def rec():
            return torch.zeros(n_steps, dtype=torch.float64, device=self.pot.device) if record else None

        e_pot, e_kin = rec(), rec()
        if temperature_k is None:
            binding.reann_md_step(self.pot.ctx, self.nl, self.pos, vel, mass, dt_fs, n_steps, e_pot, e_kin)
            return (e_pot, e_kin) if record else None
        e_bath = rec()
        binding.reann_md_step_nvt(self.pot.ctx, self.nl, self.pos, vel, mass, dt_fs, n_steps, temperature_k, tau_fs,
                                  e_pot, e_kin, e_bath)
        return (e_pot, e_kin, e_bath) if record else None

    def md_info(self):
        return binding.reann_md_info(self.pot.ctx, self.nl)

    def layer(self, t: int):
        import torch

        rho = torch.zeros((self.n, self.pot.spec.n_feat), dtype=torch.float32, device=self.pot.device)
        coef = torch.zeros((self.n, 8), dtype=torch.float32, device=self.pot.device)
        binding.reann_get_layer(self.pot.ctx, self.nl, t, rho, coef)
        return rho, coef

    def neighbors(self):
        return binding.reann_nlist_export(self.pot.ctx, self.nl)

    def info(self):
        return binding.reann_nlist_info(self.nl)

    def ranks(self) -> dict:
        """Per virtual rank: local atoms, ghost slots, ghost slots owned by another rank."""
        return binding.reann_decomp_info(self.nl)

    def check(self) -> None:
        binding.reann_ctx_check(self.pot.ctx)

    def close(self) -> None:
        if getattr(self, "nl", None) is not None:
            binding.reann_nlist_free(self.nl)
            self.nl = None

    def __del__(self):  # pragma: no cover
        try:
            self.close()
        except Exception:
            pass
