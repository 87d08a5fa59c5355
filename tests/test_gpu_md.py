"""NVE velocity-Verlet MD through reann_md_step (FP64 integrator, graph-replayed steps)."""

from __future__ import annotations

import numpy as np
import pytest

import oracle
from synth import MASS_AMU, make_model, maxwell_boltzmann, water_box

from gpu_helpers import F_TOL_MAX, assert_parity, potential

pytestmark = pytest.mark.gpu

ACCEL = 9.648533212e-3  # (eV/A)/amu -> A/fs^2


def _setup(n_mol, seed, T=3):
    import torch

    s = water_box(n_mol, seed=seed)
    spec = make_model(T=T)
    pot = potential(spec)
    sy = pot.system(s.pos, s.species, s.cell, skin=1.0)
    m = MASS_AMU[s.species]
    v = maxwell_boltzmann(m, 300.0, seed=seed)
    vel = torch.as_tensor(v, device="cuda").contiguous()
    mass = torch.as_tensor(m, device="cuda").contiguous()
    return s, spec, pot, sy, vel, mass


def test_one_step_is_velocity_verlet():
    import torch

    s, spec, pot, sy, vel, mass = _setup(64, 1)
    dt = 0.5
    x0, v0 = sy.pos.clone(), vel.clone()
    sy.evaluate()
    f0 = sy.forces.double().clone()
    vh = v0 + 0.5 * dt * ACCEL * f0 / mass[:, None]
    x1 = x0 + dt * vh
    sy.evaluate(x1.contiguous())
    f1 = sy.forces.double().clone()
    v1 = vh + 0.5 * dt * ACCEL * f1 / mass[:, None]
    e_pot, e_kin = sy.md(vel, mass, dt, 1)
    sy.check()
    torch.cuda.synchronize()
    np.testing.assert_allclose(sy.pos.cpu().numpy(), x1.cpu().numpy(), rtol=0, atol=1e-12)
    np.testing.assert_allclose(vel.cpu().numpy(), v1.cpu().numpy(), rtol=0, atol=1e-12)
    ke = 0.5 * (mass[:, None] * v1 * v1).sum().item() / ACCEL
    assert e_kin[0].item() == pytest.approx(ke, rel=1e-12)
    ref = oracle.energy_forces(spec, x1.cpu().numpy(), s.species, s.cell)
    assert abs(e_pot[0].item() - ref["energy"]) / s.n_atoms < 1e-6


def test_nve_conserves_energy_across_device_rebuilds():
    import torch

    # dt 0.25 fs: the random model heats this box and drives molecules into close
    # contacts, where the Verlet error of a single trajectory (~dt^2) dominates the
    # drift statistic at 0.5 fs; rebuild errors would show as jumps at any dt
    s, spec, pot, sy, vel, mass = _setup(512, 2)
    n_steps, dt = 2000, 0.25
    e_pot, e_kin = sy.md(vel, mass, dt, n_steps)
    sy.check()
    torch.cuda.synchronize()
    steps, rebuilds = sy.md_info()
    assert steps == n_steps
    assert rebuilds >= 1  # atoms moved beyond skin/2: the list was rebuilt on the device
    etot = ((e_pot + e_kin) / s.n_atoms).cpu().numpy()
    t_ps = np.arange(1, n_steps + 1) * dt * 1e-3
    slope, icpt = np.polyfit(t_ps, etot, 1)  # eV/atom/ps
    fluct = float((etot - (slope * t_ps + icpt)).std())  # about the linear drift
    print(f"[md] rebuilds={rebuilds} drift={slope * 1e3:.4f} meV/atom/ps "
          f"fluct={fluct * 1e3:.4f} meV/atom max step {np.abs(np.diff(etot)).max() * 1e3:.4f} meV/atom "
          f"ekin/N={e_kin[-1].item() / s.n_atoms:.4f}")
    assert abs(slope) < 1e-3  # |drift| < 1 meV/atom/ps
    assert fluct < 2e-4
    # no jump where the list was rebuilt: the largest step-to-step change of E_tot is
    # of the size of the ordinary Verlet fluctuation
    assert np.abs(np.diff(etot)).max() < 2e-4
    # the trajectory's last state agrees with a fresh build at the final positions
    ref = oracle.energy_forces(spec, sy.pos.cpu().numpy(), s.species, s.cell)
    assert abs(e_pot[-1].item() - ref["energy"]) / s.n_atoms < 1e-6
    fresh = pot.system(sy.pos.cpu().numpy(), s.species, s.cell)
    fresh.evaluate()
    fresh.check()
    torch.cuda.synchronize()
    # After 1 ps the random model has heated the box to ~1,100 K and the end state
    # holds close contacts (down to ~0.1 A) with forces up to ~8 eV/A.  FP32
    # rounding in the edge sums is relative to the force (measured <= 2e-5 |F|
    # per atom), so the absolute bar, set for forces of order 1 eV/A, scales with
    # the largest force here.
    f_scale = max(1.0, float(np.abs(ref["forces"]).max()))
    assert_parity({"energy": fresh.energy.item(), "forces": fresh.forces.double().cpu().numpy()},
                  {k: ref[k] for k in ("energy", "forces")}, s.n_atoms, f_tol=F_TOL_MAX * f_scale)
    fresh.close()
    sy.close()


KB = 8.617333262e-5  # eV/K


def test_one_nvt_step_is_the_stated_splitting():
    """One reann_md_step_nvt step against the Nose-Hoover splitting written out
    here: thermostat half step, half kick, drift, forces, half kick, thermostat
    half step (xi, eta start at 0)."""
    import torch

    s, spec, pot, sy, vel, mass = _setup(64, 4)
    dt, T0, tau = 0.5, 300.0, 20.0
    n = s.n_atoms
    gkt = (3 * n - 3) * KB * T0
    q = gkt * tau * tau
    m = mass.double()[:, None]

    def ekin(v):
        return 0.5 * (m * v * v).sum().item() / ACCEL

    def half(K, xi, eta):
        xi += 0.25 * dt * (2 * K - gkt) / q
        eta += 0.5 * dt * xi
        sc = np.exp(-0.5 * dt * xi)
        K *= sc * sc
        xi += 0.25 * dt * (2 * K - gkt) / q
        return K, xi, eta, sc

    x0, v0 = sy.pos.clone(), vel.clone()
    sy.evaluate()
    f0 = sy.forces.double().clone()
    K, xi, eta, sc = half(ekin(v0), 0.0, 0.0)
    v = sc * v0 + 0.5 * dt * ACCEL * f0 / m
    x1 = x0 + dt * v
    sy.evaluate(x1.contiguous())
    f1 = sy.forces.double().clone()
    v = v + 0.5 * dt * ACCEL * f1 / m
    K, xi, eta, sc = half(ekin(v), xi, eta)
    v = sc * v
    e_pot, e_kin, e_bath = sy.md(vel, mass, dt, 1, temperature_k=T0, tau_fs=tau)
    sy.check()
    torch.cuda.synchronize()
    np.testing.assert_allclose(sy.pos.cpu().numpy(), x1.cpu().numpy(), rtol=0, atol=1e-12)
    np.testing.assert_allclose(vel.cpu().numpy(), v.cpu().numpy(), rtol=0, atol=1e-12)
    assert e_kin[0].item() == pytest.approx(K, rel=1e-12)
    assert e_bath[0].item() == pytest.approx(0.5 * q * xi * xi + gkt * eta, rel=1e-10, abs=1e-12)


def test_nvt_holds_temperature_and_conserves_extended_energy():
    """4 ps of NVT at 300 K on a 2,048-atom Cu box (the random water model, held
    at 300 K, lets molecules fall into 0.1 A contacts where 0.5 fs steps no
    longer resolve the motion; the crystal stays on its lattice).  Measured on
    GB300: late mean 298.2 K, extended-energy drift -0.096 meV/atom/ps at
    dt = 1 fs (-0.024 at 0.5 fs: second order in dt)."""
    import torch

    from synth import fcc_box

    s = fcc_box(8, seed=3)
    spec = make_model(T=3)
    pot = potential(spec)
    sy = pot.system(s.pos, s.species, s.cell, skin=1.0)
    m = MASS_AMU[s.species]
    vel = torch.as_tensor(maxwell_boltzmann(m, 300.0, seed=3), device="cuda").contiguous()
    mass = torch.as_tensor(m, device="cuda").contiguous()
    n_steps, dt, T0, tau = 4000, 1.0, 300.0, 100.0
    e_pot, e_kin, e_bath = sy.md(vel, mass, dt, n_steps, temperature_k=T0, tau_fs=tau)
    sy.check()
    torch.cuda.synchronize()
    n = s.n_atoms
    temp = 2.0 * e_kin.cpu().numpy() / ((3 * n - 3) * KB)
    h = ((e_pot + e_kin + e_bath) / n).cpu().numpy()
    t_ps = np.arange(1, n_steps + 1) * dt * 1e-3
    slope = np.polyfit(t_ps, h, 1)[0]
    late = temp[n_steps // 2:]
    print(f"[nvt] T mean(late)={late.mean():.1f} K std={late.std():.1f} K "
          f"drift={slope * 1e3:.4f} meV/atom/ps fluct={h.std() * 1e3:.4f} meV/atom rebuilds={sy.md_info()[1]}")
    assert abs(slope) < 5e-4  # |drift| of the conserved quantity < 0.5 meV/atom/ps
    assert abs(late.mean() - T0) < 0.03 * T0
    assert e_bath.cpu().numpy()[-1] / n > 0.5  # the bath took up the released potential energy
    sy.close()
