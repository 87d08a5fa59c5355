#!/usr/bin/env python
"""REANN energy + force throughput on GB300 (atom-evaluations per second, T = 3).

One step is one pass of the whole hot path over the 8,192-molecule periodic
water box (24,576 atoms, 1.0 g/cm^3, skin 1 A, T = 3): device-side neighbour
list rebuild (cell list, ghost slots), then the energy/force evaluation
(T density layers with per-layer ghost refresh, per-element networks, FP64
energy sum, reverse pass).  Inputs are synthetic (seeded water box, seeded
random-weight model); the paper's datasets and trained weights are not used.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

* ``value``: atoms x ranks / device time per step, device time from CUDA events
  around each step on the library's stream; the L2 cache (129 MB) is flushed by
  writing a 256 MiB buffer before every timed step (outside the events).
* ``e2e``: the same step through the C ABI with host buffers
  (``reann_energy_forces_host`` with a forced rebuild): pinned host positions
  in, host forces and energy out, copies inside the timed region.
* ``roofline``: the region with the largest device time, its algorithmic FLOPs
  per launch (the FLOP_PER_* counts below) over its mean launch time, against the FP32
  SIMT peak of the GPU (SMs x 128 lanes x 2 FLOP x max SM clock); beside it the
  same fraction with the scope table's coarser counts (``frac_alu_survey``), the
  edge kernel's algorithmic HBM bytes over its time against the measured copy
  bandwidth (``frac_hbm``), and ncu's L2 throughput share (``frac_l2``).
* ``cpu_baseline``: the FP64 oracle (test infrastructure) evaluating the same
  box once on the host cores, rank 0 only.
* ``--impl reference``: the oracle is the reference arm; each step is one full
  oracle evaluation of the same box, the run bounded at about two minutes.

With N > 1 (torchrun) every rank runs an independent replica (the path needs
no data exchange on one structure per GPU); timing is max over ranks.
"""

from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

N_MOLECULES = 8192
T_LAYERS = 3
SKIN = 1.0
FLUSH_BYTES = 256 << 20

# Algorithmic FP32 FLOPs (FMA = 2) of each timed region, from the formulas of
# Eq. 1 (forward), Eqs. 3-5 (reverse) and the 48-64-64-{8,1} networks (Eq. 2).
FLOP_PER_LIVE_EDGE_FWD = 176          # 80 FMA of b += c phi A, 8 c*phi, 8 phi*f_c
FLOP_PER_ATOM_FWD = 2880              # contraction 10x16x8 FMA + 160 squares
FLOP_PER_LIVE_EDGE_ADJ = 640          # 80 x (2 FMA combination + 2 FMA radial/angular sums)
FLOP_PER_LIVE_EDGE_ADJ_CBAR = 160     # 80 FMA of cbar (layers t >= 1)
FLOP_PER_ATOM_MLP_FWD = {8: 15360, 1: 14464}
FLOP_PER_ATOM_MLP_BWD = {8: 15360, 1: 14464}  # the vector-Jacobian product W3, W2, W1 (no recompute)
FLOP_PER_ATOM_BBAR = 5440             # g (1280 FMA) + gbar (160) + bbar (1280 FMA)

# The same regions counted as the hot-path scope table counts them (a coarser
# operation count: ~130 FP32 operations per live edge forward, twice that in
# the reverse pass), reported beside the counts above.
FLOP_PER_LIVE_EDGE_FWD_COARSE = 130
FLOP_PER_LIVE_EDGE_ADJ_COARSE = 260
FLOP_PER_ATOM_CONTRACTION_COARSE = 2 * 1280

# Algorithmic HBM bytes per atom and layer of the edge kernels: the neighbour
# row (4 B per listed entry within r_c + skin), the atom's position (16 B) and
# coefficients (32 B), the b checkpoint (320 B), and for the forward pass the
# features rho (192 B); neighbours' positions and coefficients are re-reads
# served by L2.
BYTES_PER_ATOM_EDGE_FIXED = {"density_fwd": 16 + 32 + 320 + 192, "density_adj": 16 + 32 + 320}

# DRAM traffic and L2 throughput (share of peak) per launch of the dominant
# kernel, from one ncu capture of this workload; valid only for the kernel
# source they were taken on (keyed by its hash), null otherwise.
TRAFFIC = {  # {(region, source_sha of the kernel source): bytes per launch}
    ("density_adj", "3dae6077f620"): 22066603,  # mean of the three launches of one step
}
L2_FRAC = {  # {(region, source_sha): lts__t_sectors throughput as a fraction of peak}
    ("density_adj", "3dae6077f620"): 0.319,
}


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=400)
    p.add_argument("--warmup", type=int, default=20)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-md", action="store_true")
    p.add_argument("--no-t-scaling", action="store_true")
    p.add_argument("--md-steps", type=int, default=1000)
    p.add_argument("--no-serve", action="store_true")
    p.add_argument("--no-decomp", action="store_true")
    p.add_argument("--no-hea", action="store_true")
    p.add_argument("--no-pairs", action="store_true")
    p.add_argument("--serve-requests", type=int, default=10000)
    return p.parse_args()


def run_hea(args, steps: int = 10):
    """Five-element fcc high-entropy alloy (eight-element model), T = 3: the same step
    (rebuild + energy/forces) on 32,000 and 1,048,576 atoms, FP32 and BF16 networks."""
    import torch

    from paper_2505_06711_gb300 import Potential, binding
    from synth import hea_box, make_model

    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    out = {"workload": "fcc random solid solution of Co, Cr, Fe, Mn, Ni in equal shares, a = 3.59 A, "
                       f"skin {SKIN} A, T = {T_LAYERS}, step = rebuild + energy/forces"}
    pot = Potential(make_model(T=T_LAYERS, n_elem=8))
    for k in (20, 64):
        s = hea_box(k, seed=0)
        sy = pot.system(s.pos, s.species, s.cell, skin=SKIN)
        res = {"atoms": s.n_atoms}
        for name, prec in (("fp32", binding.REANN_MLP_FP32), ("bf16_mlp", binding.REANN_MLP_BF16)):
            binding.reann_ctx_set_mlp_precision(pot.ctx, prec)

            def step():
                binding.reann_nlist_rebuild(pot.ctx, sy.nl, sy.pos)
                binding.reann_energy_forces(pot.ctx, sy.nl, sy.pos, T_LAYERS, sy.energy, sy.forces, None)

            for _ in range(3):
                step()
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
            for a, b in ev:
                flush.zero_()
                a.record()
                step()
                b.record()
            torch.cuda.synchronize()
            binding.reann_ctx_check(pot.ctx)
            ms = sum(a.elapsed_time(b) for a, b in ev) / steps
            res[name] = {"ms_per_step": ms, "atom_evals_per_s": s.n_atoms / (ms * 1e-3)}
        binding.reann_ctx_set_mlp_precision(pot.ctx, binding.REANN_MLP_FP32)
        out[f"hea{k}"] = res
        sy.close()
    pot.close()
    return out


def run_pairs(args, steps: int = 50):
    """The orbital-pair-product feature variant (108 features over 8 orbitals, the count Sec. 2.1
    states) on the same 24,576-atom water box and step (rebuild + energy/forces), FP32 networks."""
    import torch

    from paper_2505_06711_gb300 import Potential, binding
    from synth import make_model, water_box

    s = water_box(8192, seed=0)
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    pot = Potential(make_model(T=T_LAYERS, pairs=True))
    sy = pot.system(s.pos, s.species, s.cell, skin=SKIN)

    def step():
        binding.reann_nlist_rebuild(pot.ctx, sy.nl, sy.pos)
        binding.reann_energy_forces(pot.ctx, sy.nl, sy.pos, T_LAYERS, sy.energy, sy.forces, None)

    for _ in range(5):
        step()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for a, b in ev:
        flush.zero_()
        a.record()
        step()
        b.record()
    torch.cuda.synchronize()
    binding.reann_ctx_check(pot.ctx)
    ms = sum(a.elapsed_time(b) for a, b in ev) / steps
    sy.close()
    pot.close()
    return {"workload": f"water box 8192 H2O ({s.n_atoms} atoms), T = {T_LAYERS}, 108 pair features, FP32",
            "ms_per_step": ms, "atom_evals_per_s": s.n_atoms / (ms * 1e-3)}


def run_decomp(args, steps: int = 100):
    """The paper's spatial decomposition (Sec. 2.2) as virtual ranks on one GPU.

    Same 24,576-atom water box and T = 3 evaluation; the undivided list against
    2x2x2 and 4x4x4 subdomains, whose ghost slots are refreshed from their
    owners before every layer (c) and in the reverse pass (bbar).  Reports the
    evaluation time (no rebuild) and the halo sizes; forces are bitwise those
    of the undivided list (tests/test_gpu_decomp.py).
    """
    import torch

    from paper_2505_06711_gb300 import Potential
    from synth import make_model, water_box

    s = water_box(8192, seed=0)
    pot = Potential(make_model(T=T_LAYERS))
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    out = {"workload": f"water box 8192 H2O ({s.n_atoms} atoms), T = {T_LAYERS}, evaluation only"}
    for label, ranks in (("1x1x1", None), ("2x2x2", (2, 2, 2)), ("4x4x4", (4, 4, 4))):
        sy = pot.system(s.pos, s.species, s.cell, skin=SKIN, ranks=ranks)
        for _ in range(5):
            sy.evaluate(atom_energy=False)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for a, b in ev:
            flush.zero_()
            a.record()
            sy.evaluate(atom_energy=False)
            b.record()
        torch.cuda.synchronize()
        sy.check()
        ms = sum(a.elapsed_time(b) for a, b in ev) / steps
        info = sy.ranks()
        remote = int(info["remote"].sum())
        out[label] = {
            "ranks": len(info["local"]),
            "ms_per_eval": ms,
            "atom_evals_per_s": s.n_atoms / (ms * 1e-3),
            "ghost_slots": int(info["ghosts"].sum()),
            "remote_ghost_slots": remote,
            # per layer: c (8 FP32) forward and bbar (80 FP32) backward for every remote ghost
            "exchange_bytes_per_layer": {"forward_c": remote * 32, "reverse_bbar": remote * 320},
        }
        sy.close()
    pot.close()
    return out


def run_serve(args):
    """Continuous-batching serving: Poisson arrivals of mixed water / Cu structures, T = 3, BF16 networks.

    Request mix: 50/50 water (16..2048 molecules) / fcc Cu (3..20 cells per
    side), log-uniform sizes, per-request jitter.  Baseline: the same requests
    served one at a time in FP32 (build, evaluate, read back), which also sets
    the arrival rate of the main stream (70 % of that capacity).  Latency is
    completion minus arrival, completion = results back on the host.
    """
    import math

    from paper_2505_06711_gb300 import Potential, binding
    from paper_2505_06711_gb300.serving import (Server, latency_stats, make_requests, make_templates, serve_alone,
                                                serve_stream)
    from synth import make_model

    spec = make_model(T=3, seed=1234)
    templates = make_templates(seed=0)
    pot = Potential(spec)
    serve_alone(pot, make_requests(templates, 16, math.inf, seed=100))  # warm-up
    n_alone = max(64, min(1000, args.serve_requests // 10))
    alone_reqs = make_requests(templates, n_alone, math.inf, seed=101)
    _, st = serve_alone(pot, alone_reqs)
    pot.close()
    alone_rps = n_alone / st["wall_s"]
    alone_atoms = sum(r.n_atoms for r in alone_reqs) / st["wall_s"]
    pool = {"max_atoms": 1 << 17, "max_ghosts": 1 << 18, "max_structures": 256, "stride": 160}
    reqs = make_requests(templates, args.serve_requests, 0.7 * alone_rps, seed=103)
    # the same main stream on a pool with FP32 networks (faster than BF16 ones after their rework)
    server = Server(spec, pool["max_atoms"], pool["max_ghosts"], pool["max_structures"], pool["stride"],
                    precision=binding.REANN_MLP_FP32)
    try:
        serve_stream(server, make_requests(templates, 64, alone_rps, seed=102))  # warm-up, graph capture
        res, st = serve_stream(server, reqs)
        main_fp32 = {"load": 0.7, "rate_per_s": 0.7 * alone_rps, "requests": len(reqs), **latency_stats(res),
                     **st}
    finally:
        server.close()
    server = Server(spec, pool["max_atoms"], pool["max_ghosts"], pool["max_structures"], pool["stride"],
                    precision=binding.REANN_MLP_BF16)
    try:
        serve_stream(server, make_requests(templates, 64, alone_rps, seed=102))  # warm-up, graph capture
        res, st = serve_stream(server, reqs)
        main = {"load": 0.7, "rate_per_s": 0.7 * alone_rps, "requests": len(reqs), **latency_stats(res), **st}
        sweep = []
        n_sweep = max(200, args.serve_requests // 5)
        for load in (1.0, 2.0, 4.0, math.inf):
            rq = make_requests(templates, n_sweep, load * alone_rps, seed=104)
            r, t = serve_stream(server, rq)
            sweep.append({"load": load if math.isfinite(load) else "all at t=0", "requests": n_sweep,
                          **latency_stats(r), **t})
    finally:
        server.close()
    saturated = sweep[-1]["atom_evals_per_s"]
    return {
        "workload": "Poisson arrivals; 50/50 water 16..2048 molecules / Cu fcc 3..20 cells, log-uniform sizes, "
                    "jitter N(0, 0.02 A); T = 3; pooled launches with BF16 atomic networks (main and sweep), "
                    "the main stream also with FP32 ones",
        "pool": pool,
        "alone_fp32": {"requests": n_alone, "requests_per_s": alone_rps, "atom_evals_per_s": alone_atoms},
        "main": main,
        "main_fp32_networks": main_fp32,
        "sweep": sweep,
        "saturated_over_alone_atom_evals": saturated / alone_atoms,
    }


NET_PRECISIONS = (("fp32", 0), ("bf16_mlp", 1), ("fp8_mlp", 3))  # REANN_MLP_FP32, _BF16, _FP8


def run_t_scaling(args, steps: int = 10):
    """1,048,576-atom fcc Cu (64^3 cells), same step at T = 3 and T = 5: cost linear in T (Sec. 2.2);
    FP32 networks, then BF16 and FP8 E4M3 network GEMMs (FP32 accumulation).  Their errors against
    the FP64 oracle on the 4,000-atom Cu box are measured by the tests (test_gpu_bf16, test_gpu_fp8)."""
    import torch

    from paper_2505_06711_gb300 import Potential, binding
    from synth import fcc_box, make_model

    s = fcc_box(64, seed=0)
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    out = {"workload": f"fcc Cu 64^3 cells ({s.n_atoms} atoms), skin {SKIN} A, step = rebuild + energy/forces"}
    for T in (3, 5):
        pot = Potential(make_model(T=T))
        sy = pot.system(s.pos, s.species, s.cell, skin=SKIN)
        ctx, nl = pot.ctx, sy.nl
        res = {}
        for name, prec in NET_PRECISIONS:
            binding.reann_ctx_set_mlp_precision(ctx, prec)

            def step():
                binding.reann_nlist_rebuild(ctx, nl, sy.pos)
                binding.reann_energy_forces(ctx, nl, sy.pos, T, sy.energy, sy.forces, None)

            step()
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
            for a, b in ev:
                flush.zero_()
                a.record()
                step()
                b.record()
            torch.cuda.synchronize()
            binding.reann_ctx_check(ctx)
            ms = sum(a.elapsed_time(b) for a, b in ev) / steps
            res[name] = {"ms_per_step": ms, "atom_evals_per_s": s.n_atoms / (ms * 1e-3)}
        binding.reann_ctx_profile(ctx, True)
        step()
        prof = binding.reann_ctx_profile_read(ctx)
        binding.reann_ctx_profile(ctx, False)
        res["rebuild_ms"] = prof["nlist_rebuild"][0]
        out[f"T{T}"] = res
        sy.close()
        pot.close()
    for name, _ in NET_PRECISIONS:
        t3 = out["T3"][name]["ms_per_step"] - out["T3"]["rebuild_ms"]
        t5 = out["T5"][name]["ms_per_step"] - out["T5"]["rebuild_ms"]
        out[f"{name}_eval_cost_ratio_T5_over_T3"] = t5 / t3
    out["ideal_ratio"] = 5.0 / 3.0
    return out


def run_md(structure, pot, args, dt_fs: float = 0.5, temperature_k: float = 300.0):
    """NVE velocity Verlet on the same box (Maxwell-Boltzmann start): drift and atom-steps/s.

    A first call of the same length captures the step graph and equilibrates
    briefly; the second call is timed (CUDA events on the context stream) and
    its energies give the drift (slope of a linear fit of E_tot/N vs time).
    """
    import numpy as np
    import torch

    from synth import MASS_AMU, maxwell_boltzmann

    n = structure.n_atoms
    sy = pot.system(structure.pos, structure.species, structure.cell, skin=SKIN)
    m = MASS_AMU[structure.species]
    vel = torch.as_tensor(maxwell_boltzmann(m, temperature_k, seed=0), device="cuda").contiguous()
    mass = torch.as_tensor(m, device="cuda").contiguous()
    k = args.md_steps
    sy.md(vel, mass, dt_fs, k)  # capture + first stretch
    _, r0 = sy.md_info()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record()
    e_pot, e_kin = sy.md(vel, mass, dt_fs, k)
    b.record()
    torch.cuda.synchronize()
    sy.check()
    steps, r1 = sy.md_info()
    ms = a.elapsed_time(b)
    etot = ((e_pot + e_kin) / n).cpu().numpy()
    t_ps = np.arange(1, k + 1) * dt_fs * 1e-3
    slope = float(np.polyfit(t_ps, etot, 1)[0])
    out = {
        "workload": f"NVE velocity Verlet, {n}-atom water box, dt {dt_fs} fs, {k} timed steps after {k} untimed, "
                    f"Maxwell-Boltzmann {temperature_k:.0f} K start, FP64 integrator, FP32 networks",
        "atom_steps_per_s": n * k / (ms * 1e-3),
        "ms_per_step": ms / k,
        "drift_meV_per_atom_per_ps": slope * 1e3,
        "etot_std_meV_per_atom": float(etot.std() * 1e3),
        "rebuilds_timed": r1 - r0,
        "steps": steps,
        "temperature_end_K": float(2 * e_kin[-1].item() / (3 * n - 3) / 8.617333262e-5),
    }
    sy.close()
    return out


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(x: float, dist=None, device="cpu") -> float:
    """Largest value of x over all ranks (identity without a process group)."""
    if dist is None:
        return float(x)
    import torch

    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate(n_atoms_per_rank: int, ms_per_step: float, ws: int) -> float:
    """Whole-job atom-evaluations per second: every rank evaluates its own replica."""
    return ws * n_atoms_per_rank / (ms_per_step * 1e-3)


class ClockSampler:
    """nvidia-smi clock/throttle samples every 200 ms while the timed region runs."""

    FIELDS = (
        "index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
        "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
        "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap"
    )

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL,
            )
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "", 1).isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "", 1).isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower().startswith("active")})
        return {
            "sm_mhz": statistics.median(sm) if sm else None,
            "sm_max_mhz": max(mx) if mx else None,
            "reasons": reasons,
            "samples": len(rows),
        }


def source_sha(name: str) -> str:
    """sha1[:12] of a kernel source's code: line comments and blank lines do not count."""
    path = os.path.join(ROOT, "paper_2505_06711_gb300", "csrc", name)
    code = []
    for line in open(path, encoding="utf-8").read().splitlines():
        line = line.split("//", 1)[0].rstrip()
        if line:
            code.append(line)
    return hashlib.sha1("\n".join(code).encode()).hexdigest()[:12]


REGION_SOURCE = {
    "density_fwd": "density.cu", "density_adj": "density.cu", "bbar": "density.cu", "mlp_fwd": "mlp_fp32.cu",
    "mlp_bwd": "mlp_fp32.cu", "nlist_rebuild": "nlist.cu", "live_edges": "nlist.cu",
}


def region_flops(region: str, n_atoms: int, n_live: int, T: int, launches: int) -> float | None:
    """Algorithmic FLOPs of all launches of one region in one step."""
    if region == "density_fwd":
        return T * (n_live * FLOP_PER_LIVE_EDGE_FWD + n_atoms * FLOP_PER_ATOM_FWD)
    if region == "density_adj":
        return T * n_live * FLOP_PER_LIVE_EDGE_ADJ + (T - 1) * n_live * FLOP_PER_LIVE_EDGE_ADJ_CBAR
    if region == "mlp_fwd":
        return n_atoms * ((T - 1) * FLOP_PER_ATOM_MLP_FWD[8] + FLOP_PER_ATOM_MLP_FWD[1])
    if region == "mlp_bwd":  # the FP32 backward networks also take the bbar step
        return n_atoms * ((T - 1) * FLOP_PER_ATOM_MLP_BWD[8] + FLOP_PER_ATOM_MLP_BWD[1] + T * FLOP_PER_ATOM_BBAR)
    if region == "bbar":
        return T * n_atoms * FLOP_PER_ATOM_BBAR
    return None


def region_flops_coarse(region: str, n_atoms: int, n_live: int, T: int) -> float | None:
    """The same, with the scope table's coarse per-edge counts."""
    if region == "density_fwd":
        return T * (n_live * FLOP_PER_LIVE_EDGE_FWD_COARSE + n_atoms * FLOP_PER_ATOM_CONTRACTION_COARSE)
    if region == "density_adj":
        return T * n_live * FLOP_PER_LIVE_EDGE_ADJ_COARSE
    return None


def region_bytes(region: str, n_atoms: int, n_pairs: int, T: int) -> float | None:
    """Algorithmic HBM bytes of all launches of an edge region in one step."""
    fixed = BYTES_PER_ATOM_EDGE_FIXED.get(region)
    if fixed is None:
        return None
    return T * (4.0 * n_pairs + n_atoms * fixed)


def measured_peaks() -> tuple[float, str]:
    """HBM copy bandwidth (GB/s) from the machine's measured peaks, else the fallback figure."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def launches_per_step(T: int) -> int:
    """Library kernel launches per step (single-domain list, any network precision):
    rebuild 13 (sort-or-keep gate; wrap + keys + histogram, 3 sort kernels (scan,
    scatter, rank) and the gather, which return at once on rebuilds that keep the
    atom order; the keep-order wrap; ghost-count scan; ghosts + extended keys +
    histogram, 3 sort kernels, search), evaluation 2 (positions with c0, live
    edges) + 2T forward (density, network; the energy network also sums its
    tiles) + 1 (total energy) + 2T reverse (network with bbar, density adjoint;
    the last one writes forces and atomic energies)."""
    return 13 + 2 + 2 * T + 1 + 2 * T


def cpu_baseline(structure, spec):
    import oracle

    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    times = []
    t_start = time.perf_counter()
    while len(times) < 4 and (time.perf_counter() - t_start) < 10.0:
        t0 = time.perf_counter()
        oracle.energy_forces(spec, structure.pos, structure.species, structure.cell, n_threads=cores)
        times.append(time.perf_counter() - t0)
    t = statistics.mean(times)
    # the same oracle on the small boxes: all cores and one core, and its brute-force list alone
    from synth import fcc_box, water_box

    detail = {}
    for name, sbox in (("water_192", water_box(64, seed=0)), ("cu_4000", fcc_box(10, seed=0))):
        for label, nt in (("all_cores", cores), ("1_core", 1)):
            t0 = time.perf_counter()
            oracle.energy_forces(spec, sbox.pos, sbox.species, sbox.cell, n_threads=nt)
            detail[f"{name}_{label}_atom_evals_per_s"] = sbox.n_atoms / (time.perf_counter() - t0)
        t0 = time.perf_counter()
        oracle.neighbors(sbox.pos, sbox.cell, spec.r_c + SKIN, n_threads=cores)
        detail[f"{name}_list_only_ms"] = (time.perf_counter() - t0) * 1e3
    return {
        "value": structure.n_atoms / t,
        "unit": "atom-evals/s",
        "cores": cores,
        "kind": "oracle",
        "sample": f"{len(times)} full FP64 evaluations (brute-force list + forward + reverse) of the "
                  f"{structure.n_atoms}-atom water box, mean {t:.2f} s each",
        "detail": detail,
    }


def base_line(args, ws, value, ms, dtype):
    return {
        "metric": "energy+force atom-evals/s at T=3",
        "value": value,
        "unit": "atom-evals/s",
        "n_gpus": ws,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": dtype,
        "data": "synthetic (seeded water box, seeded random-weight REANN model)",
        "config": {
            "workload": f"water box {N_MOLECULES} H2O ({3 * N_MOLECULES} atoms), 1.0 g/cm^3, T={T_LAYERS}, "
                        f"r_c=5 A, skin={SKIN} A, 8 Gaussians, L=2, 16 orbitals, networks 48-64-64 SiLU",
            "atoms_per_gpu": 3 * N_MOLECULES,
            "step": "device neighbour-list rebuild + energy/forces (forward T layers + reverse)",
            "cache": "L2 flushed (256 MiB write) before every timed step",
            "parallelism": f"replicas x{ws}",
        },
    }


REFERENCE_BUDGET_S = 120.0


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle
    from synth import make_model, water_box

    s = water_box(N_MOLECULES, seed=0)
    spec = make_model(T=T_LAYERS)
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    # one evaluation of the box takes seconds: the run is bounded in time (at most one warm-up
    # evaluation, timed evaluations until REFERENCE_BUDGET_S has passed, at least 3), so that
    # any --steps / --warmup ends within a few minutes; the line states how many were timed
    for _ in range(min(args.warmup, 1)):
        oracle.energy_forces(spec, s.pos, s.species, s.cell, n_threads=cores)
    times = []
    t_start = time.perf_counter()
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.energy_forces(spec, s.pos, s.species, s.cell, n_threads=cores)
        times.append(time.perf_counter() - t0)
        if len(times) >= 3 and time.perf_counter() - t_start > REFERENCE_BUDGET_S:
            break
    t = statistics.mean(times)
    value = s.n_atoms / t
    line = base_line(args, 1, value, t * 1e3, "f64")
    line["impl"] = "reference"
    line["config"]["step"] = "one FP64 oracle evaluation (brute-force list + forward + reverse) on the host cores"
    line["config"]["cache"] = "host CPU run (no GPU cache to flush)"
    line["cpu_baseline"] = {"value": value, "unit": "atom-evals/s", "cores": cores, "kind": "oracle",
                            "sample": f"full {s.n_atoms}-atom box per step; {len(times)} of the {args.steps} "
                                      f"requested steps timed (the run is bounded at {REFERENCE_BUDGET_S:.0f} s)"}
    line["e2e"] = {"value": value, "unit": "atom-evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    print(json.dumps(line), flush=True)


def run_ours(args):
    import numpy as np
    import torch

    from paper_2505_06711_gb300 import Potential, binding
    from synth import make_model, water_box

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    s = water_box(N_MOLECULES, seed=0)
    spec = make_model(T=T_LAYERS)
    pot = Potential(spec)
    sy = pot.system(s.pos, s.species, s.cell, skin=SKIN)
    ctx, nl = pot.ctx, sy.nl
    pos = sy.pos
    energy = torch.zeros(1, dtype=torch.float64, device="cuda")
    forces = torch.zeros((s.n_atoms, 3), dtype=torch.float32, device="cuda")
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()

    def step():
        binding.reann_nlist_rebuild(ctx, nl, pos)
        binding.reann_energy_forces(ctx, nl, pos, T_LAYERS, energy, forces, None)

    for _ in range(args.warmup):
        flush.zero_()
        step()
    torch.cuda.synchronize()
    binding.reann_ctx_check(ctx)
    n_atoms, n_ghosts, n_pairs, n_live = binding.reann_nlist_info(nl)

    def timed(profile: bool):
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        binding.reann_ctx_profile(ctx, profile)
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for k in range(args.steps):
            flush.zero_()
            ev[k][0].record(stream)
            step()
            ev[k][1].record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        if dist:
            dist.barrier()
        prof = binding.reann_ctx_profile_read(ctx)
        binding.reann_ctx_profile(ctx, False)
        binding.reann_ctx_check(ctx)
        return sum(a.elapsed_time(b) for a, b in ev) / args.steps, wall, prof

    # pass 1: the reported step time (no per-region events); pass 2: per-region events for the roofline
    clocks = ClockSampler(local)
    clocks.start()
    ms, wall, _ = timed(False)
    ms_prof, _, prof = timed(True)
    ms = max_over_ranks(ms, dist, "cuda")
    value = aggregate(n_atoms, ms, ws)

    breakdown = {k: round(v[0] / args.steps, 5) for k, v in prof.items() if v[1]}

    # end to end through the C ABI with host buffers
    e2e = None
    if not args.no_e2e:
        h_pos = torch.from_numpy(np.ascontiguousarray(s.pos)).pin_memory()
        h_en = torch.zeros(1, dtype=torch.float64).pin_memory()
        h_f = torch.zeros((s.n_atoms, 3), dtype=torch.float32).pin_memory()
        for _ in range(args.warmup):
            binding.reann_energy_forces_host(ctx, nl, h_pos, T_LAYERS, h_en, h_f, 1)
        tt = []
        for _ in range(args.steps):
            flush.zero_()
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            binding.reann_energy_forces_host(ctx, nl, h_pos, T_LAYERS, h_en, h_f, 1)
            tt.append(time.perf_counter() - t1)
        e_ms = statistics.mean(tt) * 1e3
        e_ms = max_over_ranks(e_ms, dist, "cuda")
        e2e = {
            "value": aggregate(n_atoms, e_ms, ws),
            "unit": "atom-evals/s",
            "ms_per_step": e_ms,
            "ms_per_step_median": statistics.median(tt) * 1e3,
            "h2d_bytes_per_step": int(h_pos.numel() * 8),
            "d2h_bytes_per_step": int(h_f.numel() * 4 + 8),
        }

    # the same step with the atomic networks on tcgen05 tensor cores
    variants = {"fp32": {"value": value, "ms_per_step": ms, "mlp_ms_per_step": breakdown.get("mlp_fwd", 0.0)
                         + breakdown.get("mlp_bwd", 0.0)}}
    for name, prec in (("bf16_mlp", binding.REANN_MLP_BF16), ("bf16x3_mlp", binding.REANN_MLP_BF16X3),
                       ("fp8_mlp", binding.REANN_MLP_FP8)):
        binding.reann_ctx_set_mlp_precision(ctx, prec)
        for _ in range(args.warmup):
            step()
        v_ms, _, _ = timed(False)
        _, _, v_prof = timed(True)
        v_ms = max_over_ranks(v_ms, dist, "cuda")
        variants[name] = {
            "value": aggregate(n_atoms, v_ms, ws),
            "ms_per_step": v_ms,
            "mlp_ms_per_step": (v_prof["mlp_fwd"][0] + v_prof["mlp_bwd"][0]) / args.steps,
        }
    binding.reann_ctx_set_mlp_precision(ctx, binding.REANN_MLP_FP32)

    # the sampler ran through both timed passes, the end-to-end calls and the variants
    clk = clocks.stop()
    # roofline of the dominant region
    dom = max(prof.items(), key=lambda kv: kv[1][0])
    region, (tot_ms, nl_launch) = dom
    per_step_ms = tot_ms / args.steps
    launches = nl_launch / args.steps
    flops = region_flops(region, n_atoms, n_live, T_LAYERS, launches)
    props = torch.cuda.get_device_properties(local)
    max_mhz = (clk or {}).get("sm_max_mhz") or 2070.0
    peak_tflops = props.multi_processor_count * 128 * 2 * max_mhz * 1e6 / 1e12
    roof = None
    if flops is not None and launches > 0:
        launch_s = per_step_ms / launches * 1e-3
        achieved = flops / launches / launch_s / 1e12
        key = (region, source_sha(REGION_SOURCE.get(region, "density.cu")))
        hbm_gbs, hbm_src = measured_peaks()
        coarse = region_flops_coarse(region, n_atoms, n_live, T_LAYERS)
        nbytes = region_bytes(region, n_atoms, n_pairs, T_LAYERS)
        roof = {
            "bound": "alu",
            "kernel": region,
            "achieved": achieved,
            "peak": peak_tflops,
            "unit": "TFLOP/s",
            "frac": achieved / peak_tflops,
            "traffic": TRAFFIC.get(key),
            "peak_source": f"derived: {props.multi_processor_count} SMs x 128 FP32 lanes x 2 FLOP x {max_mhz:.0f} MHz",
            "flop_count": "per live edge as the kernels' formulas need them (DESIGN section 6)",
            "frac_alu_survey": (coarse / launches / launch_s / 1e12 / peak_tflops) if coarse else None,
            "flop_count_survey": "scope table: 130 per live edge forward + 2560 per atom contraction, 260 reverse",
            "achieved_hbm_gbs": (nbytes / launches / launch_s / 1e9) if nbytes else None,
            "frac_hbm": (nbytes / launches / launch_s / 1e9 / hbm_gbs) if nbytes else None,
            "hbm_peak_gbs": hbm_gbs,
            "hbm_peak_source": f"{hbm_src} copy bandwidth",
            "frac_l2": L2_FRAC.get(key),
            "launches_per_step": launches,
            "mean_launch_ms": per_step_ms / launches,
            "timed_in": "second timed pass of the same steps with per-region CUDA events on the library stream",
            "ms_per_step_with_events": ms_prof,
        }

    md = None if args.no_md else run_md(s, pot, args)
    t_scaling = None if args.no_t_scaling else run_t_scaling(args)
    serve = None if args.no_serve or ws > 1 else run_serve(args)
    decomp = None if args.no_decomp else run_decomp(args)
    hea = None if args.no_hea else run_hea(args)
    pairs = None if args.no_pairs else run_pairs(args)

    if rank == 0:
        line = base_line(args, ws, value, ms, "f32")
        line["variants"] = variants
        line["md"] = md
        line["t_scaling_cu_1m"] = t_scaling
        line["serve"] = serve
        line["decomposition"] = decomp
        line["hea"] = hea
        line["pair_features"] = pairs
        line["e2e"] = e2e
        line["roofline"] = roof
        line["gpu_launches"] = launches_per_step(T_LAYERS) * args.steps
        line["clocks"] = clk
        line["wall_s_timed_region"] = wall
        line["breakdown_ms_per_step"] = breakdown
        line["structure"] = {"atoms": n_atoms, "ghosts": n_ghosts, "pairs_rc_skin": n_pairs, "pairs_rc": n_live}
        line["energy_eV"] = float(energy.item())
        if not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(s, spec)
        print(json.dumps(line), flush=True)
    sy.close()
    pot.close()
    if dist:
        dist.destroy_process_group()


def main():
    args = parse()
    from paper_2505_06711_gb300 import build

    build.build()  # no-op when up to date
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
