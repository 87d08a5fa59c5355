"""Continuous-batching energy/force serving on top of the reann_serve_* ABI.

Requests (periodic structures) arrive over time.  The loop admits every
arrived request whose footprint fits the resident pool (owned atoms, ghost
slots, structure slots) -- its neighbour list is built on a second context and
stream while the previous pool launch is still on the GPU -- launches one
evaluation for everything admitted since the last launch as soon as no launch
is outstanding, and returns results as launches complete, releasing their
pool space for requests still waiting.  Latency is completion minus arrival.
"""

from __future__ import annotations

import collections
import dataclasses
import math
import time

import numpy as np

from . import Potential, binding


@dataclasses.dataclass
class Request:
    arrival: float  # s since the start of the stream
    pos: np.ndarray  # (n, 3) float64
    species: np.ndarray  # (n,) int32
    cell: np.ndarray  # (3, 3)


@dataclasses.dataclass
class Result:
    energy: float
    forces: np.ndarray
    latency: float


class Server:
    """A resident pool on one GPU plus the contexts that feed it."""

    def __init__(self, spec, max_atoms: int, max_ghosts: int, max_structures: int, stride: int = 160,
                 precision: int = binding.REANN_MLP_BF16, skin: float = 1.0):
        import torch

        self.max_atoms, self.max_structures, self.skin = max_atoms, max_structures, skin
        self.eval = Potential(spec, precision=precision)
        self.build_stream = torch.cuda.Stream()
        self.build = Potential(spec, stream=self.build_stream)
        self.srv = binding.reann_serve_create(self.eval.ctx, max_atoms, max_ghosts, max_structures, stride)
        self.energies = torch.zeros(max_structures, dtype=torch.float64, device="cuda")
        self.forces = torch.zeros((max_atoms + 1, 3), dtype=torch.float32, device="cuda")

    def submit(self, req: Request):
        import torch

        with torch.cuda.stream(self.build_stream):
            pos = torch.as_tensor(req.pos, device="cuda").contiguous()
            sp = torch.as_tensor(req.species, device="cuda").contiguous()
        self.build_stream.synchronize()
        return binding.reann_serve_submit(self.srv, self.eval.ctx, self.build.ctx, pos, sp, req.cell, self.skin)

    def launch(self):
        import torch

        slots = binding.reann_serve_launch(self.srv, self.eval.ctx, self.energies, self.forces, self.max_structures)
        ev = torch.cuda.Event()
        ev.record()
        return slots, ev

    def collect(self, slots):
        """Host copies of the launched slots' results: {slot: (energy, forces)}."""
        e = self.energies.cpu().numpy()
        out = {}
        for s in slots:
            off, n = binding.reann_serve_slot(self.srv, s)
            out[s] = (float(e[s]), self.forces[off : off + n].cpu().numpy())
        return out

    def release(self, slot: int) -> None:
        binding.reann_serve_release(self.srv, self.eval.ctx, slot)

    def close(self) -> None:
        if getattr(self, "srv", None) is not None:
            import torch

            torch.cuda.synchronize()
            binding.reann_serve_free(self.srv)
            self.srv = None
        self.eval.close()
        self.build.close()


def serve_stream(server: Server, requests: list[Request]):
    """Continuous batching over a timed request stream; returns (results by request index, stats)."""
    n = len(requests)
    results: list[Result | None] = [None] * n
    waiting = collections.deque()
    admitted: dict[int, int] = {}  # slot -> request index, not yet launched
    in_flight = None  # (slots, event, {slot: request index})
    nxt = 0
    launches = 0
    t0 = time.perf_counter()
    while True:
        now = time.perf_counter() - t0
        while nxt < n and requests[nxt].arrival <= now:
            waiting.append(nxt)
            nxt += 1
        while waiting:
            slot = server.submit(requests[waiting[0]])
            if slot is None:
                break  # pool full: wait for releases
            admitted[slot] = waiting.popleft()
        if in_flight is not None and in_flight[1].query():
            slots, _, owners = in_flight
            done = time.perf_counter() - t0
            for s, (e, f) in server.collect(slots).items():
                k = owners[s]
                results[k] = Result(e, f, done - requests[k].arrival)
                server.release(s)
            in_flight = None
        if in_flight is None and admitted:
            slots, ev = server.launch()
            in_flight = (slots, ev, {s: admitted.pop(s) for s in slots})
            launches += 1
            continue
        if nxt >= n and not waiting and not admitted and in_flight is None:
            break
        if in_flight is None and not waiting and nxt < n:
            time.sleep(max(0.0, min(requests[nxt].arrival - (time.perf_counter() - t0), 0.002)))
    wall = time.perf_counter() - t0
    return results, {"wall_s": wall, "launches": launches}


def serve_alone(pot: Potential, requests: list[Request], skin: float = 1.0):
    """Each request on its own (build, evaluate, read), one at a time, same arrival times."""
    import torch

    n = len(requests)
    results: list[Result | None] = [None] * n
    t0 = time.perf_counter()
    for k, req in enumerate(requests):
        now = time.perf_counter() - t0
        if req.arrival > now:
            time.sleep(req.arrival - now)
        sy = pot.system(req.pos, req.species, req.cell, skin=skin)
        sy.evaluate(atom_energy=False)
        torch.cuda.synchronize()
        e, f = float(sy.energy.item()), sy.forces.cpu().numpy()
        results[k] = Result(e, f, time.perf_counter() - t0 - req.arrival)
        sy.close()
    return results, {"wall_s": time.perf_counter() - t0}


def make_templates(n_water: int = 12, n_cu: int = 12, seed: int = 0):
    """Distinct periodic structures spanning the request sizes: water 16..2048 molecules, Cu 3..20 cells."""
    from synth import fcc_box, water_box

    waters = sorted({int(round(x)) for x in np.geomspace(16, 2048, n_water)})
    cus = sorted({int(round(x)) for x in np.geomspace(3, 20, n_cu)})
    return [water_box(m, seed=seed + m) for m in waters] + [fcc_box(k, seed=seed + k) for k in cus]


def make_requests(templates, n: int, rate_per_s: float, seed: int = 0, jitter: float = 0.02) -> list[Request]:
    """Poisson arrivals; 50/50 water/Cu; sizes log-uniform (template chosen by log-size); fresh jitter."""
    rng = np.random.default_rng(seed)
    water = [t for t in templates if t.name.startswith("water")]
    cu = [t for t in templates if t.name.startswith("fcc")]
    t = 0.0
    reqs = []
    for _ in range(n):
        t += rng.exponential(1.0 / rate_per_s)
        group = water if rng.random() < 0.5 else cu
        s = group[rng.integers(len(group))]  # templates are geometrically spaced: uniform index = log-uniform size
        pos = s.pos + rng.normal(0.0, jitter, size=s.pos.shape)
        reqs.append(Request(t, pos, s.species, s.cell))
    return reqs


def latency_stats(results) -> dict:
    lat = np.array([r.latency for r in results]) * 1e3
    return {"p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "mean_ms": float(lat.mean()), "max_ms": float(lat.max())}


def capacity_alone(pot: Potential, templates, n: int = 64, seed: int = 1) -> float:
    """Requests per second of one-at-a-time FP32 serving (no arrival gaps)."""
    reqs = make_requests(templates, n, rate_per_s=math.inf, seed=seed)
    for r in reqs:
        r.arrival = 0.0
    _, st = serve_alone(pot, reqs)
    return n / st["wall_s"]
