"""Continuous-batching energy/force serving on top of the reann_serve_* ABI.

Requests (periodic structures) arrive over time.  Builder threads admit
arrived requests whose footprint fits the resident pool (owned atoms, ghost
slots, structure slots) -- each neighbour list is built on a builder's own
context and stream while the previous pool launch is still on the GPU -- and
the serving thread launches one evaluation for everything admitted since the
last launch as soon as no launch is outstanding, returns results as launches
complete and releases their pool space for requests still waiting.  Latency
is completion minus arrival.
"""

from __future__ import annotations

import collections
import dataclasses
import gc
import math
import threading
import time

import numpy as np

from . import Potential, binding


@dataclasses.dataclass
class Request:
    arrival: float  # s since the start of the stream
    base: np.ndarray  # (n, 3) float64 template positions (shared, not copied)
    species: np.ndarray  # (n,) int32
    cell: np.ndarray  # (3, 3)
    jitter: np.ndarray | None = None  # (n, 3) displacement added at submission (a view into a shared bank)

    @property
    def pos(self) -> np.ndarray:
        return self.base if self.jitter is None else self.base + self.jitter

    @property
    def n_atoms(self) -> int:
        return len(self.base)


@dataclasses.dataclass
class Result:
    energy: float
    forces: np.ndarray
    latency: float


class Server:
    """A resident pool on one GPU plus the contexts that feed it.

    ``builders`` contexts, each on its own stream, build submissions
    concurrently (one per thread); the evaluation context owns the pool.
    """

    def __init__(self, spec, max_atoms: int, max_ghosts: int, max_structures: int, stride: int = 160,
                 precision: int = binding.REANN_MLP_FP32, skin: float = 1.0, builders: int = 4):
        import torch

        self.max_atoms, self.max_structures, self.skin = max_atoms, max_structures, skin
        self.eval = Potential(spec, precision=precision)
        self.build_streams = [torch.cuda.Stream() for _ in range(builders)]
        self.builds = [Potential(spec, stream=st) for st in self.build_streams]
        self.srv = binding.reann_serve_create(self.eval.ctx, max_atoms, max_ghosts, max_structures, stride)
        self.energies = torch.zeros(max_structures, dtype=torch.float64, device="cuda")
        self.forces = torch.zeros((max_atoms + 1, 3), dtype=torch.float32, device="cuda")

    def submit(self, req: Request, builder: int = 0):
        """Slot of the admitted request, or None when the pool has no room for it now."""
        import torch

        st = self.build_streams[builder]
        with torch.cuda.stream(st):
            pos = torch.as_tensor(req.pos, device="cuda").contiguous()
            sp = torch.as_tensor(req.species, device="cuda").contiguous()
        st.synchronize()
        return binding.reann_serve_submit(self.srv, self.eval.ctx, self.builds[builder].ctx, pos, sp, req.cell,
                                          self.skin)

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

    def free_slots(self) -> int:
        return binding.reann_serve_usage(self.srv)[2]

    def close(self) -> None:
        if getattr(self, "srv", None) is not None:
            import torch

            torch.cuda.synchronize()
            binding.reann_serve_free(self.srv)
            self.srv = None
        self.eval.close()
        for b in self.builds:
            b.close()


def serve_stream(server: Server, requests: list[Request]):
    """Continuous batching over a timed request stream; returns (results by request index, stats).

    Builder threads (one per build context) take arrived requests and submit
    them, so neighbour-list builds run concurrently and overlap the launch in
    flight; the calling thread starts a launch of everything admitted whenever
    none is in flight and hands results back as launches complete.  A refused
    admission (pool full) parks the builders until the next release.
    """
    n = len(requests)
    results: list[Result | None] = [None] * n
    cv = threading.Condition()
    waiting = collections.deque()  # arrived, not yet admitted
    admitted: dict[int, int] = {}  # slot -> request index, not yet launched
    # full: a submission refused since the last release (builders park until the next one);
    # epoch counts release rounds so that a refusal older than a release is simply retried
    st = {"full": False, "stop": False, "error": None, "epoch": 0}

    def builder(b: int) -> None:
        while True:
            with cv:
                while not st["stop"] and (not waiting or st["full"]):
                    cv.wait()
                if st["stop"]:
                    return
                k = waiting.popleft()
                epoch = st["epoch"]
            try:
                slot = server.submit(requests[k], b)
            except Exception as exc:  # surfaced by the calling thread
                with cv:
                    st["error"], st["stop"] = exc, True
                    cv.notify_all()
                return
            with cv:
                if slot is None:
                    waiting.appendleft(k)
                    if st["epoch"] == epoch:
                        st["full"] = True
                else:
                    admitted[slot] = k
                cv.notify_all()

    threads = [threading.Thread(target=builder, args=(b,), daemon=True) for b in range(len(server.builds))]
    # the cyclic garbage collector stays off while requests are in flight (a full pass over
    # the stream's result arrays stalls every thread for tens of milliseconds)
    gc_was_enabled = gc.isenabled()
    gc.disable()
    for t in threads:
        t.start()
    in_flight = None  # (slots, event, {slot: request index})
    nxt = 0
    done_count = 0
    launches = 0
    batch = []
    t0 = time.perf_counter()
    try:
        while done_count < n:
            busy = False
            now = time.perf_counter() - t0
            if nxt < n and requests[nxt].arrival <= now:
                with cv:
                    while nxt < n and requests[nxt].arrival <= now:
                        waiting.append(nxt)
                        nxt += 1
                    cv.notify_all()
            if st["error"] is not None:
                raise st["error"]
            if in_flight is not None and in_flight[1].query():
                slots, _, owners = in_flight
                got = server.collect(slots)
                done = time.perf_counter() - t0
                for s, (e, f) in got.items():
                    k = owners[s]
                    results[k] = Result(e, f, done - requests[k].arrival)
                    server.release(s)
                done_count += len(slots)
                in_flight = None
                busy = True
                with cv:
                    st["full"] = False
                    st["epoch"] += 1
                    cv.notify_all()
            if in_flight is None:
                with cv:
                    pending = bool(admitted)
                if pending:
                    slots, ev = server.launch()
                    owners = {}
                    with cv:
                        for s in slots:  # a builder may still be recording a slot it just admitted
                            cv.wait_for(lambda: s in admitted)
                            owners[s] = admitted.pop(s)
                    in_flight = (slots, ev, owners)
                    launches += 1
                    batch.append(len(slots))
                    busy = True
                else:
                    with cv:
                        refused = st["full"] and not admitted
                    if refused and server.free_slots() == server.max_structures:
                        raise RuntimeError("a request does not fit even the empty pool")
            if not busy:
                time.sleep(20e-6)
    finally:
        with cv:
            st["stop"] = True
            cv.notify_all()
        for t in threads:
            t.join()
        if gc_was_enabled:
            gc.enable()
    wall = time.perf_counter() - t0
    atoms = sum(r.n_atoms for r in requests)
    return results, {"wall_s": wall, "launches": launches, "mean_batch": float(np.mean(batch)) if batch else 0.0,
                     "atoms": atoms, "atom_evals_per_s": atoms / wall}


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


def make_requests(templates, n: int, rate_per_s: float, seed: int = 0, jitter: float = 0.02,
                  bank_values: int = 3 << 20) -> list[Request]:
    """Poisson arrivals; 50/50 water/Cu; sizes log-uniform; per-request jitter.

    Templates are geometrically spaced in size, so a uniformly drawn index is a
    log-uniform size.  Each request's displacement is a window, at its own
    random offset, of one seeded bank of N(0, jitter) values: every request gets
    different positions without holding thousands of full copies in memory.
    A rate of ``math.inf`` puts every arrival at time zero.
    """
    rng = np.random.default_rng(seed)
    water = [t for t in templates if t.name.startswith("water")]
    cu = [t for t in templates if t.name.startswith("fcc")]
    largest = max(len(t.pos) for t in templates)
    bank = rng.normal(0.0, jitter, size=max(bank_values, 6 * largest))
    t = 0.0
    reqs = []
    for _ in range(n):
        if math.isfinite(rate_per_s):
            t += rng.exponential(1.0 / rate_per_s)
        group = water if rng.random() < 0.5 else cu
        s = group[rng.integers(len(group))]
        k = 3 * len(s.pos)
        off = int(rng.integers(0, len(bank) - k + 1))
        reqs.append(Request(t, s.pos, s.species, s.cell, bank[off : off + k].reshape(-1, 3)))
    return reqs


def latency_stats(results) -> dict:
    lat = np.array([r.latency for r in results]) * 1e3
    return {"p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "mean_ms": float(lat.mean()), "max_ms": float(lat.max())}


def capacity_alone(pot: Potential, templates, n: int = 64, seed: int = 1) -> tuple[float, float]:
    """(requests/s, atom-evals/s) of one-at-a-time serving with no arrival gaps."""
    reqs = make_requests(templates, n, rate_per_s=math.inf, seed=seed)
    _, st = serve_alone(pot, reqs)
    return n / st["wall_s"], sum(r.n_atoms for r in reqs) / st["wall_s"]
