"""Continuous-batching pool (reann_serve_*): many structures evaluated by one pass.

Every structure keeps its own neighbour rows, network tiles and FP64 energy
segment inside the pool, so its forces are bitwise those of evaluating it on
its own (a System), in any mix and at any pool offset; energies differ from a
System's only by the order of the FP64 sum.
"""

from __future__ import annotations

import numpy as np
import pytest

import oracle
from gpu_helpers import assert_parity
from synth import fcc_box, make_model, water_box

pytestmark = pytest.mark.gpu

MIXED = ["water16", "water200", "fcc3", "fcc5"]


@pytest.fixture(scope="module")
def spec():
    return make_model(T=3, seed=1234)


@pytest.fixture(scope="module")
def structs():
    return {
        "water16": water_box(16, seed=3),
        "water200": water_box(200, seed=4),
        "fcc3": fcc_box(3, seed=5),
        "fcc5": fcc_box(5, seed=6),
    }


def _server(spec, precision, max_atoms=4096, max_ghosts=60000, max_structures=8, stride=160):
    from paper_2505_06711_gb300.serving import Server

    return Server(spec, max_atoms, max_ghosts, max_structures, stride=stride, precision=precision)


def _submit(srv, s):
    from paper_2505_06711_gb300.serving import Request

    return srv.submit(Request(0.0, s.pos, s.species, s.cell))


def _run(srv, names, structs):
    """Submit the named structures, launch once, return {name: (energy, forces, offset)}."""
    slots = {name: _submit(srv, structs[name]) for name in names}
    assert all(v is not None for v in slots.values())
    launched, _ = srv.launch()
    assert sorted(launched) == sorted(slots.values())
    res = srv.collect(launched)
    from paper_2505_06711_gb300 import binding

    out = {}
    for name, sl in slots.items():
        off, n = binding.reann_serve_slot(srv.srv, sl)
        assert n == len(structs[name].pos)
        out[name] = (res[sl][0], res[sl][1], off)
    return out, slots


def _system(spec, s, precision):
    import torch

    from paper_2505_06711_gb300 import Potential

    pot = Potential(spec, precision=precision)
    sy = pot.system(s.pos, s.species, s.cell)
    sy.evaluate(atom_energy=False)
    sy.check()
    torch.cuda.synchronize()
    e, f = float(sy.energy.item()), sy.forces.cpu().numpy()
    sy.close()
    pot.close()
    return e, f


@pytest.mark.parametrize("precision", [0, 1, 2], ids=["fp32", "bf16", "bf16x3"])
def test_pool_matches_system(spec, structs, precision):
    srv = _server(spec, precision)
    try:
        out, _ = _run(srv, MIXED, structs)
        for name in MIXED:
            e_ref, f_ref = _system(spec, structs[name], precision)
            e, f, off = out[name]
            n = len(f)
            print(f"[serve] {name} N={n} off={off} dE={e - e_ref:.3e} max|dF|={np.abs(f - f_ref).max():.3e}")
            assert np.array_equal(f, f_ref), f"{name}: pool forces differ from a System's"
            assert abs(e - e_ref) <= 1e-12 * max(1.0, abs(e_ref)), f"{name}: energy {e} vs {e_ref}"
    finally:
        srv.close()


def test_pool_fp32_vs_oracle(spec, structs):
    srv = _server(spec, 0)
    try:
        out, _ = _run(srv, ["water200", "fcc5"], structs)
        for name in ("water200", "fcc5"):
            s = structs[name]
            ref = oracle.energy_forces(spec, s.pos, s.species, s.cell)
            e, f, _ = out[name]
            assert_parity({"energy": e, "forces": f.astype(np.float64)}, ref, len(s.pos))
    finally:
        srv.close()


def test_mix_is_bitwise_alone(spec, structs):
    srv = _server(spec, 1)
    try:
        alone = {}
        for name in MIXED:
            o, slots = _run(srv, [name], structs)
            alone[name] = o[name]
            srv.release(slots[name])
        mixed, _ = _run(srv, list(reversed(MIXED)), structs)
        offsets = {name: mixed[name][2] for name in MIXED}
        assert len(set(offsets.values())) == len(MIXED)
        assert any(offsets[k] != alone[k][2] for k in MIXED), "the mix should move structures to new offsets"
        for name in MIXED:
            assert mixed[name][0] == alone[name][0], f"{name}: energy differs in the mix"
            assert np.array_equal(mixed[name][1], alone[name][1]), f"{name}: forces differ in the mix"
    finally:
        srv.close()


def test_lifecycle_retire_release_reuse(spec, structs):
    from paper_2505_06711_gb300 import binding

    srv = _server(spec, 0)
    try:
        ref = {name: _system(spec, structs[name], 0) for name in MIXED}
        a = _submit(srv, structs["water200"])
        b = _submit(srv, structs["fcc3"])
        l1, _ = srv.launch()
        assert sorted(l1) == sorted([a, b])
        c = _submit(srv, structs["fcc5"])
        l2, _ = srv.launch()
        assert l2 == [c]
        # a and b were evaluated once; the second launch must leave their rows alone
        res = srv.collect([a, b, c])
        for sl, name in ((a, "water200"), (b, "fcc3"), (c, "fcc5")):
            assert np.array_equal(res[sl][1], ref[name][1]), name
            assert abs(res[sl][0] - ref[name][0]) <= 1e-12 * abs(ref[name][0])
        off_a, _ = binding.reann_serve_slot(srv.srv, a)
        srv.release(a)
        d = _submit(srv, structs["water16"])  # fits in the first free range: a's
        off_d, _ = binding.reann_serve_slot(srv.srv, d)
        assert off_d == off_a
        # a pending slot released before any launch is never evaluated
        e = _submit(srv, structs["fcc3"])
        srv.release(e)
        l3, _ = srv.launch()
        assert l3 == [d]
        res = srv.collect([d, b, c])
        assert np.array_equal(res[d][1], ref["water16"][1])
        assert np.array_equal(res[b][1], ref["fcc3"][1])
        assert np.array_equal(res[c][1], ref["fcc5"][1])
        l4, _ = srv.launch()
        assert l4 == []
        with pytest.raises(binding.ReannError):
            srv.release(e)  # already released
    finally:
        srv.close()


def test_admission(spec, structs):
    from paper_2505_06711_gb300 import binding

    srv = _server(spec, 0, max_atoms=700, max_structures=2)
    try:
        w = _submit(srv, structs["water200"])  # 600 atoms
        assert w is not None
        assert _submit(srv, structs["fcc3"]) is None  # 600 + 108 > 700
        free_atoms, _, free_slots = binding.reann_serve_usage(srv.srv)
        assert free_atoms == 100 and free_slots == 1
        small = _submit(srv, structs["water16"])  # 48 atoms fit
        assert small is not None
        assert _submit(srv, structs["water16"]) is None  # no structure slot left
        srv.launch()
        srv.release(w)
        f = _submit(srv, structs["fcc3"])
        assert f is not None
        srv.launch()
        res = srv.collect([f])
        assert np.array_equal(res[f][1], _system(spec, structs["fcc3"], 0)[1])
    finally:
        srv.close()


def test_stride_too_small(spec, structs):
    from paper_2505_06711_gb300 import binding

    srv = _server(spec, 0, stride=16)
    try:
        with pytest.raises(binding.ReannError):
            _submit(srv, structs["fcc3"])
        assert binding.reann_serve_usage(srv.srv)[2] == 8  # nothing was admitted
    finally:
        srv.close()


def test_serve_stream(spec):
    from paper_2505_06711_gb300 import Potential
    from paper_2505_06711_gb300.serving import Server, latency_stats, make_requests, serve_alone, serve_stream

    templates = [water_box(m, seed=m) for m in (16, 40, 100)] + [fcc_box(k, seed=k) for k in (3, 4, 6)]
    reqs = make_requests(templates, 40, rate_per_s=4000.0, seed=7)
    srv = Server(spec, 4096, 60000, 16, precision=1)
    try:
        res, st = serve_stream(srv, reqs)
    finally:
        srv.close()
    assert all(r is not None for r in res)
    pot = Potential(spec, precision=1)
    try:
        alone, _ = serve_alone(pot, reqs)
    finally:
        pot.close()
    for r, a in zip(res, alone):
        assert np.array_equal(r.forces, a.forces)
        assert abs(r.energy - a.energy) <= 1e-12 * abs(a.energy)
    lat = latency_stats(res)
    print(f"[serve] {len(reqs)} requests, {st['launches']} launches, wall {st['wall_s']:.3f} s, {lat}")
    assert 1 <= st["launches"] <= len(reqs)
