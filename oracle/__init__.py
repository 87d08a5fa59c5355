"""FP64 CPU oracle for the REANN energy/force path -- test infrastructure only.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg
may import this package.  The product path (``paper_2505_06711_gb300``) never
does, and this package never imports the product.

The arithmetic lives in ``reann_oracle.c`` (plain C, FP64, brute-force
neighbour search, hand-derived reverse pass), compiled here with ``gcc`` and
loaded through ctypes.  See that file's header for what it computes and the
paper passages it follows (Sec. 2.1 Eqs. 1-2, Sec. 2.2 Eqs. 3-5).
"""

from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "reann_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libreann_oracle.so")
_lock = threading.Lock()
_lib = None

ERRORS = {0: "ok", -1: "bad argument", -3: "out of memory", -4: "bad geometry", -7: "capacity"}


class OracleError(RuntimeError):
    pass


def build(force: bool = False) -> str:
    """Compile the oracle shared library (gcc, OpenMP, no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i64, i32, dbl, ptr, c_int = ctypes.c_int64, ctypes.c_int32, ctypes.c_double, ctypes.c_void_p, ctypes.c_int
            lib.oracle_neighbors.argtypes = [i64, ptr, ptr, dbl, i64, ptr, ptr, ptr, ptr, c_int]
            lib.oracle_neighbors.restype = c_int
            lib.oracle_energy_forces.argtypes = [c_int] * 7 + [dbl, dbl, c_int, ptr, i64, ptr, ptr, ptr, ptr, ptr, ptr, ptr, ptr, ptr, c_int]
            lib.oracle_energy_forces.restype = c_int
            lib.oracle_max_threads.argtypes = []
            lib.oracle_max_threads.restype = c_int
            _lib = lib
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _check(rc):
    if rc != 0:
        raise OracleError(f"oracle error {rc}: {ERRORS.get(rc, '?')}")


def max_threads() -> int:
    return int(_load().oracle_max_threads())


def neighbors(pos, cell, r_cut: float, n_threads: int = 0):
    """Brute-force list of (i, j, shift) with |r_j + shift.cell - r_i| < r_cut.

    Shifts are integer lattice vectors relative to the given (possibly
    unwrapped) positions.  ``cell=None`` means no periodic images.
    Returns (i int32[E], j int32[E], shift int32[E,3]).
    """
    lib = _load()
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    n = pos.shape[0]
    cellp = None if cell is None else np.ascontiguousarray(cell, dtype=np.float64).reshape(9)
    cnt = np.zeros(1, np.int64)
    cap = max(1, n * 64)
    while True:
        oi = np.empty(cap, np.int32)
        oj = np.empty(cap, np.int32)
        osh = np.empty((cap, 3), np.int32)
        rc = lib.oracle_neighbors(n, _p(pos), _p(cellp), float(r_cut), cap, _p(oi), _p(oj), _p(osh), _p(cnt), n_threads)
        if rc == -7:
            cap = int(cnt[0])
            continue
        _check(rc)
        k = int(cnt[0])
        return oi[:k].copy(), oj[:k].copy(), osh[:k].copy()


def energy_forces(model, pos, species, cell, want_layers: bool = False, n_threads: int = 0):
    """FP64 energy, forces (N,3), atom energies (N,), virial (3,3) [and rho (T,N,F), c (T,N,P)].

    The virial is W = -dE/d(strain) (positions and cell strained alike).

    ``model`` is a :class:`synth.model.ModelSpec`; its ``T`` is the number of
    message-passing layers.  ``cell=None`` evaluates a free cluster.
    """
    lib = _load()
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    species = np.ascontiguousarray(species, dtype=np.int32)
    n = pos.shape[0]
    cellp = None if cell is None else np.ascontiguousarray(cell, dtype=np.float64).reshape(9)
    params = np.ascontiguousarray(model.params, dtype=np.float32)
    energy = np.zeros(1, np.float64)
    forces = np.zeros((n, 3), np.float64)
    eps = np.zeros(n, np.float64)
    rho = np.zeros((model.T, n, model.n_feat), np.float64) if want_layers else None
    coef = np.zeros((model.T, n, model.n_phi), np.float64) if want_layers else None
    virial = np.zeros((3, 3), np.float64)
    rc = lib.oracle_energy_forces(
        model.n_elem, model.T, model.n_phi, model.l_max, model.n_orb, model.h1, model.h2,
        float(model.r_c), float(model.alpha), int(getattr(model, "pairs", False)), _p(params), n, _p(pos),
        _p(species), _p(cellp),
        _p(energy), _p(forces), _p(eps), _p(rho), _p(coef), _p(virial), n_threads,
    )
    _check(rc)
    out = {"energy": float(energy[0]), "forces": forces, "atom_energy": eps, "virial": virial}
    if want_layers:
        out["rho"] = rho
        out["coef"] = coef
    return out
