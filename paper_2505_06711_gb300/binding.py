"""Thin ctypes binding of the C ABI in ``include/reann.h``.

Functions carry the C names and only marshal arguments (torch CUDA tensors ->
device pointers, numpy arrays -> host pointers); every step of the
computation runs in ``libreann.so``.  There is no CPU fallback: if the library
is missing, :func:`lib` raises.
"""

from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

REANN_OK = 0
REANN_E_ARG = -1
REANN_E_MISMATCH = -2
REANN_E_NOMEM = -3
REANN_E_GEOM = -4
REANN_E_CUDA = -5
REANN_E_TIMEOUT = -6
REANN_E_CAPACITY = -7
REANN_MLP_FP32 = 0
REANN_MLP_BF16 = 1
REANN_MLP_BF16X3 = 2
REANN_MLP_FP8 = 3

_NAMES = {
    REANN_E_ARG: "REANN_E_ARG",
    REANN_E_MISMATCH: "REANN_E_MISMATCH",
    REANN_E_NOMEM: "REANN_E_NOMEM",
    REANN_E_GEOM: "REANN_E_GEOM",
    REANN_E_CUDA: "REANN_E_CUDA",
    REANN_E_TIMEOUT: "REANN_E_TIMEOUT",
    REANN_E_CAPACITY: "REANN_E_CAPACITY",
}


class ReannError(RuntimeError):
    def __init__(self, code: int, msg: str = ""):
        super().__init__(f"{_NAMES.get(code, code)}: {msg}")
        self.code = code


_lib = None
_vp, _i64, _i32, _int, _dbl = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int, ctypes.c_double

_SIGS = {
    "reann_model_create": ([_int] * 7 + [_dbl, _dbl, _vp, _i64, ctypes.POINTER(_vp)], _int),
    "reann_model_create_ex": ([_int] * 7 + [_dbl, _dbl, _int, _vp, _i64, ctypes.POINTER(_vp)], _int),
    "reann_model_free": ([_vp], None),
    "reann_model_load": ([ctypes.c_char_p, ctypes.POINTER(_vp)], _int),
    "reann_model_save": ([_vp, ctypes.c_char_p], _int),
    "reann_ctx_create": ([_vp, _vp, ctypes.POINTER(_vp)], _int),
    "reann_ctx_free": ([_vp], None),
    "reann_ctx_set_mlp_precision": ([_vp, _int], _int),
    "reann_last_error": ([_vp], ctypes.c_char_p),
    "reann_ctx_check": ([_vp], _int),
    "reann_ctx_wait_selftest": ([_vp, _i64], _int),
    "reann_build_nlist": ([_vp, _i64, _vp, _vp, _vp, _dbl, _dbl, ctypes.POINTER(_vp)], _int),
    "reann_nlist_free": ([_vp], None),
    "reann_nlist_info": ([_vp, _vp, _vp, _vp, _vp], _int),
    "reann_nlist_export": ([_vp, _vp, _i64, _vp, _vp, _vp, _vp], _int),
    "reann_energy_forces": ([_vp, _vp, _vp, _int, _vp, _vp, _vp], _int),
    "reann_energy_forces_host": ([_vp, _vp, _vp, _int, _vp, _vp, _int], _int),
    "reann_get_layer": ([_vp, _vp, _int, _vp, _vp], _int),
    "reann_energy_forces_virial": ([_vp, _vp, _vp, _int, _vp, _vp, _vp, _vp, _vp], _int),
    "reann_md_step_nvt": ([_vp, _vp, _vp, _vp, _vp, _dbl, _int, _dbl, _dbl, _vp, _vp, _vp], _int),
    "reann_build_nlist_decomposed": ([_vp, _i64, _vp, _vp, _vp, _dbl, _dbl, _vp, ctypes.POINTER(_vp)], _int),
    "reann_decomp_info": ([_vp, _vp, _vp, _vp, _vp], _int),
    "reann_nlist_rebuild": ([_vp, _vp, _vp], _int),
    "reann_ctx_profile": ([_vp, _int], _int),
    "reann_profile_regions": ([], _int),
    "reann_profile_region_name": ([_int], ctypes.c_char_p),
    "reann_ctx_profile_read": ([_vp, _vp, _vp], _int),
    "reann_serve_create": ([_vp, _i64, _i64, _int, _int, ctypes.POINTER(_vp)], _int),
    "reann_serve_free": ([_vp], None),
    "reann_serve_submit": ([_vp, _vp, _i64, _vp, _vp, _vp, _dbl, ctypes.POINTER(_int)], _int),
    "reann_serve_launch": ([_vp, _vp, _vp, _vp, ctypes.POINTER(_int)], _int),
    "reann_serve_release": ([_vp, _int], _int),
    "reann_serve_slot": ([_vp, _int, _vp, _vp], _int),
    "reann_serve_usage": ([_vp, _vp, _vp, _vp], _int),
    "reann_md_step": ([_vp, _vp, _vp, _vp, _vp, _dbl, _int, _vp, _vp], _int),
    "reann_md_info": ([_vp, _vp, _vp, _vp], _int),
    "reann_energy_sum_noalloc": ([_vp, _i64, _vp, _vp], _int),
    "reann_energy_sum_noalloc_max_atoms": ([], _i64),
}


def library_path() -> str:
    return _build.LIB


def lib():
    """Load ``libreann.so``; raise if it has not been built."""
    global _lib
    if _lib is None:
        path = library_path()
        if not os.path.exists(path):
            raise RuntimeError(f"CUDA library not built ({path}); run __graft_entry__.build()")
        handle = ctypes.CDLL(path)
        for name, (args, res) in _SIGS.items():
            fn = getattr(handle, name)
            fn.argtypes = args
            fn.restype = res
        _lib = handle
    return _lib


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        return t.ctypes.data_as(ctypes.c_void_p)
    return ctypes.c_void_p(t.data_ptr())


def _dev(t, dtype, shape=None, name="tensor"):
    import torch

    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype or not t.is_contiguous():
        raise TypeError(f"{name} must be a contiguous {dtype} tensor")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")
    return t


def _check(rc, ctx=None):
    if rc != REANN_OK:
        msg = lib().reann_last_error(ctx).decode() if ctx else ""
        raise ReannError(rc, msg)


# ------------------------------------------------------------------ model --
def reann_model_create(spec) -> ctypes.c_void_p:
    """``spec`` is a :class:`synth.model.ModelSpec` (or any object with its fields);
    a pair-feature spec (``spec.pairs``) goes through reann_model_create_ex."""
    if getattr(spec, "pairs", False):
        return reann_model_create_ex(spec, 1)
    params = np.ascontiguousarray(spec.params, dtype=np.float32)
    out = _vp()
    rc = lib().reann_model_create(
        spec.n_elem, spec.T, spec.n_phi, spec.l_max, spec.n_orb, spec.h1, spec.h2,
        float(spec.r_c), float(spec.alpha), _ptr(params), params.size, ctypes.byref(out),
    )
    _check(rc)
    return out


def reann_model_create_ex(spec, feature_pairs: int | None = None) -> ctypes.c_void_p:
    """As reann_model_create with the feature choice (default: ``spec.pairs``)."""
    fp = int(getattr(spec, "pairs", False)) if feature_pairs is None else int(feature_pairs)
    params = np.ascontiguousarray(spec.params, dtype=np.float32)
    out = _vp()
    rc = lib().reann_model_create_ex(
        spec.n_elem, spec.T, spec.n_phi, spec.l_max, spec.n_orb, spec.h1, spec.h2,
        float(spec.r_c), float(spec.alpha), fp, _ptr(params), params.size, ctypes.byref(out),
    )
    _check(rc)
    return out


def reann_model_free(model) -> None:
    lib().reann_model_free(model)


def reann_model_load(path) -> ctypes.c_void_p:
    """Model from a file written by reann_model_save or synth.model.write_model_file."""
    out = _vp()
    rc = lib().reann_model_load(os.fsencode(path), ctypes.byref(out))
    _check(rc)
    return out


def reann_model_save(model, path) -> None:
    _check(lib().reann_model_save(model, os.fsencode(path)))


# ---------------------------------------------------------------- context --
def reann_ctx_create(model, stream=None) -> ctypes.c_void_p:
    """``stream``: a torch.cuda.Stream, a raw cudaStream_t int, or None (current torch stream)."""
    import torch

    if stream is None:
        stream = torch.cuda.current_stream()
    handle = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
    out = _vp()
    _check(lib().reann_ctx_create(model, _vp(handle), ctypes.byref(out)))
    return out


def reann_ctx_free(ctx) -> None:
    lib().reann_ctx_free(ctx)


def reann_ctx_set_mlp_precision(ctx, precision: int) -> None:
    _check(lib().reann_ctx_set_mlp_precision(ctx, int(precision)), ctx)


def reann_last_error(ctx) -> str:
    return lib().reann_last_error(ctx).decode()


def reann_ctx_wait_selftest(ctx, polls: int) -> None:
    """Enqueue one bounded wait that runs out (reann_ctx_check then reports REANN_E_TIMEOUT)."""
    _check(lib().reann_ctx_wait_selftest(ctx, int(polls)), ctx)


def reann_ctx_check(ctx) -> None:
    _check(lib().reann_ctx_check(ctx), ctx)


# ---------------------------------------------------------- neighbour list --
def reann_build_nlist(ctx, pos, species, cell, r_c: float, skin: float):
    import torch

    n = pos.shape[0]
    _dev(pos, torch.float64, (n, 3), "pos")
    _dev(species, torch.int32, (n,), "species")
    c = np.ascontiguousarray(cell, dtype=np.float64).reshape(9)
    out = _vp()
    _check(lib().reann_build_nlist(ctx, n, _ptr(pos), _ptr(species), _ptr(c), float(r_c), float(skin), ctypes.byref(out)), ctx)
    return out


def reann_build_nlist_decomposed(ctx, pos, species, cell, r_c: float, skin: float, ranks):
    import torch

    n = pos.shape[0]
    _dev(pos, torch.float64, (n, 3), "pos")
    _dev(species, torch.int32, (n,), "species")
    c = np.ascontiguousarray(cell, dtype=np.float64).reshape(9)
    rk = np.ascontiguousarray(ranks, dtype=np.int32).reshape(3)
    out = _vp()
    _check(lib().reann_build_nlist_decomposed(ctx, n, _ptr(pos), _ptr(species), _ptr(c), float(r_c), float(skin),
                                              _ptr(rk), ctypes.byref(out)), ctx)
    return out


def reann_decomp_info(nl) -> dict:
    """{'local', 'ghosts', 'remote'}: per-rank counts (numpy int64 arrays)."""
    k = np.zeros(1, np.int32)
    _check(lib().reann_decomp_info(nl, _ptr(k), None, None, None))
    loc, gh, rem = (np.zeros(int(k[0]), np.int64) for _ in range(3))
    _check(lib().reann_decomp_info(nl, _ptr(k), _ptr(loc), _ptr(gh), _ptr(rem)))
    return {"local": loc, "ghosts": gh, "remote": rem}


def reann_nlist_free(nl) -> None:
    lib().reann_nlist_free(nl)


def reann_nlist_info(nl) -> tuple[int, int, int, int]:
    """(atoms, ghost slots, listed pairs within r_c + skin, live pairs within r_c of the last evaluation)."""
    a, g, p, v = (np.zeros(1, np.int64) for _ in range(4))
    _check(lib().reann_nlist_info(nl, _ptr(a), _ptr(g), _ptr(p), _ptr(v)))
    return int(a[0]), int(g[0]), int(p[0]), int(v[0])


def reann_nlist_export(ctx, nl):
    """(i, j, shift) of every listed pair, caller order, caller-relative shifts (host arrays)."""
    cnt = np.zeros(1, np.int64)
    _check(lib().reann_nlist_export(ctx, nl, 0, None, None, None, _ptr(cnt)), ctx)
    k = int(cnt[0])
    i = np.empty(max(k, 1), np.int32)
    j = np.empty(max(k, 1), np.int32)
    s = np.empty((max(k, 1), 3), np.int32)
    _check(lib().reann_nlist_export(ctx, nl, k, _ptr(i), _ptr(j), _ptr(s), _ptr(cnt)), ctx)
    return i[:k], j[:k], s[:k]


# -------------------------------------------------------------- evaluation --
def reann_energy_forces(ctx, nl, pos, T: int, energy, forces, atom_energy=None) -> None:
    import torch

    n = pos.shape[0]
    _dev(pos, torch.float64, (n, 3), "pos")
    _dev(energy, torch.float64, (1,), "energy")
    _dev(forces, torch.float32, (n, 3), "forces")
    if atom_energy is not None:
        _dev(atom_energy, torch.float32, (n,), "atom_energy")
    _check(lib().reann_energy_forces(ctx, nl, _ptr(pos), int(T), _ptr(energy), _ptr(forces), _ptr(atom_energy)), ctx)


def reann_energy_forces_virial(ctx, nl, pos, T: int, energy, forces, virial, atom_energy=None, atom_virial=None) -> None:
    import torch

    n = pos.shape[0]
    _dev(pos, torch.float64, (n, 3), "pos")
    _dev(energy, torch.float64, (1,), "energy")
    _dev(forces, torch.float32, (n, 3), "forces")
    _dev(virial, torch.float64, (3, 3), "virial")
    if atom_energy is not None:
        _dev(atom_energy, torch.float32, (n,), "atom_energy")
    if atom_virial is not None:
        _dev(atom_virial, torch.float32, (n, 9), "atom_virial")
    _check(lib().reann_energy_forces_virial(ctx, nl, _ptr(pos), int(T), _ptr(energy), _ptr(forces),
                                            _ptr(atom_energy), _ptr(virial), _ptr(atom_virial)), ctx)


def reann_energy_forces_host(ctx, nl, pos, T: int, energy, forces, rebuild: int = 0) -> None:
    """Host buffers: numpy arrays or pinned CPU torch tensors (pos f64 N x 3, energy f64 [1], forces f32 N x 3)."""
    for a in (pos, energy, forces):
        if isinstance(a, np.ndarray):
            if not a.flags.c_contiguous:
                raise TypeError("host buffers must be contiguous")
        elif getattr(a, "is_cuda", True) or not a.is_contiguous():
            raise TypeError("host buffers must be contiguous numpy arrays or CPU tensors")
    _check(lib().reann_energy_forces_host(ctx, nl, _ptr(pos), int(T), _ptr(energy), _ptr(forces), int(rebuild)), ctx)


def reann_get_layer(ctx, nl, layer: int, rho=None, coef=None) -> None:
    _check(lib().reann_get_layer(ctx, nl, int(layer), _ptr(rho), _ptr(coef)), ctx)


def reann_nlist_rebuild(ctx, nl, pos) -> None:
    import torch

    _dev(pos, torch.float64, None, "pos")
    _check(lib().reann_nlist_rebuild(ctx, nl, _ptr(pos)), ctx)


# ---------------------------------------------------------------- serving --
def reann_serve_create(ctx, max_atoms: int, max_ghosts: int, max_structures: int, stride: int):
    out = _vp()
    _check(lib().reann_serve_create(ctx, int(max_atoms), int(max_ghosts), int(max_structures), int(stride),
                                    ctypes.byref(out)), ctx)
    return out


def reann_serve_free(srv) -> None:
    lib().reann_serve_free(srv)


def reann_serve_submit(srv, ctx, build_ctx, pos, species, cell, skin: float):
    """Slot id, or None when the pool refuses admission (REANN_E_NOMEM)."""
    import torch

    n = pos.shape[0]
    _dev(pos, torch.float64, (n, 3), "pos")
    _dev(species, torch.int32, (n,), "species")
    c = np.ascontiguousarray(cell, dtype=np.float64).reshape(9)
    slot = _int(-1)
    rc = lib().reann_serve_submit(srv, build_ctx, n, _ptr(pos), _ptr(species), _ptr(c), float(skin), ctypes.byref(slot))
    if rc == REANN_E_NOMEM:
        return None
    _check(rc, ctx)
    return int(slot.value)


def reann_serve_launch(srv, ctx, energies, forces, max_structures: int) -> list[int]:
    slots = np.zeros(max_structures, np.int32)
    cnt = _int(0)
    _check(lib().reann_serve_launch(srv, _ptr(energies), _ptr(forces), _ptr(slots), ctypes.byref(cnt)), ctx)
    return slots[: cnt.value].tolist()


def reann_serve_release(srv, ctx, slot: int) -> None:
    _check(lib().reann_serve_release(srv, int(slot)), ctx)


def reann_serve_slot(srv, slot: int) -> tuple[int, int]:
    o, n = np.zeros(1, np.int64), np.zeros(1, np.int64)
    _check(lib().reann_serve_slot(srv, int(slot), _ptr(o), _ptr(n)))
    return int(o[0]), int(n[0])


def reann_serve_usage(srv) -> tuple[int, int, int]:
    a, g = np.zeros(1, np.int64), np.zeros(1, np.int64)
    s = np.zeros(1, np.int32)
    _check(lib().reann_serve_usage(srv, _ptr(a), _ptr(g), _ptr(s)))
    return int(a[0]), int(g[0]), int(s[0])


# --------------------------------------------------------------------- MD --
def reann_md_step(ctx, nl, pos, vel, mass, dt_fs: float, n_steps: int, e_pot=None, e_kin=None) -> None:
    import torch

    n = pos.shape[0]
    _dev(pos, torch.float64, (n, 3), "pos")
    _dev(vel, torch.float64, (n, 3), "vel")
    _dev(mass, torch.float64, (n,), "mass")
    for name, a in (("e_pot", e_pot), ("e_kin", e_kin)):
        if a is not None:
            _dev(a, torch.float64, None, name)
            if a.numel() < n_steps:
                raise ValueError(f"{name} holds fewer than n_steps entries")
    _check(lib().reann_md_step(ctx, nl, _ptr(pos), _ptr(vel), _ptr(mass), float(dt_fs), int(n_steps), _ptr(e_pot),
                               _ptr(e_kin)), ctx)


def reann_md_step_nvt(ctx, nl, pos, vel, mass, dt_fs: float, n_steps: int, temperature_k: float, tau_fs: float,
                      e_pot=None, e_kin=None, e_bath=None) -> None:
    import torch

    n = pos.shape[0]
    _dev(pos, torch.float64, (n, 3), "pos")
    _dev(vel, torch.float64, (n, 3), "vel")
    _dev(mass, torch.float64, (n,), "mass")
    for name, a in (("e_pot", e_pot), ("e_kin", e_kin), ("e_bath", e_bath)):
        if a is not None:
            _dev(a, torch.float64, None, name)
            if a.numel() < n_steps:
                raise ValueError(f"{name} holds fewer than n_steps entries")
    _check(lib().reann_md_step_nvt(ctx, nl, _ptr(pos), _ptr(vel), _ptr(mass), float(dt_fs), int(n_steps),
                                   float(temperature_k), float(tau_fs), _ptr(e_pot), _ptr(e_kin), _ptr(e_bath)), ctx)


def reann_md_info(ctx, nl) -> tuple[int, int]:
    """(steps of the last reann_md_step call, rebuilds since the first call)."""
    s, r = np.zeros(1, np.int64), np.zeros(1, np.int64)
    _check(lib().reann_md_info(ctx, nl, _ptr(s), _ptr(r)), ctx)
    return int(s[0]), int(r[0])


# ---------------------------------------------------------- no-allocation --
def reann_energy_sum_noalloc(atom_energy, n_atoms: int, energy, stream=None) -> int:
    """FP64 sum of per-atom energies with the library's fixed scratch (no device allocation).

    For callers that must not allocate (graph capture, engine-owned memory);
    returns the C return code instead of raising, so those callers can branch on it.
    """
    import torch

    if stream is None:
        stream = torch.cuda.current_stream()
    handle = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
    return int(lib().reann_energy_sum_noalloc(_ptr(atom_energy), int(n_atoms), _ptr(energy), _vp(handle)))


def reann_energy_sum_noalloc_max_atoms() -> int:
    return int(lib().reann_energy_sum_noalloc_max_atoms())


# --------------------------------------------------------------- profiling --
def reann_ctx_profile(ctx, enable: bool) -> None:
    _check(lib().reann_ctx_profile(ctx, int(bool(enable))), ctx)


def reann_profile_regions() -> int:
    return int(lib().reann_profile_regions())


def reann_profile_region_name(region: int) -> str:
    return lib().reann_profile_region_name(int(region)).decode()


def reann_ctx_profile_read(ctx) -> dict:
    """{region name: (total ms, launches)} since profiling was enabled (synchronous)."""
    k = reann_profile_regions()
    ms = np.zeros(k, np.float64)
    cnt = np.zeros(k, np.int64)
    _check(lib().reann_ctx_profile_read(ctx, _ptr(ms), _ptr(cnt)), ctx)
    return {reann_profile_region_name(r): (float(ms[r]), int(cnt[r])) for r in range(k)}
