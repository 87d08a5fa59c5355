"""Model files (reann_model_load / reann_model_save), host only.

A file written by the seeded generator's writer (synth.model.write_model_file)
is loaded by the library and saved again: the saved bytes must equal the
written ones, which pins every header field and every parameter bit of the
loaded model.  Damaged files (truncated, padded, wrong magic, wrong version,
a parameter count that does not match the shape) are refused with
REANN_E_ARG.  The GPU test in test_gpu_api.py evaluates a loaded model.
"""

from __future__ import annotations

import ctypes

import numpy as np
import pytest

from synth import make_model, write_model_file


@pytest.fixture(scope="module")
def lib():
    from paper_2505_06711_gb300 import binding, build

    build.build()
    return binding


def _load_rc(binding, path):
    out = ctypes.c_void_p()
    rc = binding.lib().reann_model_load(str(path).encode(), ctypes.byref(out))
    if rc == binding.REANN_OK:
        binding.reann_model_free(out)
    return rc


@pytest.mark.parametrize("kw", [dict(T=3), dict(T=5, n_elem=8), dict(T=2, pairs=True)])
def test_load_then_save_reproduces_the_file(lib, tmp_path, kw):
    spec = make_model(**kw)
    src, dst = tmp_path / "m.reann", tmp_path / "again.reann"
    write_model_file(spec, src)
    m = lib.reann_model_load(src)
    lib.reann_model_save(m, dst)
    lib.reann_model_free(m)
    a, b = src.read_bytes(), dst.read_bytes()
    assert len(a) == 72 + 4 * spec.params.size
    assert a == b


def test_saved_model_equals_created_model(lib, tmp_path):
    spec = make_model(T=3)
    m = lib.reann_model_create(spec)
    path = tmp_path / "created.reann"
    lib.reann_model_save(m, path)
    lib.reann_model_free(m)
    raw = path.read_bytes()
    assert raw[:8] == b"REANNMDL"
    params = np.frombuffer(raw[72:], dtype="<f4")
    assert np.array_equal(params.view(np.uint32), np.ascontiguousarray(spec.params, np.float32).view(np.uint32))


def test_damaged_files_are_refused(lib, tmp_path):
    spec = make_model(T=3)
    good = tmp_path / "good.reann"
    write_model_file(spec, good)
    raw = good.read_bytes()
    assert _load_rc(lib, good) == lib.REANN_OK
    cases = {
        "truncated": raw[:-1],
        "padded": raw + b"\0",
        "header_only": raw[:72],
        "short_header": raw[:40],
        "magic": b"REANNMDX" + raw[8:],
        "version": raw[:8] + np.array([2], "<u4").tobytes() + raw[12:],
        # one parameter fewer, with a matching count field: the shape check refuses it
        "count": raw[:64] + np.array([spec.params.size - 1], "<i8").tobytes() + raw[72:-4],
        "n_phi": raw[:20] + np.array([7], "<i4").tobytes() + raw[24:],
        "nan_param": raw[:72] + np.array([np.nan], "<f4").tobytes() + raw[76:],
    }
    for name, data in cases.items():
        p = tmp_path / f"{name}.reann"
        p.write_bytes(data)
        assert _load_rc(lib, p) == lib.REANN_E_ARG, name
    assert _load_rc(lib, tmp_path / "missing.reann") == lib.REANN_E_ARG
