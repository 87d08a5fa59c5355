"""Host-side checks of the C ABI that need no GPU.

* the library builds for sm_103a and exports every entry point declared in
  ``include/reann.h``;
* model creation validates shapes on the host (no CUDA call);
* creating a context without a usable device fails with a clean error code.
"""

from __future__ import annotations

import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "reann.h")


@pytest.fixture(scope="module")
def libpath():
    from paper_2505_06711_gb300 import build

    return build.build()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(reann_\w+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("reann_build_nlist", "reann_energy_forces", "reann_model_create", "reann_ctx_create"):
        assert required in names


def test_every_declared_symbol_is_exported(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_symbol(libpath):
    from paper_2505_06711_gb300 import binding

    for name in declared_functions():
        assert hasattr(binding, name), name


def test_model_create_validates_on_host(libpath):
    from paper_2505_06711_gb300 import binding
    from synth import make_model

    spec = make_model(T=3)
    h = binding.reann_model_create(spec)
    binding.reann_model_free(h)
    bad = make_model(T=3, n_orb=8)
    with pytest.raises(binding.ReannError) as e:
        binding.reann_model_create(bad)
    assert e.value.code == binding.REANN_E_ARG
    spec2 = make_model(T=2)
    spec2.params = spec2.params[:-1]
    with pytest.raises(binding.ReannError):
        binding.reann_model_create(spec2)
    spec3 = make_model(T=2)
    spec3.params = spec3.params.copy()
    spec3.params[5] = np.nan
    with pytest.raises(binding.ReannError):
        binding.reann_model_create(spec3)


def test_pair_feature_model_validates_on_host(libpath):
    from paper_2505_06711_gb300 import binding
    from synth import make_model

    spec = make_model(T=3, pairs=True)
    assert spec.n_orb == 8 and spec.n_feat == 108
    m = binding.reann_model_create(spec)  # dispatches to reann_model_create_ex
    binding.reann_model_free(m)
    with pytest.raises(binding.ReannError):
        binding.reann_model_create_ex(spec, 0)  # a pair parameter vector read as Eq. 1's layout
    with pytest.raises(binding.ReannError):
        binding.reann_model_create_ex(make_model(T=3), 1)  # n_orb 16 with pair features
    with pytest.raises(binding.ReannError):
        binding.reann_model_create_ex(spec, 2)


def test_ctx_without_device_fails_cleanly(libpath):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a device is present")
    from paper_2505_06711_gb300 import binding
    from synth import make_model

    lib = binding.lib()
    h = binding.reann_model_create(make_model(T=1))
    out = ctypes.c_void_p()
    rc = lib.reann_ctx_create(h, None, ctypes.byref(out))
    binding.reann_model_free(h)
    assert rc == binding.REANN_E_CUDA
    assert not out.value
