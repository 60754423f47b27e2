"""CPU-side checks of the C ABI library: it builds for sm_103a, loads, and
exports every entry point declared in include/daeti.h (no GPU calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "daeti.h")).read()
    return sorted(set(re.findall(r"^\s*(?:int|void|const char\*)\s+(daeti_\w+)\s*\(", src, re.M)))


@pytest.fixture(scope="module")
def lib_path():
    from paper_2011_04747_gb300 import build

    return build.build()


def test_library_exports_every_declared_symbol(lib_path):
    lib = ctypes.CDLL(lib_path)
    names = _declared()
    assert len(names) >= 25
    for n in names:
        assert hasattr(lib, n), n


def test_binding_covers_every_declared_symbol():
    from paper_2011_04747_gb300 import binding

    assert set(_declared()) == set(binding.declared_symbols())


def test_binding_loads_and_fails_loudly_without_gpu(lib_path):
    import torch

    from paper_2011_04747_gb300 import binding

    binding.load_library()
    o = binding.daeti_options()
    binding.load_library().daeti_default_options(ctypes.byref(o))
    assert o.struct_size == ctypes.sizeof(binding.daeti_options)
    assert o.precision == binding.FP32_KAHAN and abs(o.dt - 0.1) < 1e-15 and o.graph_steps == 20
    if not torch.cuda.is_available():
        with pytest.raises(binding.DaetiError):
            binding.Solver()


def test_missing_library_raises(tmp_path):
    from paper_2011_04747_gb300 import binding

    saved = binding._lib
    binding._lib = None
    try:
        with pytest.raises(ImportError):
            binding.load_library(str(tmp_path / "nope.so"))
    finally:
        binding._lib = saved
