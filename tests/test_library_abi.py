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


def test_binding_structs_match_the_header_layout(tmp_path):
    """The ctypes mirrors of daeti_options and daeti_tuning have the header's
    size and field offsets (compiled and printed by the host C compiler)."""
    import shutil
    import subprocess

    from paper_2011_04747_gb300 import binding

    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    structs = {"daeti_options": binding.daeti_options, "daeti_tuning": binding.daeti_tuning}
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "daeti.h"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append(f'printf("{name} size %zu\\n", sizeof({name}));')
        for field, _ in cls._fields_:
            lines.append(f'printf("{name} {field} %zu\\n", offsetof({name}, {field}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for name, cls in structs.items():
        assert got[(name, "size")] == ctypes.sizeof(cls), name
        for field, _ in cls._fields_:
            assert got[(name, field)] == getattr(cls, field).offset, (name, field)
