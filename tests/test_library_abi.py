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


def test_fast_division_matches_integer_division(tmp_path):
    """The multiply-and-shift quotient the 3D y-run diffusion kernel uses to
    find a thread's (x, y, z) equals n / d for every divisor 1..4096 and 2^k,
    2^k +- 1, with n at 0, 1, d - 1, d, d + 1, multiples of d +- 1 and
    2^31 - 1, plus 200 000 seeded random (n, d) pairs (compiled by the host
    C++ compiler from the same header as the kernel)."""
    import shutil
    import subprocess

    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    src = tmp_path / "fd.cpp"
    src.write_text(r'''
#include <cstdio>
#include <cstdint>
#include "fastdiv.h"
using namespace daeti;
static uint64_t s = 0x9e3779b97f4a7c15ull;
static uint32_t rnd() { s ^= s << 13; s ^= s >> 7; s ^= s << 17; return (uint32_t)(s >> 11); }
static int bad = 0;
static void check(unsigned d, long long n) {
    if (n < 0 || n > 2147483647LL) return;
    const FastDiv f = fast_div(d);
    if (fdiv((int)n, f) != (int)(n / d)) { if (bad < 5) std::printf("n=%lld d=%u\n", n, d); ++bad; }
}
int main() {
    unsigned ds[200]; int nd = 0;
    for (int k = 0; k < 31; ++k) { ds[nd++] = 1u << k; ds[nd++] = (1u << k) + 1; if (k) ds[nd++] = (1u << k) - 1; }
    ds[nd++] = 2147483647u;
    for (unsigned d = 1; d <= 4096 + nd; ++d) {
        const unsigned dd = d <= 4096 ? d : ds[d - 4097];
        const long long top = 2147483647LL;
        const long long q = top / dd;
        const long long ns[] = {0, 1, (long long)dd - 1, dd, (long long)dd + 1, q * dd, q * dd - 1, top, top - 1,
                                (q / 2) * dd + dd - 1, (q / 2) * dd};
        for (long long n : ns) check(dd, n);
    }
    for (int t = 0; t < 200000; ++t) {
        const unsigned d = 1 + rnd() % ((t & 1) ? 5000u : 2147483647u);
        check(d, (long long)(rnd() & 0x7fffffffu));
    }
    std::printf("bad %d\n", bad);
    return bad != 0;
}
''')
    exe = tmp_path / "fd"
    inc = os.path.join(ROOT, "paper_2011_04747_gb300", "csrc")
    subprocess.run([cxx, "-O2", "-std=c++17", "-I", inc, str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    assert out.returncode == 0, out.stdout
    assert "bad 0" in out.stdout
