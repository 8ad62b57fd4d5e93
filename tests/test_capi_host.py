"""The C-ABI library loads without a GPU, exports every symbol include/privft.h
declares, and its host-only parameter utilities agree with the oracle's
independent computation (prime rule, Gaussian table)."""
import os
import re
import subprocess

import pytest

import paper_1908_06972_gb300 as pft
from oracle import params as P

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def built():
    pft.build()
    return pft.lib()


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            names |= set(re.findall(r"^\s*(?:int|const char\*)\s+(pft_\w+)\s*\(", txt, re.M))
    return names


def test_every_declared_symbol_is_exported(built):
    decl = _declared()
    assert len(decl) >= 40
    out = subprocess.run(["nm", "-D", "--defined-only", pft._build.SO], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (pft_\w+)", out))
    assert decl <= exported, sorted(decl - exported)
    assert set(pft.exported_symbols()) <= decl
    for name in decl:
        assert hasattr(built, name)


def test_library_primes_follow_the_rule(built):
    for logn, bits in ((12, 40), (12, 60), (16, 50), (16, 60), (15, 40)):
        assert pft.pft_gen_primes(logn, bits, 8) == P.primes_of_bits(bits, logn, 8)
    q0 = P.primes_of_bits(60, 16, 1)
    assert pft.pft_gen_primes(16, 60, 4, exclude=q0) == P.primes_of_bits(60, 16, 4, exclude=q0)


def test_library_gauss_table_matches_oracle(built):
    assert pft.pft_gauss_cdt(3.2) == P.gauss_cdt("3.2")


def test_no_cpu_fallback_when_missing(monkeypatch, tmp_path):
    monkeypatch.setattr(pft._build, "SO", str(tmp_path / "missing.so"))
    monkeypatch.setattr(pft, "_LIB", None)
    with pytest.raises(pft.NativeLibraryMissing):
        pft.lib()


def test_struct_layouts_match_the_header(tmp_path):
    """The ctypes mirrors of the header's structs have the C compiler's sizes and offsets."""
    import ctypes

    src = tmp_path / "layout.c"
    src.write_text('#include <stddef.h>\n#include <stdio.h>\n#include "privft.h"\n'
                   "int main(void) {\n"
                   '  printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu\\n", sizeof(pft_job), offsetof(pft_job, a),\n'
                   "         offsetof(pft_job, b), offsetof(pft_job, p), offsetof(pft_job, out),\n"
                   "         offsetof(pft_job, after), offsetof(pft_job, wait_flag), offsetof(pft_job, wait_value),\n"
                   "         sizeof(pft_server_done));\n"
                   "  return 0;\n}\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    J = pft.pft_job
    want = [ctypes.sizeof(J), J.a.offset, J.b.offset, J.p.offset, J.out.offset, J.after.offset, J.wait_flag.offset,
            J.wait_value.offset, ctypes.sizeof(pft.pft_server_done)]
    assert got == want
