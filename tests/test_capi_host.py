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
