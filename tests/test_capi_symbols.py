"""The C-ABI library builds for sm_103a, loads on a CPU-only host and exports
every entry point declared in include/tmop.h (no compute call is made)."""
import ctypes
import os
import re
import subprocess

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "tmop.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(tmop_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_seven_calls():
    names = _declared()
    for n in ("tmop_setup", "tmop_energy", "tmop_gradient", "tmop_hessian_setup",
              "tmop_hessian_apply", "tmop_hessian_diag", "tmop_newton_step"):
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_2205_12721_b300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    for n in _declared():
        assert hasattr(lib, n), n
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (tmop_\w+)", out))
    assert set(_declared()) <= exported


def test_binding_names_match_header():
    from paper_2205_12721_b300 import capi
    assert set(capi.EXPORTS) == set(_declared())


def test_no_oracle_in_product_path():
    """The product package never imports or links the oracle."""
    pkg = os.path.join(ROOT, "paper_2205_12721_b300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".cpp", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(import|from)\s+oracle\b", txt, re.M), f
                assert "liboracle" not in txt and "tmop_oracle" not in txt, f
