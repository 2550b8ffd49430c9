"""The oracle and the CUDA path share no code: neither includes, imports or
links the other, and the product path (the package, its CUDA sources and the
public header) never touches the oracle.  Only the seeded input generators
(fw_inputs, which hold none of the method's arithmetic) serve both."""

import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _files(d, exts):
    out = []
    for base, _, names in os.walk(os.path.join(ROOT, d)):
        if "_build" in base or "__pycache__" in base:
            continue
        out += [os.path.join(base, n) for n in names if n.endswith(exts)]
    return out


def test_cuda_path_does_not_touch_the_oracle():
    for f in _files("paper_2404_08364_gb300", (".cu", ".cuh", ".py", ".h")) + _files("include", (".h",)):
        src = open(f).read()
        assert not re.search(r"^\s*(import|from)\s+oracle\b", src, re.M), f
        assert not re.search(r'#include\s+[<"][^>"]*oracle', src), f
        assert "liboracle" not in src, f


def test_oracle_does_not_touch_the_cuda_path():
    for f in _files("oracle", (".c", ".h", ".py")):
        src = open(f).read()
        assert not re.search(r"^\s*(import|from)\s+paper_2404_08364_gb300\b", src, re.M), f
        assert not re.search(r'#include\s+[<"](cuda|fw\.h|fw_internal)', src), f
        assert "libfw" not in src, f


def test_inputs_hold_no_method_arithmetic():
    for f in _files("fw_inputs", (".py",)):
        src = open(f).read()
        assert not re.search(r"^\s*(import|from)\s+(oracle|paper_2404_08364_gb300)\b", src, re.M), f
        for word in ("philox", "node2vec", "reservoir"):
            assert word not in src.lower(), (f, word)
