"""The C ABI library builds, loads without a GPU and exports every function
include/fw.h declares (no compute calls here)."""

import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "fw.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s*(fw_[a-z_0-9]+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_library_exports_every_declared_symbol():
    from paper_2404_08364_gb300.build import build
    path = build()
    L = ctypes.CDLL(path)
    names = declared_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(L, n), f"{n} declared in fw.h but not exported"
    from paper_2404_08364_gb300 import _fw
    assert set(_fw.SIGNATURES) == set(names), "binding and header disagree"
    assert _fw.lib().fw_version() >> 16 == 1
    assert _fw.lib().fw_strerror(-4) == b"CSR row not strictly ascending"


def test_struct_layouts_match_header():
    from paper_2404_08364_gb300 import _fw
    # fw_params: int32 mode, float p, float q, int32 scale, int32 len, int8[16], double
    assert ctypes.sizeof(_fw.Params) == 4 * 5 + 16 + 4 + 8  # 4 bytes padding before the double
    assert _fw.Params.ppr_stop.offset == 40
    assert ctypes.sizeof(_fw.Stats) == 9 * 8
    assert ctypes.sizeof(_fw.Tuning) == 16


def test_missing_library_fails_loudly(tmp_path):
    from paper_2404_08364_gb300 import _fw
    import pytest
    saved = _fw._lib
    _fw._lib = None
    try:
        with pytest.raises(_fw.FwError):
            _fw.lib(str(tmp_path / "nope.so"))
    finally:
        _fw._lib = saved


def test_batch_size_follows_eq3():
    """Eq. 3 (Section 5.2): two result pools of |P_G| queries fit in the
    budget and two of |P_G| + 1 do not; a query needs its L + 1 path words
    plus its start and its path length (4 bytes each)."""
    from paper_2404_08364_gb300 import _fw
    L = _fw.lib()
    for budget, max_len in [(0, 80), (1, 0), (10 ** 9, 80), (123456789, 999), (2 ** 40, 80), (2 ** 20, 3)]:
        P = L.fw_batch_size(budget, max_len)
        per_query = (max_len + 1) * 4 + 4 + 4
        assert 2 * P * per_query <= budget
        assert 2 * (P + 1) * per_query > budget
    assert L.fw_batch_size(10 ** 6, -1) == 0
