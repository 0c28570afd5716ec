"""The C-ABI library builds for sm_103a, loads without a GPU and exports every symbol
that include/d2ip.h declares (no compute calls)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    with open(os.path.join(ROOT, "include", "d2ip.h")) as f:
        src = f.read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(d2ip_[a-z0-9_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol(d2ip):
    lib = ctypes.CDLL(d2ip.LIB_PATH)
    names = _declared()
    assert len(names) >= 30
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) <= set(d2ip.exported_symbols())


def test_no_device_is_reported_not_crashed(d2ip):
    import torch
    if torch.cuda.is_available():
        return
    try:
        d2ip.d2ip_create(0)
    except d2ip.D2IPError as e:
        assert e.status == -6
    else:
        raise AssertionError("d2ip_create succeeded without a GPU")
