"""The C ABI library builds for sm_103a, loads on this machine and exports every symbol that
include/gbkm.h declares (no GPU needed: nothing is called but gbkm_version)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not fn.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", fn)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w]*\s*\**\s*\b([A-Za-z_]\w*)\s*\(", src, flags=re.M):
            if m.group(1) not in ("if", "while", "for", "return", "sizeof"):
                names.append(m.group(1))
    return names


def test_header_declares_the_entry_points():
    names = set(_declared())
    for want in ["kmeans_project_block", "kmeans_seed_pp", "kmeans_assign", "kmeans_update",
                 "kmeans_cost", "kmeans_row_norms", "kmeans_quantize", "gbkm_create", "gbkm_sync"]:
        assert want in names


def test_library_exports_every_declared_symbol():
    from paper_1502_04265_gb300 import build

    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing
    lib.gbkm_version.restype = ctypes.c_int
    assert lib.gbkm_version() >= 10000


def test_binding_refuses_cpu_tensors():
    import pytest
    import torch

    from paper_1502_04265_gb300 import _binding

    _binding.load(build_if_missing=True)
    with pytest.raises(ValueError):
        _binding._ptr(torch.zeros(3))
