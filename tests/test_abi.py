"""CPU-side checks of the C ABI: the library builds, loads and exports every
entry point declared in include/mr.h (no compute call without a GPU)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"^\s*(?:[A-Za-z_][\w\s\*]*?)\b(mr_\w+)\s*\(", src, flags=re.M))
    return names


def test_library_builds_and_exports_every_declared_symbol():
    import paper_1309_0215_gb300 as pkg
    pkg.build()
    lib = pkg.load()
    declared = _declared()
    assert declared, "no declarations found"
    missing = [n for n in sorted(declared) if not hasattr(lib, n)]
    assert not missing, missing
    assert set(pkg.EXPORTS) <= declared


def test_status_strings_without_gpu():
    import paper_1309_0215_gb300 as pkg
    lib = pkg.load()
    for s in range(9):
        assert lib.mr_status_str(s).startswith(b"MR_")


def test_create_fails_cleanly_without_gpu():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import paper_1309_0215_gb300 as pkg
    with pytest.raises(RuntimeError):
        pkg.Context()
