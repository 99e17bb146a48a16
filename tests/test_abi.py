"""The C-ABI library builds, loads without a GPU and exports every declared entry point."""
import os
import re
import subprocess

import pytest

from paper_1310_4502_gb300 import build as B
from paper_1310_4502_gb300 import hot

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "hot.h")


def declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(hot_[a-z_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    lib = B.build()
    names = declared()
    assert "hot_build_tree" in names and "hot_evaluate_forces" in names
    out = subprocess.run(["nm", "-D", "--defined-only", lib], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (hot_[a-z_]+)$", out, flags=re.M))
    assert set(names) <= exported, set(names) - exported
    assert set(names) == set(hot.EXPORTS)


def test_library_loads_and_reports_errors_without_gpu():
    L = hot.load()
    for name in hot.EXPORTS:
        assert hasattr(L, name)
    assert hot.strerror(hot.HOT_EINVAL) == "invalid argument"
    assert hot.strerror(hot.HOT_ESTATE) == "call out of order"
    # host-side bookkeeping only: callable without a device, nothing held yet
    assert hot.memory_stats() == (0, 0)


def test_binding_rejects_cpu_tensors():
    torch = pytest.importorskip("torch")

    class Fake:
        pass

    with pytest.raises(ValueError):
        hot._need(torch.zeros(3, dtype=torch.float64))
