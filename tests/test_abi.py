"""The C ABI library builds for sm_103a and exports every function that
include/vsr.h declares (no GPU needed: nothing is called)."""
import ctypes
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    with open(os.path.join(ROOT, "include", "vsr.h")) as f:
        src = f.read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(vsr_[a-z_0-9]+)\s*\(", src)))


@pytest.mark.skipif(shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"),
                    reason="no CUDA toolkit")
def test_library_exports_every_declared_symbol():
    from paper_2003_10558_gb300 import build, vsr
    path = build.build()
    lib = ctypes.CDLL(path)
    names = _declared()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(vsr.EXPORTS)
    # status strings need no device
    L = vsr.load()
    assert L.vsr_status_str(0) == b"ok"
    assert L.vsr_version().startswith(b"vsr")


def test_product_does_not_import_oracle():
    pkg = os.path.join(ROOT, "paper_2003_10558_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                with open(os.path.join(dirpath, f)) as fh:
                    txt = fh.read()
                assert "import oracle" not in txt and "from oracle" not in txt and "vsr_oracle" not in txt, f
