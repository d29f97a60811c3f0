"""Host-side checks of the C ABI: the library builds for sm_103a and exports
every function that include/axpcg.h declares (no compute calls)."""
import ctypes
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "axpcg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ax_[a-z_0-9]+)\s*\(", src)))


@pytest.mark.skipif(shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"),
                    reason="no CUDA toolkit")
def test_library_builds_and_exports_header_symbols():
    import paper_1002_3094_gb300 as P
    lib_path = P.build()
    lib = ctypes.CDLL(lib_path)
    names = _declared()
    assert len(names) >= 10
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(P.EXPORTED)
    P.load_library()
    assert "sm_103a" in P.ax_version()
    assert P.ax_status_string(P.AX_ERR_INVALID_ARG) == "invalid argument"


def test_binding_has_no_cpu_fallback():
    """The package never imports the oracle, so the product path cannot route
    through it; its only compute is the CUDA library."""
    pkg = os.path.join(ROOT, "paper_1002_3094_gb300")
    for f in os.listdir(pkg):
        if f.endswith(".py"):
            src = open(os.path.join(pkg, f)).read()
            assert "import oracle" not in src and "from oracle" not in src, f
