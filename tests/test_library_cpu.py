"""CPU-side checks of the CUDA library: it builds for sm_103a, loads without a GPU, exports
every entry point declared in include/gazemap.h, and refuses to run without an sm_103a device
(no CPU fallback). No kernel is launched here."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "gazemap.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(gm_[a-z0-9_]+)\s*\(", src)))


def test_library_builds_and_exports_every_declared_symbol():
    from paper_2601_07571_gb300 import build
    path = build.build()
    assert os.path.exists(path)
    import ctypes
    lib = ctypes.CDLL(path)
    declared = _declared()
    assert len(declared) >= 20
    missing = [n for n in declared if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    from paper_2601_07571_gb300 import gazemap
    missing = [n for n in _declared() if n not in gazemap._SIGS]
    assert not missing, missing


def test_no_cpu_fallback_without_gpu():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import paper_2601_07571_gb300 as G
    with pytest.raises(G.GazeMapError):
        G.gm_create(0)
