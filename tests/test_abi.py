"""Host-side checks of the C ABI (no GPU needed): libcf.so loads, exports
every function include/cf.h declares, and rejects bad arguments before any
CUDA work."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "cf.h")).read()
    return sorted(set(re.findall(r"^\s*(?:int|const char \*)\s*(cf_\w+)\s*\(", src, re.M)))


def test_library_exports_every_declared_symbol():
    import paper_2511_07418_b300 as cf
    names = _declared()
    assert len(names) >= 14
    for n in names:
        assert hasattr(cf._lib, n), n
    assert sorted(cf.EXPORTED) == names


def test_arguments_are_rejected_on_the_host():
    import paper_2511_07418_b300 as cf
    lib = cf._lib
    out = ctypes.c_void_p()
    assert lib.cf_build(None, None, None, 0, None, ctypes.byref(out)) == 1  # CF_EINVAL
    assert "hand" in cf._cf_last_error().decode()
    hd = cf.HandDesc(0, 3, 10)
    assert cf._cf_build(ctypes.byref(hd), None, None, 0, None, ctypes.byref(out)) == 1
    assert "n_fingers" in cf._cf_last_error().decode()
    pts = cf.Points(None, None, None, None, None, None, 0)
    prm = cf.score_params(T=4, k=7, mu=0.5, K=8, eps=0.01, centroid=[0, 0, 0], rho=0.05, seed=0)
    assert cf._cf_score(ctypes.byref(pts), 3, None, None, 1, ctypes.byref(prm), None, None, None, None, None) == 1
    assert "k=7" in cf._cf_last_error().decode()
    prm = cf.score_params(T=4, k=3, mu=0.5, K=16, eps=0.01, centroid=[0, 0, 0], rho=0.05, seed=0)
    assert cf._cf_score(ctypes.byref(pts), 3, None, None, 1, ctypes.byref(prm), None, None, None, None, None) == 1
    assert "> 32" in cf._cf_last_error().decode()
    assert cf._cf_query(None, ctypes.byref(pts), None, 0, None, None, None) == 1


def test_oracle_and_library_share_no_source():
    """The oracle is test infrastructure: the CUDA sources never include or
    name it, and the oracle never includes the library's headers."""
    csrc = os.path.join(ROOT, "paper_2511_07418_b300", "csrc")
    for f in os.listdir(csrc):
        s = open(os.path.join(csrc, f)).read()
        assert "oracle" not in s.lower(), f
    s = open(os.path.join(ROOT, "oracle", "cf_oracle.c")).read()
    assert '#include "cf' not in s
    py = open(os.path.join(ROOT, "paper_2511_07418_b300", "__init__.py")).read()
    assert "import oracle" not in py and "from oracle" not in py
