"""The C-ABI library builds, loads without a GPU, and exports every symbol include/fhmg.h declares."""
import ctypes
import os
import re

import pytest

from tests.conftest import ROOT


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(fhmg_\w+)\s*\(", src))
    return names


@pytest.fixture(scope="module")
def libpath():
    from paper_1706_07632_gb300 import build
    return build.build()


def test_exports_every_declared_symbol(libpath):
    names = _declared()
    assert len(names) >= 20
    L = ctypes.CDLL(libpath)
    missing = [n for n in sorted(names) if not hasattr(L, n)]
    assert not missing, missing


def test_binding_covers_header(libpath):
    import paper_1706_07632_gb300 as fh
    assert _declared() <= set(fh._SIGS)


def test_invalid_arguments_are_rejected_on_host(libpath):
    import paper_1706_07632_gb300 as fh
    with pytest.raises(fh.FhmgError) as e:
        fh.HMatrix(1.5, 2.0, 1.0, 64, 64, 0, 1e-10)
    assert e.value.status == fh.FHMG_EINVAL
    with pytest.raises(fh.FhmgError):
        fh.HMatrix(0.5, 2.0, 1.0, 96, 64, 0, 1e-10)       # M / leaf not a power of two
    with pytest.raises(fh.FhmgError):
        fh.HMatrix(0.5, 0.5, 1.0, 64, 64, 0, 1e-10)       # gamma < 1
