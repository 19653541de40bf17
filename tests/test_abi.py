"""The C ABI library builds for sm_103a, loads without a GPU and exports every declared call."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names += re.findall(r"\b(esmp2_[a-z0-9_]+)\s*\(", txt)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2003_12923_gb300 import build
    from paper_2003_12923_gb300 import esmp2
    build.build()
    return esmp2.load()


def test_declared_symbols_exported(lib):
    names = _declared()
    assert len(names) >= 12
    for n in names:
        assert hasattr(lib, n), n


def test_binding_covers_abi():
    from paper_2003_12923_gb300 import esmp2
    assert sorted(esmp2.EXPORTS) == sorted(n for n in _declared() if n in esmp2.EXPORTS)
    assert set(_declared()) <= set(esmp2.EXPORTS)


def test_missing_library_fails_loudly(tmp_path):
    from paper_2003_12923_gb300 import esmp2
    with pytest.raises(OSError):
        esmp2.load(str(tmp_path / "nope.so"))
