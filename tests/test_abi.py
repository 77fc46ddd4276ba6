"""The C ABI library: builds, loads, exports every symbol include/prnu.h
declares, and fails loudly when missing (CPU only; no compute calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "prnu.h")


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(prnu_\w+)\s*\(", text)))


@pytest.fixture(scope="module")
def built():
    from paper_1909_04573_gb300 import build
    build.build()
    return build.LIB


def test_header_declarations_match_binding():
    from paper_1909_04573_gb300 import prnu as P
    assert _declared() == sorted(P.EXPORTS)


def test_library_exports_every_declared_symbol(built):
    L = ctypes.CDLL(built)
    for name in _declared():
        assert hasattr(L, name), name


def test_binding_loads_and_default_params(built):
    from paper_1909_04573_gb300 import prnu as P
    p = P.default_params()
    assert (p.levels, p.sigma0, p.n_windows, list(p.windows)) == (4, 3.0, 4, [3, 5, 7, 9])
    assert p.pad_mode == 0 and p.dtype == 0


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    from paper_1909_04573_gb300 import prnu as P
    monkeypatch.setattr(P, "LIB_PATH", str(tmp_path / "nope.so"))
    monkeypatch.setattr(P, "_lib", None)
    with pytest.raises(ImportError):
        P.lib()


def test_product_package_never_imports_the_oracle():
    pkg = os.path.join(ROOT, "paper_1909_04573_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(from|import)\s+oracle\b", text, flags=re.M), f
                assert "prnu_oracle" not in text, f
