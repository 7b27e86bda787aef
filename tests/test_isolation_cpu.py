"""The library and the oracle stay apart, and the library has no fallback.

* The package (Python binding, CUDA/C++ sources, headers) never imports, includes or loads
  anything from oracle/, and the oracle never imports the package: the two share only the
  seeded input generator (paper_1912_06636_gb300/synth.py), which the oracle side receives as
  plain arrays.
* Without the built libnao.so the binding raises instead of computing anything itself."""
import re
from pathlib import Path

import pytest

from paper_1912_06636_gb300 import nao

ROOT = Path(__file__).resolve().parents[1]
PKG = ROOT / "paper_1912_06636_gb300"


def _sources(root, suffixes):
    return [p for p in root.rglob("*") if p.suffix in suffixes and "lib" not in p.relative_to(root).parts]


def test_package_never_touches_the_oracle():
    bad = []
    for p in _sources(PKG, {".py"}):
        text = p.read_text()
        if re.search(r"^\s*(from\s+oracle\b|import\s+oracle\b)", text, flags=re.M) or "liboracle" in text:
            bad.append(str(p.relative_to(ROOT)))
    for p in _sources(PKG, {".cu", ".cpp", ".h", ".cuh"}) + _sources(ROOT / "include", {".h"}):
        text = p.read_text()
        if re.search(r'#\s*include\s*[<"][^>"]*oracle', text) or "or_" + "hamiltonian" in text:
            bad.append(str(p.relative_to(ROOT)))
    assert not bad, bad


def test_oracle_never_imports_the_package():
    for p in _sources(ROOT / "oracle", {".py", ".c", ".h"}):
        text = p.read_text()
        assert "paper_1912_06636_gb300" not in text, p
        assert "libnao" not in text and "nao.h" not in text, p


def test_missing_library_fails_loudly(monkeypatch):
    monkeypatch.setattr(nao, "_lib", None)
    monkeypatch.setattr(nao, "_LIB_PATH", PKG / "lib" / "no_such_libnao.so")
    with pytest.raises(ImportError):
        nao.load()
    with pytest.raises(ImportError):
        nao.nao_default_options()
