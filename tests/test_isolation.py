"""The oracle and the CUDA path share no code, and the product path has no CPU fallback.

- nothing in the package (Python binding, CUDA sources, headers) imports, includes or loads
  anything under oracle/;
- the oracle imports nothing from the package (the tests hand it the seeded inputs);
- the oracle's C source includes only its own header and the C standard library;
- the binding raises when the CUDA library is missing instead of computing anything itself.
"""
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_1101_0423_gb300")


def package_sources():
    files = []
    for pat in ("*.py", "csrc/*.cu", "csrc/*.cuh", "csrc/*.h"):
        files += glob.glob(os.path.join(PKG, pat))
    files += glob.glob(os.path.join(ROOT, "include", "*.h"))
    return files


def code_lines(path):
    """Source lines with comments and docstrings removed (a comment may mention the oracle)."""
    text = open(path).read()
    if path.endswith(".py"):
        text = re.sub(r'"""[\s\S]*?"""', "", text)
        return [ln.split("#", 1)[0] for ln in text.splitlines()]
    text = re.sub(r"/\*[\s\S]*?\*/", "", text)
    return [ln.split("//", 1)[0] for ln in text.splitlines()]


def test_package_does_not_use_the_oracle():
    files = package_sources()
    assert len(files) > 8
    for f in files:
        for ln in code_lines(f):
            assert not re.search(r"\boracle\b|dwf_oracle", ln), f"{os.path.relpath(f, ROOT)}: {ln.strip()}"


def test_oracle_does_not_use_the_package():
    for f in glob.glob(os.path.join(ROOT, "oracle", "*.py")) + glob.glob(os.path.join(ROOT, "oracle", "*.[ch]")):
        for ln in code_lines(f):
            assert "paper_1101_0423_gb300" not in ln and "csrc" not in ln, f"{os.path.relpath(f, ROOT)}: {ln.strip()}"


def test_oracle_c_includes_only_its_header_and_libc():
    allowed = {"dwf_oracle.h", "complex.h", "math.h", "stdlib.h", "string.h", "stddef.h", "stdio.h", "stdint.h"}
    for f in glob.glob(os.path.join(ROOT, "oracle", "*.[ch]")):
        for inc in re.findall(r'#include\s*[<"]([^>"]+)[>"]', open(f).read()):
            assert inc in allowed, f"{os.path.basename(f)} includes {inc}"


def test_binding_raises_without_the_library(monkeypatch, tmp_path):
    from paper_1101_0423_gb300 import dwf
    monkeypatch.setattr(dwf, "_lib", None)
    monkeypatch.setattr(dwf, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError, match="CUDA library missing"):
        dwf.load(build_if_missing=False)
