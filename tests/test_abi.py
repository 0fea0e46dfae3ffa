"""CPU-side checks of the boundary: the library builds for sm_103a, loads,
exports every entry point include/knit.h declares, and the CUDA path shares
no code with the oracle."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _header_functions():
    src = open(os.path.join(ROOT, "include", "knit.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(knit_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_1010_2627_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_library_exports_every_declared_symbol(lib):
    names = _header_functions()
    assert {"knit_system_create", "knit_transmission", "knit_ldos",
            "knit_lead_selfenergy"} <= set(names)
    for n in names:
        assert hasattr(lib, n), n
    out = subprocess.run(["nm", "-D", "--defined-only", lib._name], capture_output=True,
                         text=True).stdout
    for n in names:
        assert re.search(rf"\sT\s{n}$", out, re.M), n


def test_version_string_without_gpu(lib):
    lib.knit_version.restype = ctypes.c_char_p
    assert b"sm_103a" in lib.knit_version()


def test_binding_signatures_cover_header():
    from paper_1010_2627_gb300 import knit
    assert set(_header_functions()) == set(knit._SIGS)


def test_oracle_and_cuda_path_are_independent():
    csrc = os.path.join(ROOT, "paper_1010_2627_gb300", "csrc")
    for f in os.listdir(csrc):
        text = open(os.path.join(csrc, f)).read()
        assert "oracle" not in text.lower(), f
    for f in ("knit.py", "build.py", "inputs.py", "__init__.py"):
        text = open(os.path.join(ROOT, "paper_1010_2627_gb300", f)).read()
        assert "import oracle" not in text and "from oracle" not in text, f
    for f in os.listdir(os.path.join(ROOT, "oracle")):
        if f.endswith((".py", ".c", ".h")):
            text = open(os.path.join(ROOT, "oracle", f)).read()
            assert not re.search(r"^\s*(import|from)\s+paper_1010_2627_gb300", text, re.M), f
            assert "knit.h" not in text and "libknit" not in text, f


def test_binding_fails_loudly_without_library(tmp_path, monkeypatch):
    from paper_1010_2627_gb300 import knit
    monkeypatch.setattr(knit, "_lib", None)
    monkeypatch.setattr(knit, "lib_path", lambda: str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError, match="no fallback"):
        knit.load()


def test_every_declaration_is_documented():
    """Each entry point of include/knit.h has its own comment right above it
    (what it computes, argument layout, ownership, errors)."""
    lines = open(os.path.join(ROOT, "include", "knit.h")).read().split("\n")
    missing = []
    for i, line in enumerate(lines):
        m = re.match(r"^(?:knit_status|int64_t|const char \*)\s*(knit_\w+)\s*\(", line)
        if not m:
            continue
        j = i - 1
        while j >= 0 and not lines[j].strip():
            j -= 1
        if not lines[j].rstrip().endswith("*/"):
            missing.append(m.group(1))
    assert not missing, missing


def _header_arities():
    src = open(os.path.join(ROOT, "include", "knit.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    out = {}
    for m in re.finditer(r"\b(knit_[a-z0-9_]+)\s*\(([^;{]*?)\)\s*;", src):
        name, params = m.group(1), " ".join(m.group(2).split())
        out[name] = 0 if params in ("", "void") else params.count(",") + 1
    return out


def test_binding_argument_counts_match_header():
    """The ctypes signatures take as many arguments as the C declarations
    (a mismatch would pass garbage through the ABI)."""
    from paper_1010_2627_gb300 import knit
    ar = _header_arities()
    assert set(ar) == set(knit._SIGS)
    bad = {n: (ar[n], len(knit._SIGS[n][1])) for n in ar if ar[n] != len(knit._SIGS[n][1])}
    assert not bad, bad
