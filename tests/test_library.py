"""Host-side checks of the C-ABI library: it builds, loads and exports every
entry point that include/scocg.h declares.  No compute call (no GPU here)."""
import ctypes
import re
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parents[1]


def declared_functions():
    text = (ROOT / "include" / "scocg.h").read_text()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(scocg_[a-z_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def so():
    from paper_0802_0748_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ["scocg_create_csr", "scocg_create_hubbard", "scocg_solve", "scocg_grad",
              "scocg_solve_full", "scocg_apply", "scocg_destroy", "scocg_strerror"]:
        assert n in names


def test_library_exports_every_declared_symbol(so):
    lib = ctypes.CDLL(str(so))
    for n in declared_functions():
        assert hasattr(lib, n), n


def test_binding_names_match_header(so):
    from paper_0802_0748_gb300 import scocg
    for n in declared_functions():
        assert hasattr(scocg, n), n


def test_strerror_without_gpu(so):
    from paper_0802_0748_gb300 import scocg
    assert scocg.strerror(0) == "ok"
    assert "symmetric" in scocg.strerror(-6)
    assert scocg.strerror(12345) == "unknown status"


def test_opts_struct_matches_header():
    """ctypes mirror of scocg_opts has the header's fields in order."""
    from paper_0802_0748_gb300 import scocg
    text = (ROOT / "include" / "scocg.h").read_text()
    body = text[text.index("typedef struct {\n    int precision;"):text.index("} scocg_opts;")]
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    fields = re.findall(r"\b(?:int|double)\s+(\w+);", body)
    assert fields == [f for f, _ in scocg.Opts._fields_]


def test_product_path_fails_loudly_without_library(tmp_path, monkeypatch):
    from paper_0802_0748_gb300 import scocg
    monkeypatch.setattr(scocg, "_lib", None)
    monkeypatch.setattr(scocg, "LIB_PATH", tmp_path / "missing.so")
    with pytest.raises(RuntimeError, match="not built"):
        scocg.lib()
