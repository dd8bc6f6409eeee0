"""The C ABI: the built library loads and exports every function that
include/parrep.h declares (no GPU needed, no compute call)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "parrep.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:[A-Za-z_][\w\s\*]*?)\b(parrep_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_entry_points():
    names = declared_functions()
    for n in ["parrep_create", "parrep_run", "parrep_histogram", "parrep_fim", "parrep_rer", "parrep_destroy",
              "parrep_ssa", "parrep_ssa_noalloc", "parrep_dephase", "parrep_cycle_log"]:
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_1705_06807_gb300 import build

    lib_path = build.build()
    lib = ctypes.CDLL(lib_path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    from paper_1705_06807_gb300 import _lib

    assert sorted(_lib.EXPORTS) == declared_functions()
    L = _lib.load()
    for n in _lib.EXPORTS:
        assert getattr(L, n).argtypes is not None or n in ("parrep_default_options",)


def test_product_path_fails_loudly_without_the_library(monkeypatch, tmp_path):
    from paper_1705_06807_gb300 import _lib

    monkeypatch.setattr(_lib, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(_lib, "_lib", None)
    with pytest.raises(ImportError):
        _lib.load()


def test_create_without_gpu_reports_an_error_code():
    """On a machine without a usable GPU the ABI returns ECUDA, it does not
    fall back to the CPU."""
    import torch

    if torch.cuda.is_available():
        pytest.skip("GPU present")
    from paper_1705_06807_gb300 import ParRep, ParRepError, configs as K

    with pytest.raises(ParRepError) as e:
        ParRep(K.schlogl_classic(), 64, 1.0, 1.0, x0=[85])
    assert e.value.code == -3
