"""The C-ABI library loads and exports every entry point that include/dlmcol.h declares (CPU)."""
import ctypes
import os

import pytest

from paper_2109_05948_gb300 import build as libbuild
from paper_2109_05948_gb300 import dlmcol


@pytest.fixture(scope="module")
def lib():
    libbuild.build()
    return dlmcol.lib()


def test_header_declares_the_boundary():
    syms = dlmcol.header_symbols()
    for name in ("dlm_tabucol_batch", "dlm_create", "dlm_sync", "dlm_graph_create"):
        assert name in syms


def test_every_declared_symbol_is_exported(lib):
    missing = [s for s in dlmcol.header_symbols() if not hasattr(lib, s)]
    assert missing == []


def test_binding_declares_signatures_for_every_symbol(lib):
    assert [s for s in dlmcol.header_symbols() if s not in dlmcol._SIGS] == []


def test_library_has_no_torch_or_oracle_dependency(lib):
    """The library's dynamic dependencies (ELF NEEDED entries) and exported symbols name neither
    torch nor the oracle."""
    import shutil
    import subprocess

    if not shutil.which("readelf") or not shutil.which("nm"):
        pytest.skip("readelf / nm not available")
    so = dlmcol.LIB_PATH
    dyn = subprocess.run(["readelf", "-d", so], capture_output=True, text=True, check=True).stdout
    needed = [ln.split("[", 1)[1].rstrip("]") for ln in dyn.splitlines() if "(NEEDED)" in ln]
    assert needed and not [x for x in needed if "torch" in x or "c10" in x or "oracle" in x], needed
    syms = subprocess.run(["nm", "-D", "--defined-only", so], capture_output=True, text=True, check=True).stdout
    names = [ln.split()[-1] for ln in syms.splitlines() if ln.strip()]
    assert "dlm_tabucol_batch" in names
    assert not [x for x in names if x.startswith("oracle_")]


def test_create_without_gpu_fails_cleanly(lib):
    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    assert lib.dlm_create(ctypes.byref(h), 0, None) in (dlmcol.DLM_ECUDA, dlmcol.DLM_EUNSUPPORTED)
    assert not h.value


def test_oracle_is_not_imported_by_the_product():
    import sys

    pkg = os.path.dirname(dlmcol.__file__)
    for fn in os.listdir(pkg):
        if fn.endswith(".py"):
            src = open(os.path.join(pkg, fn)).read()
            assert "import oracle" not in src and "from oracle" not in src, fn
