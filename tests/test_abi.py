"""CPU checks of the boundary: the C-ABI library loads without a GPU and
exports every function that include/dnasa.h declares; the binding refuses
CPU tensors (there is no CPU fallback)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "dnasa.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s+\**([a-z_][a-z0-9_]*)\s*\(",
                       src, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ["dnasa_create", "dnasa_destroy", "dnasa_pack", "sa_build", "lcp_build", "sa_lcp_build",
              "overlap_search", "assemble"]:
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_1404_3456_gb300 import build

    lib_path = build.build()
    lib = ctypes.CDLL(lib_path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_signatures_cover_header():
    from paper_1404_3456_gb300 import binding

    assert set(declared_functions()) <= set(binding.exported_symbols())


def test_binding_rejects_cpu_tensors():
    torch = pytest.importorskip("torch")
    from paper_1404_3456_gb300 import binding

    with pytest.raises(ValueError):
        binding._ptr(torch.zeros(4, dtype=torch.uint8))


def test_oracle_is_not_imported_by_the_product():
    """The product path never imports the oracle (and vice versa)."""
    pkg = os.path.join(ROOT, "paper_1404_3456_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f
                assert "dnasa_oracle" not in txt, f
    for f in os.listdir(os.path.join(ROOT, "oracle")):
        if f.endswith((".py", ".c")):
            txt = open(os.path.join(ROOT, "oracle", f)).read()
            assert "paper_1404_3456_gb300.binding" not in txt and "libdnasa" not in txt, f
