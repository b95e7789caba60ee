"""The C-ABI library loads without a GPU and exports every entry point include/vmesh.h
declares; the binding refuses to run without CUDA instead of falling back to the CPU; the
product package never loads the oracle.  No CUDA call is made here."""
import ast
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    hdr = open(os.path.join(ROOT, "include", "vmesh.h")).read()
    return sorted(set(re.findall(r"^vm_status\s+(vm_\w+)\s*\(", hdr, flags=re.M)))


def test_library_exports_every_declared_entry_point():
    from paper_1803_03949_b300 import build as vbuild
    from paper_1803_03949_b300.vmesh import EXPORTS, load_library

    vbuild.build()
    lib = load_library()
    names = _declared()
    assert len(names) >= 18
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(EXPORTS) == names


def test_missing_library_fails_loudly(tmp_path):
    from paper_1803_03949_b300 import vmesh

    with pytest.raises(ImportError):
        _load_fresh(vmesh, str(tmp_path / "nope.so"))


def _load_fresh(vmesh, path):
    saved = vmesh._lib
    vmesh._lib = None
    try:
        return vmesh.load_library(path)
    finally:
        vmesh._lib = saved


def test_no_cpu_fallback_without_cuda():
    import torch

    from paper_1803_03949_b300 import Volume

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(RuntimeError):
        Volume(0.01, 0.04, 1 << 10, 64, 1024, 1024)


def test_product_package_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_1803_03949_b300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if not f.endswith(".py"):
                continue
            tree = ast.parse(open(os.path.join(dirpath, f)).read())
            for node in ast.walk(tree):
                if isinstance(node, ast.Import):
                    assert all(not a.name.startswith("oracle") for a in node.names), f
                if isinstance(node, ast.ImportFrom):
                    assert not (node.module or "").startswith("oracle"), f
    for dirpath, _, files in os.walk(os.path.join(pkg, "csrc")):
        for f in files:
            assert "oracle" not in open(os.path.join(dirpath, f)).read().lower() or f.endswith(".md"), f
