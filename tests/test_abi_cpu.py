"""CPU-side checks of the C ABI: the library builds, loads without a GPU and
exports every entry point include/sph.h declares; the binding's structure
mirrors the header."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "sph.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(sph_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_1603_02421_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("sph_init", "sph_add_particles", "sph_inflow", "sph_step", "sph_run",
              "sph_breakup_length", "sph_destroy", "sph_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing


def test_binding_covers_every_declared_symbol():
    from paper_1603_02421_gb300 import binding
    assert set(_declared()) <= set(binding._SIGS)
    for n in _declared():
        assert hasattr(binding, n) or n in ("sph_last_error",)


def test_params_struct_matches_header():
    from paper_1603_02421_gb300 import binding
    src = open(os.path.join(ROOT, "include", "sph.h")).read()
    body = src[src.index("typedef struct {", src.index("enum { SPH_FLUID")):
               src.index("} sph_params;")]
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    fields = []
    for decl in body.split(";"):
        decl = decl.strip().replace("typedef struct {", "").strip()
        if not decl:
            continue
        types = {"int", "double", "long", "void", "unsigned", "*"}
        toks = [t for t in decl.replace("*", " * ").replace(",", " , ").split()
                if t not in types]
        fields += [t for t in toks if t != ","]
    assert fields == [f for f, _ in binding.sph_params._fields_]


def test_init_without_gpu_fails_cleanly(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_1603_02421_gb300 import binding
    from paper_1603_02421_gb300 import workloads as wl
    p = binding.make_params(wl.test_params(), capacity=16)
    with pytest.raises(binding.SphError) as e:
        binding.sph_init(p)
    assert e.value.status in (-4, -1)


def test_product_path_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_1603_02421_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "oracle" not in re.sub(r"#.*|//.*", "", txt).lower() or f == "workloads.py"
