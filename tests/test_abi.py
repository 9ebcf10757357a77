"""The C-ABI library builds for sm_103a, loads, and exports every function
that include/mgglam.h declares (no GPU needed: nothing is called); without
it the binding raises instead of falling back to anything."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    src = open(os.path.join(ROOT, "include", "mgglam.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*[A-Za-z_][\w \*]*?\b((?:mg|pm|dpm)_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2110_00566_gb300 import binding, build
    build.build()
    return binding.lib()


def test_header_declares_the_boundary():
    names = header_functions()
    for n in ("mg_solve_dgp", "mg_solve_kmouflage", "pm_cic_deposit", "pm_step", "mg_solve_adjoint",
              "mg_ctx_create", "mg_ctx_destroy"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in header_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_the_header(lib):
    from paper_2110_00566_gb300 import binding
    assert set(binding.DECLARED) == set(header_functions())


def test_product_package_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_2110_00566_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f
                assert "liboracle" not in txt and "mg_oracle" not in txt, f


def test_library_is_built_for_sm_103a(lib):
    from paper_2110_00566_gb300 import build
    assert "arch=compute_103a,code=sm_103a" in " ".join(build.ARCH)


def test_missing_library_fails_loudly(monkeypatch):
    """Without the built library every entry point raises: there is no CPU
    fallback for the product path to route through."""
    from paper_2110_00566_gb300 import binding as B
    monkeypatch.setattr(B, "_lib", None)
    monkeypatch.setattr(B, "LIB_PATH", os.path.join(os.path.dirname(B.LIB_PATH), "no_such_libmgglam.so"))
    with pytest.raises(ImportError, match="no CPU fallback"):
        B.lib()
    with pytest.raises(ImportError):
        B.Context(0)
