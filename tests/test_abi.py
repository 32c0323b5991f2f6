"""The C-ABI library builds for sm_103a, loads without a GPU, and exports every
entry point include/ms.h declares; the binding wraps each of them.  No
compute call is made here."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    hdr = open(os.path.join(ROOT, "include", "ms.h")).read()
    return re.findall(r"^(?:ms_status|const char \*|int32_t)\s*(ms_\w+)\(", hdr, re.M)


@pytest.fixture(scope="module")
def lib():
    from paper_2001_01624_gb300 import build
    build.build()
    import paper_2001_01624_gb300 as pkg
    return pkg.lib()


def test_header_declares_entry_points():
    names = _declared()
    for required in ("ms_assemble_tpfa", "ms_build_basis", "ms_add_adaptive_basis", "ms_galerkin", "ms_solve"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_wraps_every_declared_symbol():
    from paper_2001_01624_gb300 import binding
    assert sorted(_declared()) == sorted(binding.exported_symbols())
    for n in _declared():
        assert callable(getattr(binding, n)), n


def test_abi_version_and_status_strings(lib):
    from paper_2001_01624_gb300 import binding as b
    assert b.ms_abi_version() == 10
    assert lib.ms_status_string(b.MS_ERR_NOT_CONVERGED) == b"not converged"


def test_library_built_for_sm103a(lib):
    from paper_2001_01624_gb300 import build
    assert "arch=compute_103a,code=sm_103a" in " ".join(build.ARCH)
