"""The C-ABI library loads and exports every function that include/nys.h declares."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "nys.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^(?:const\s+)?(?:int|char\s*\*|const\s+char\s*\*)\s*\**\s*([a-z_][a-z0-9_]*)\s*\(",
                       text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as g
    g.build()
    from paper_2411_08178_gb300 import _abi
    return _abi.load()


def test_header_parses():
    names = declared_functions()
    assert "nys_sketch" in names and "pgd_step" in names and "precond_apply" in names
    assert len(names) >= 25


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_declares_every_symbol(lib):
    from paper_2411_08178_gb300 import _abi
    assert set(declared_functions()) == set(_abi.PROTOTYPES)


def test_version_and_error_without_gpu(lib):
    assert b"sm_103a" in lib.nys_version()
    # no device call: the global error string is readable
    assert isinstance(lib.nys_last_error(None), bytes)
    # invalid arguments are rejected before any CUDA call
    assert lib.nys_create(None, 0, None) == 1
