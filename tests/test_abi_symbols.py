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


def _null_args(argtypes):
    import ctypes as C
    ints = (C.c_int, C.c_int32, C.c_int64, C.c_uint64, C.c_uint32, C.c_size_t)
    return [0 if a in ints else 0.0 if a in (C.c_double, C.c_float) else None for a in argtypes]


def test_null_handles_and_pointers_are_rejected_without_a_device_call(lib):
    # every entry point checks its handles and pointers before touching the
    # device: destroy/release of NULL is a no-op, everything else NYS_EINVAL
    from paper_2411_08178_gb300 import _abi
    for name, (_, argtypes) in _abi.PROTOTYPES.items():
        if name in ("nys_version", "nys_last_error"):
            continue
        r = getattr(lib, name)(*_null_args(argtypes))
        if name.endswith(("_destroy", "_release")) or name == "nys_destroy":
            assert r == _abi.NYS_OK, name
        else:
            assert r == _abi.NYS_EINVAL, (name, r)
        assert isinstance(lib.nys_last_error(None), bytes)


def test_binding_rejects_host_and_strided_tensors():
    import torch
    from paper_2411_08178_gb300 import api
    with pytest.raises(ValueError):
        api._ptr(torch.zeros(4))
    with pytest.raises(ValueError):
        api.dtype_code(torch.zeros(4, dtype=torch.int32))
