"""The C-ABI library loads and exports every symbol declared in include/slim.h
(no compute call: these run without a GPU)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as g
    g.build()
    from paper_2605_16082_gb300 import slim
    return slim.lib()


def header_symbols():
    src = open(os.path.join(ROOT, "include", "slim.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(slim_[a-z0-9_]+)\s*\(", src)))


def test_header_symbols_exported(lib):
    syms = header_symbols()
    assert len(syms) >= 15
    for s in syms:
        assert hasattr(lib, s), s


def test_binding_lists_every_symbol():
    from paper_2605_16082_gb300 import slim
    assert sorted(slim.EXPORTED) == header_symbols()


def test_params_default_and_status_strings(lib):
    from paper_2605_16082_gb300 import slim
    p = slim.slim_params_default()
    assert p.g == 9.81 and p.penalty_v == 4.0 and p.tile_prisms == 256
    assert slim.slim_status_string(0) == "ok"
    assert "argument" in slim.slim_status_string(1)


def test_null_arguments_are_rejected(lib):
    import ctypes as C
    from paper_2605_16082_gb300 import slim
    assert lib.slim_params_default(None) == 1
    out = C.c_void_p()
    assert lib.slim_mesh_create(None, 0, None, 0, None, None, None, 0, None, 256, C.byref(out)) == 1
    assert out.value is None
    assert lib.slim_state_alloc(None, 0, None, C.byref(out)) == 1
    assert lib.slim_step(None, 0.0, 1.0, None) == 1
    assert lib.slim_state_check(None, None) == 1
