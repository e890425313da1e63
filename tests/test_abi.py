"""The C-ABI library builds for sm_103a, loads, and exports every symbol that
include/snnsp.h declares (no GPU needed: nothing here launches a kernel)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_symbols():
    src = open(os.path.join(ROOT, "include", "snnsp.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(snn_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib_path():
    from paper_2510_19764_gb300 import build
    return build.build()


def test_header_declares_expected_calls():
    decl = _declared_symbols()
    for name in ("snn_create_ragged", "snn_step_neurons", "snn_propagate", "snn_eprop_update", "snn_rewire_deepr",
                 "snn_rewire_topo"):
        assert name in decl


def test_library_exports_every_declared_symbol(lib_path):
    lib = ctypes.CDLL(lib_path)
    for name in _declared_symbols():
        assert hasattr(lib, name), name


def test_binding_covers_every_declared_symbol(lib_path):
    from paper_2510_19764_gb300 import abi
    assert sorted(abi.EXPORTED) == _declared_symbols()
    lib = abi.load()
    assert lib.snn_abi_version() == 5
    for name in abi.EXPORTED:
        assert callable(getattr(abi, name)), name


def test_argument_errors_are_synchronous_and_need_no_gpu(lib_path):
    from paper_2510_19764_gb300 import abi
    d = abi.RaggedDesc()
    d.P, d.Q, d.C = 0, 4, 4
    with pytest.raises(abi.SnnError) as e:
        abi.snn_create_ragged(d, False)
    assert e.value.status == abi.SNN_EINVAL
    assert "P, Q, C" in abi.load().snn_last_error().decode()
    with pytest.raises(abi.SnnError):
        abi.snn_eprop_update(None, None, 0, None)


def test_struct_layouts_match_header():
    from paper_2510_19764_gb300 import abi
    assert ctypes.sizeof(abi.RaggedDesc) == 24 + 8 * 8 + 8
    assert ctypes.sizeof(abi.RewireStats) == 32
    assert ctypes.sizeof(abi.Adam) == 64
    assert ctypes.sizeof(abi.ClassifierDesc) == 168
    assert ctypes.sizeof(abi.Batch) == 8 + 19 * 8
    assert ctypes.sizeof(abi.TopoParams) == 24 + 15 * 8
    assert ctypes.sizeof(abi.TopoRewire) == 6 * 8 + 8
    assert ctypes.sizeof(abi.TopoState) == 10 * 8
