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
    assert lib.snn_abi_version() == 6
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
    # the entry points added for the analysis, the DEEP R variants and the row updates
    # check their handles before touching the device
    for call in (lambda: abi.snn_topo_connectivity(None, 8),
                 lambda: abi.snn_ragged_set_deepr_guide(None, abi.DeeprGuide()),
                 lambda: abi.snn_ragged_add_row(None, None),
                 lambda: abi.snn_ragged_remove_row(None, None),
                 lambda: abi.snn_test_wait_timeout(None, False, 16)):
        with pytest.raises(abi.SnnError) as e:
            call()
        assert e.value.status == abi.SNN_EINVAL


_STRUCTS = {"RaggedDesc": "snn_ragged_desc", "RewireStats": "snn_rewire_stats", "Adam": "snn_adam",
            "ClassifierDesc": "snn_classifier_desc", "Batch": "snn_batch", "TopoParams": "snn_topo_params",
            "TopoRewire": "snn_topo_rewire", "TopoState": "snn_topo_state", "DeeprGuide": "snn_deepr_guide"}


def test_struct_layouts_match_header(tmp_path):
    """Every ctypes structure has the size and field offsets that a C compiler gives the
    header's structure of the same fields (compiled with gcc from include/snnsp.h)."""
    import shutil
    import subprocess
    from paper_2510_19764_gb300 import abi
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "snnsp.h"', "int main(void) {"]
    for py, c in _STRUCTS.items():
        lines.append(f'printf("{py} size %zu\\n", sizeof({c}));')
        for f in getattr(abi, py)._fields_:
            lines.append(f'printf("{py} {f[0]} %zu\\n", offsetof({c}, {f[0]}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = {}
    for ln in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.splitlines():
        py, field, val = ln.split()
        got[(py, field)] = int(val)
    for py in _STRUCTS:
        cls = getattr(abi, py)
        assert ctypes.sizeof(cls) == got[(py, "size")], py
        for f in cls._fields_:
            assert getattr(cls, f[0]).offset == got[(py, f[0])], (py, f[0])
