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
    assert lib.snn_abi_version() == 8
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
                 lambda: abi.snn_test_wait_timeout(None, False, 16),
                 lambda: abi.snn_multi_run(None),
                 lambda: abi.snn_multi_post(None, [0]),
                 lambda: abi.snn_classifier_set_row_schedule(None, 0)):
        with pytest.raises(abi.SnnError) as e:
            call()
        assert e.value.status == abi.SNN_EINVAL


_STRUCTS = {"RaggedDesc": "snn_ragged_desc", "RewireStats": "snn_rewire_stats", "Adam": "snn_adam",
            "ClassifierDesc": "snn_classifier_desc", "Batch": "snn_batch", "TopoParams": "snn_topo_params",
            "TopoRewire": "snn_topo_rewire", "TopoState": "snn_topo_state", "DeeprGuide": "snn_deepr_guide",
            "TopoDerived": "snn_topo_derived", "MultiInstance": "snn_multi_instance"}


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


def test_c_caller_gets_the_printed_table_values(tmp_path, lib_path):
    """A plain C program linked against libsnnsp.so fills only the parameters Tab. 2 prints
    (g_max 0.2, A_+ = 0.1 g_max, B = 1.2, tau_+ 20 ms, tau_- 64 ms, tau_ref 5 ms) and gets
    the derived values the kernels use from the library: A_+ = 0.02, A_- = B A_+ tau_+ /
    tau_- = 0.0075, refractory steps 5 at h = 1 ms and 50 at h = 0.1 ms; and Adam's
    bias-correction products for step 3 (0.9^3, 0.999^3 by running products)."""
    import shutil
    import subprocess
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    src = tmp_path / "caller.c"
    src.write_text(r"""
#include <stdio.h>
#include <string.h>
#include "snnsp.h"
int main(void) {
    snn_topo_params p;
    memset(&p, 0, sizeof p);
    p.L = 32; p.L_f = 32; p.radius2 = 9; p.t_stim = 20;
    p.dt = 1.0; p.tau_m = 20.0; p.V_rest = -70.0; p.E_exc = 0.0; p.V_theta = -54.0; p.V_reset = -70.0;
    p.tau_s = 5.0; p.g_leak = 1.0; p.tau_ref = 5.0; p.f_base = 20.0; p.f_in = 100.0;
    p.g_max = 0.2; p.tau_plus = 20.0; p.tau_minus = 64.0; p.A_plus_rel = 0.1; p.B = 1.2;
    snn_topo_derived d;
    if (snn_topo_derive(&p, &d) != SNN_OK) return 1;
    printf("%d %.17g %.17g\n", d.n_ref, d.A_plus, d.A_minus);
    p.dt = 0.1;
    if (snn_topo_derive(&p, &d) != SNN_OK) return 2;
    printf("%d\n", d.n_ref);
    p.tau_ref = -1.0;
    if (snn_topo_derive(&p, &d) != SNN_EINVAL) return 3;
    double b[2];
    if (snn_adam_bias(0.9, 0.999, 3, b) != SNN_OK) return 4;
    printf("%.17g %.17g\n", b[0], b[1]);
    return 0;
}
""")
    exe = tmp_path / "caller"
    libdir = os.path.dirname(lib_path)
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe),
                    "-L", libdir, "-lsnnsp", f"-Wl,-rpath,{libdir}"], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()
    assert int(out[0]) == 5 and int(out[3]) == 50
    assert float(out[1]) == pytest.approx(0.02, rel=1e-15)
    assert float(out[2]) == pytest.approx(1.2 * 0.02 * 20.0 / 64.0, rel=1e-15)
    assert float(out[2]) == pytest.approx(0.0075, rel=1e-15)
    assert float(out[4]) == 0.9 * 0.9 * 0.9 and float(out[5]) == 0.999 * 0.999 * 0.999
