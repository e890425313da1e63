"""ctypes binding of include/snnsp.h — argument marshalling only.

Every function below has the name of the C entry point it calls, takes the same
arguments (torch CUDA tensors stand in for device pointers, a torch.cuda.Stream or None
for the stream) and raises SnnError when the C call returns a non-zero status.  All
computation happens in libsnnsp.so; importing this module on a machine where the
library cannot be loaded raises instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libsnnsp.so")

SNN_OK, SNN_EINVAL, SNN_ENOMEM, SNN_ECAPACITY, SNN_ECUDA, SNN_ETIMEOUT, SNN_ESTATE = 0, -1, -2, -3, -4, -5, -6
SNN_F32, SNN_F64 = 0, 1
SNN_EPROP_GRAD, SNN_EPROP_APPLY = 0, 1
SNN_FIXED_FRAC_BITS = 40
SNN_STEP_INPUTS_READY = 1
SNN_STEP_PACKED_READY = 2
SNN_ROWS_PAIRS, SNN_ROWS_PER_WARP, SNN_ROWS_PER_BLOCK, SNN_ROWS_WIDE, SNN_ROWS_QUAD = 0, 1, 2, 3, 4
SNN_MULTI_HOST_POSTS = 1

EXPORTED = [
    "snn_last_error", "snn_abi_version", "snn_create_ragged", "snn_destroy_ragged", "snn_ragged_status",
    "snn_propagate", "snn_rewire_deepr", "snn_create_classifier", "snn_destroy_classifier", "snn_step_neurons",
    "snn_eprop_update", "snn_topo_input", "snn_topo_neurons", "snn_stdp_update", "snn_rewire_topo", "snn_topo_run",
    "snn_philox", "snn_rewire_deepr_noalloc", "snn_classifier_set_schedule", "snn_rewire_deepr_dev",
    "snn_draw_inputs", "snn_step_neurons_ex", "snn_topo_connectivity", "snn_ragged_set_deepr_guide",
    "snn_test_wait_timeout", "snn_ragged_add_row", "snn_ragged_remove_row", "snn_adam_bias", "snn_topo_derive",
    "snn_classifier_set_row_schedule", "snn_multi_create", "snn_multi_destroy", "snn_multi_run", "snn_multi_post",
    "snn_multi_status", "snn_multi_set_trace", "snn_classifier_pack", "snn_create_prop_plan",
    "snn_prop_plan_pack", "snn_propagate_tiled", "snn_destroy_prop_plan",
]


class SnnError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"status {status}: {msg}")
        self.status = status


vp = C.c_void_p
i32 = C.c_int32
i64 = C.c_int64
u64 = C.c_uint64
f64 = C.c_double


class RaggedDesc(C.Structure):
    _fields_ = [("P", i32), ("Q", i32), ("C", i32), ("dtype", i32), ("no_autapse", i32), ("reserved", i32),
                ("row_len", vp), ("ind", vp), ("w", vp), ("m", vp), ("v", vp), ("grad", vp),
                ("sign_bits", vp), ("conn_bits", vp), ("seed", u64)]


class RewireStats(C.Structure):
    _fields_ = [("removed", i64), ("formed", i64), ("overflow", i64), ("attempts", i64)]


class ClassifierDesc(C.Structure):
    _fields_ = [("n_in", i32), ("N", i32), ("K", i32), ("dtype", i32),
                ("tau_m", f64), ("v_thr", f64), ("beta", f64), ("tau_a", f64), ("dt", f64),
                ("n_classes", i32), ("n_bins", i32), ("in_thr", vp), ("in_seed", u64),
                ("w_in", vp), ("w_rec", vp), ("W_out", vp), ("b_out", vp), ("W_out_m", vp), ("W_out_v", vp),
                ("b_m", vp), ("b_v", vp), ("G_out", vp), ("G_b", vp), ("max_B", i32), ("max_T", i32)]


class Batch(C.Structure):
    _fields_ = [("B", i32), ("T", i32), ("labels", vp), ("bin_len", vp), ("trial_ids", vp),
                ("v", vp), ("a", vp), ("y", vp), ("x_bits", vp), ("z_bits", vp), ("x_rec", vp), ("z_rec", vp),
                ("psi_rec", vp), ("d_rec", vp), ("ysum", vp), ("v_rec", vp), ("a_rec", vp), ("y_rec", vp),
                ("delta", vp), ("Dout", vp), ("trial_T", vp)]


class Adam(C.Structure):
    _fields_ = [("lr", f64), ("beta1", f64), ("beta2", f64), ("eps", f64), ("step", i64), ("step_dev", vp),
                ("l1", f64), ("temperature", f64), ("noise_idx", i64), ("noise_idx_dev", vp)]


class MultiInstance(C.Structure):
    _fields_ = [("cls", vp), ("batch", Batch), ("label_table", vp), ("n_label", i32), ("bin_table", vp),
                ("n_bin", i32), ("iter", vp), ("lr", f64), ("beta1", f64), ("beta2", f64), ("eps", f64), ("l1", f64),
                ("temperature", f64), ("stats", vp)]


class DeeprGuide(C.Structure):
    _fields_ = [("L", i32), ("reserved", i32), ("sigma", f64), ("pre_site", vp), ("post_site", vp)]


class TopoParams(C.Structure):
    _fields_ = [("L", i32), ("L_f", i32), ("radius2", i32), ("t_stim", i32),
                ("dt", f64), ("tau_m", f64), ("V_rest", f64), ("E_exc", f64), ("V_theta", f64), ("V_reset", f64),
                ("tau_s", f64), ("g_leak", f64), ("tau_ref", f64), ("f_base", f64), ("f_in", f64), ("g_max", f64),
                ("tau_plus", f64), ("tau_minus", f64), ("A_plus_rel", f64), ("B", f64), ("sigma_stim", f64)]


class TopoDerived(C.Structure):
    _fields_ = [("n_ref", i32), ("reserved", i32), ("A_plus", f64), ("A_minus", f64)]


class TopoRewire(C.Structure):
    _fields_ = [("p_form", f64), ("sigma", f64), ("p_elim_dep", f64), ("p_elim_pot", f64), ("g_max", f64),
                ("L", i32), ("n_att", i32), ("elim_d2", vp), ("form_d2", vp)]


class TopoState(C.Structure):
    _fields_ = [("V", vp), ("gs", vp), ("ref", vp), ("x_src", vp), ("x_tgt", vp), ("y", vp), ("ydec", vp),
                ("src_bits", vp), ("tgt_bits", vp), ("acc", vp)]


_lib = None


def load() -> C.CDLL:
    """Load libsnnsp.so (raises OSError if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise OSError(f"{LIB_PATH} is missing: build it with `python -m paper_2510_19764_gb300.build` "
                      "(there is no fallback implementation)")
    lib = C.CDLL(LIB_PATH)
    P = C.POINTER
    sig = {
        "snn_last_error": (C.c_char_p, []),
        "snn_abi_version": (i32, []),
        "snn_create_ragged": (i32, [P(RaggedDesc), i32, vp, P(vp)]),
        "snn_destroy_ragged": (i32, [vp]),
        "snn_ragged_status": (i32, [vp, vp]),
        "snn_propagate": (i32, [vp, vp, i32, vp, vp]),
        "snn_create_prop_plan": (i32, [vp, i32, P(vp)]),
        "snn_prop_plan_pack": (i32, [vp, vp]),
        "snn_propagate_tiled": (i32, [vp, vp, i32, vp, vp]),
        "snn_destroy_prop_plan": (i32, [vp]),
        "snn_rewire_deepr": (i32, [vp, i64, vp, vp]),
        "snn_create_classifier": (i32, [P(ClassifierDesc), P(vp)]),
        "snn_destroy_classifier": (i32, [vp]),
        "snn_step_neurons": (i32, [vp, P(Batch), i32, i32, vp]),
        "snn_eprop_update": (i32, [vp, P(Batch), i32, P(Adam), vp]),
        "snn_topo_input": (i32, [P(TopoParams), P(TopoState), u64, i64, vp]),
        "snn_topo_neurons": (i32, [P(TopoParams), P(TopoState), i64, vp]),
        "snn_stdp_update": (i32, [vp, P(TopoParams), vp, vp, vp, vp, vp]),
        "snn_rewire_topo": (i32, [vp, P(TopoRewire), i64, vp, vp]),
        "snn_topo_run": (i32, [P(TopoParams), P(TopoState), vp, vp, P(TopoRewire), P(TopoRewire), u64, i32, i64,
                               i32, vp, vp, vp]),
        "snn_philox": (i32, [u64, u64, vp, i64, vp, vp]),
        "snn_rewire_deepr_noalloc": (i32, [P(RaggedDesc), i64, vp, vp, vp]),
        "snn_classifier_set_schedule": (i32, [vp, i32]),
        "snn_rewire_deepr_dev": (i32, [vp, vp, vp, vp]),
        "snn_draw_inputs": (i32, [vp, P(Batch), i32, i32, vp]),
        "snn_step_neurons_ex": (i32, [vp, P(Batch), i32, i32, i32, vp]),
        "snn_topo_connectivity": (i32, [vp, i32, vp, vp, vp, vp]),
        "snn_ragged_set_deepr_guide": (i32, [vp, vp, vp]),
        "snn_test_wait_timeout": (i32, [vp, i32, i32, vp]),
        "snn_ragged_add_row": (i32, [vp, vp, vp, vp, vp]),
        "snn_ragged_remove_row": (i32, [vp, vp, vp, vp]),
        "snn_adam_bias": (i32, [f64, f64, i64, P(f64)]),
        "snn_topo_derive": (i32, [P(TopoParams), P(TopoDerived)]),
        "snn_classifier_set_row_schedule": (i32, [vp, i32]),
        "snn_multi_create": (i32, [P(MultiInstance), i32, P(vp)]),
        "snn_multi_destroy": (i32, [vp]),
        "snn_multi_run": (i32, [vp, i32, i64, vp]),
        "snn_multi_post": (i32, [vp, P(i32), i32]),
        "snn_multi_status": (i32, [vp, vp]),
        "snn_multi_set_trace": (i32, [vp, vp]),
        "snn_classifier_pack": (i32, [vp, vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def ptr(t) -> int | None:
    """Device pointer of a torch tensor (None -> NULL)."""
    if t is None:
        return None
    return t.data_ptr()


def stream_ptr(stream) -> int | None:
    if stream is None:
        return None
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


def check(status: int) -> None:
    if status != SNN_OK:
        raise SnnError(status, load().snn_last_error().decode())


# ---------------------------------------------------------------- thin wrappers

def snn_last_error() -> str:
    return load().snn_last_error().decode()


def snn_abi_version() -> int:
    return load().snn_abi_version()


def snn_create_ragged(desc: RaggedDesc, init_deepr_bitfields: bool, stream=None) -> int:
    h = vp()
    check(load().snn_create_ragged(C.byref(desc), int(bool(init_deepr_bitfields)), stream_ptr(stream), C.byref(h)))
    return h.value


def snn_destroy_ragged(h: int) -> None:
    check(load().snn_destroy_ragged(h))


def snn_ragged_status(h: int, stream=None) -> int:
    return load().snn_ragged_status(h, stream_ptr(stream))


def snn_propagate(h: int, pre_bits, B: int, post_acc, stream=None) -> None:
    check(load().snn_propagate(h, ptr(pre_bits), B, ptr(post_acc), stream_ptr(stream)))


def snn_create_prop_plan(h: int, max_B: int) -> int:
    out = vp()
    check(load().snn_create_prop_plan(h, max_B, C.byref(out)))
    return out.value


def snn_prop_plan_pack(plan: int, stream=None) -> None:
    check(load().snn_prop_plan_pack(plan, stream_ptr(stream)))


def snn_propagate_tiled(plan: int, pre_bits, B: int, post_acc, stream=None) -> None:
    check(load().snn_propagate_tiled(plan, ptr(pre_bits), B, ptr(post_acc), stream_ptr(stream)))


def snn_destroy_prop_plan(plan: int) -> None:
    check(load().snn_destroy_prop_plan(plan))


def snn_rewire_deepr(h: int, rewire_idx: int, stats=None, stream=None) -> None:
    check(load().snn_rewire_deepr(h, rewire_idx, ptr(stats), stream_ptr(stream)))


def snn_rewire_deepr_noalloc(desc: RaggedDesc, rewire_idx: int, stats=None, status=None, stream=None) -> None:
    check(load().snn_rewire_deepr_noalloc(C.byref(desc), rewire_idx, ptr(stats), ptr(status), stream_ptr(stream)))


def snn_rewire_deepr_dev(h: int, rewire_idx_dev, stats=None, stream=None) -> None:
    check(load().snn_rewire_deepr_dev(h, ptr(rewire_idx_dev), ptr(stats), stream_ptr(stream)))


def snn_create_classifier(desc: ClassifierDesc) -> int:
    h = vp()
    check(load().snn_create_classifier(C.byref(desc), C.byref(h)))
    return h.value


def snn_classifier_set_schedule(h: int, warps_per_trial: int) -> None:
    check(load().snn_classifier_set_schedule(h, warps_per_trial))


def snn_destroy_classifier(h: int) -> None:
    check(load().snn_destroy_classifier(h))


def snn_step_neurons(h: int, batch: Batch, t0: int, n_steps: int, stream=None) -> None:
    check(load().snn_step_neurons(h, C.byref(batch), t0, n_steps, stream_ptr(stream)))


def snn_draw_inputs(h: int, batch: Batch, t0: int, n_steps: int, stream=None) -> None:
    check(load().snn_draw_inputs(h, C.byref(batch), t0, n_steps, stream_ptr(stream)))


def snn_step_neurons_ex(h: int, batch: Batch, t0: int, n_steps: int, flags: int, stream=None) -> None:
    check(load().snn_step_neurons_ex(h, C.byref(batch), t0, n_steps, flags, stream_ptr(stream)))


def snn_eprop_update(h: int, batch: Batch | None, phase: int, adam: Adam | None, stream=None) -> None:
    check(load().snn_eprop_update(h, C.byref(batch) if batch is not None else None, phase,
                                  C.byref(adam) if adam is not None else None, stream_ptr(stream)))


def snn_topo_input(p: TopoParams, st: TopoState, seed: int, t: int, stream=None) -> None:
    check(load().snn_topo_input(C.byref(p), C.byref(st), seed, t, stream_ptr(stream)))


def snn_topo_neurons(p: TopoParams, st: TopoState, t: int, stream=None) -> None:
    check(load().snn_topo_neurons(C.byref(p), C.byref(st), t, stream_ptr(stream)))


def snn_stdp_update(h: int, p: TopoParams, pre_bits, post_bits, x_pre, ydec, stream=None) -> None:
    check(load().snn_stdp_update(h, C.byref(p), ptr(pre_bits), ptr(post_bits), ptr(x_pre), ptr(ydec),
                                 stream_ptr(stream)))


def snn_rewire_topo(h: int, p: TopoRewire, rewire_idx: int, stats=None, stream=None) -> None:
    check(load().snn_rewire_topo(h, C.byref(p), rewire_idx, ptr(stats), stream_ptr(stream)))


def snn_topo_run(p: TopoParams, st: TopoState, ff: int, lat: int, rw_ff: TopoRewire, rw_lat: TopoRewire,
                 input_seed: int, rewire_every: int, t0: int, n_steps: int, stats_ff=None, stats_lat=None,
                 stream=None) -> None:
    check(load().snn_topo_run(C.byref(p), C.byref(st), ff, lat, C.byref(rw_ff), C.byref(rw_lat), input_seed,
                              rewire_every, t0, n_steps, ptr(stats_ff), ptr(stats_lat), stream_ptr(stream)))


def snn_ragged_set_deepr_guide(h: int, g: "DeeprGuide | None", stream=None) -> None:
    check(load().snn_ragged_set_deepr_guide(h, C.byref(g) if g is not None else None, stream_ptr(stream)))


def snn_ragged_add_row(h: int, targets, w_new=None, stats=None, stream=None) -> None:
    check(load().snn_ragged_add_row(h, ptr(targets), ptr(w_new), ptr(stats), stream_ptr(stream)))


def snn_ragged_remove_row(h: int, targets, stats=None, stream=None) -> None:
    check(load().snn_ragged_remove_row(h, ptr(targets), ptr(stats), stream_ptr(stream)))


def snn_test_wait_timeout(h: int, arrive: bool, limit: int, stream=None) -> None:
    check(load().snn_test_wait_timeout(h, int(arrive), limit, stream_ptr(stream)))


def snn_topo_connectivity(h: int, L: int, disp_count=None, disp_wsum=None, in_degree=None, stream=None) -> None:
    check(load().snn_topo_connectivity(h, L, ptr(disp_count), ptr(disp_wsum), ptr(in_degree), stream_ptr(stream)))


def snn_philox(seed: int, purpose: int, ctr, n: int, out, stream=None) -> None:
    check(load().snn_philox(seed, purpose, ptr(ctr), n, ptr(out), stream_ptr(stream)))


def snn_adam_bias(beta1: float, beta2: float, step: int) -> tuple[float, float]:
    out = (f64 * 2)()
    check(load().snn_adam_bias(beta1, beta2, step, out))
    return out[0], out[1]


def snn_topo_derive(p: TopoParams) -> TopoDerived:
    out = TopoDerived()
    check(load().snn_topo_derive(C.byref(p), C.byref(out)))
    return out


def snn_classifier_set_row_schedule(h: int, mode: int) -> None:
    check(load().snn_classifier_set_row_schedule(h, mode))


def snn_multi_create(instances: "list[MultiInstance]") -> int:
    arr = (MultiInstance * len(instances))(*instances)
    h = vp()
    check(load().snn_multi_create(arr, len(instances), C.byref(h)))
    return h.value


def snn_multi_destroy(h: int) -> None:
    check(load().snn_multi_destroy(h))


def snn_multi_run(h: int, flags: int = 0, wait_limit_ns: int = 2_000_000_000, stream=None) -> None:
    check(load().snn_multi_run(h, flags, wait_limit_ns, stream_ptr(stream)))


def snn_multi_post(h: int, instances) -> None:
    ids = list(instances)
    arr = (i32 * max(1, len(ids)))(*ids)
    check(load().snn_multi_post(h, arr, len(ids)))


def snn_multi_status(h: int, stream=None) -> int:
    return load().snn_multi_status(h, stream_ptr(stream))


def snn_multi_set_trace(h: int, times) -> None:
    check(load().snn_multi_set_trace(h, ptr(times)))


def snn_classifier_pack(h: int, stream=None) -> None:
    check(load().snn_classifier_pack(h, stream_ptr(stream)))
