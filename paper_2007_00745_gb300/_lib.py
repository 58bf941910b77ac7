"""ctypes view of the C ABI declared in include/mb.h.

Argument marshalling only: every step of the render runs in the CUDA library.
Loading fails loudly (ImportError / OSError) when libmb.so has not been built;
there is no CPU fallback.
"""
import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libmb.so")

u8, u16, u32, u64 = ctypes.c_uint8, ctypes.c_uint16, ctypes.c_uint32, ctypes.c_uint64
i32, f64, vp, sz = ctypes.c_int, ctypes.c_double, ctypes.c_void_p, ctypes.c_size_t

MB_OK, MB_EINVAL, MB_ENOMEM, MB_ECUDA, MB_ETIMEDOUT, MB_EBUSY, MB_ENOTFOUND, MB_EDEVICE, MB_ECANCELED = range(9)
MB_SCHED_NAIVE, MB_SCHED_ALTERNATING, MB_SCHED_FCFS_ROWS, MB_SCHED_FCFS_TILES, MB_SCHED_FCFS_ITEMS = range(5)


class mb_window(ctypes.Structure):
    _fields_ = [("xmin", f64), ("xmax", f64), ("ymin", f64), ("ymax", f64)]


class mb_item(ctypes.Structure):
    _fields_ = [("tile", u32), ("row0", u16), ("rows", u16)]


class mb_cta_trace(ctypes.Structure):
    _fields_ = [("start_ns", u64), ("end_ns", u64), ("smid", u32), ("items", u32)]


class mb_opts(ctypes.Structure):
    _fields_ = [("sched", i32), ("tile", u32), ("grid", u32), ("block", u32), ("unroll", u32),
                ("stream", vp), ("items", vp), ("n_items", u32), ("tile_totals", vp), ("trace", vp), ("trace_len", u32),
                ("status", vp), ("workspace", vp), ("workspace_bytes", sz), ("split", u32), ("round_tiles", u32), ("max_seconds", u32), ("fp64_products", u32),
                ("ev_start", vp), ("ev_stop", vp), ("precision", u32),
                ("cycle_check", u32), ("learned_order", u32), ("model", vp), ("min_strips", u32)]


class mb_view(ctypes.Structure):
    _fields_ = [("w", mb_window), ("m", u32), ("n", u32), ("iter_max", u32), ("escape_r2", f64), ("out", vp)]


class mb_request(ctypes.Structure):
    _fields_ = [("w", mb_window), ("m", u32), ("n", u32), ("iter_max", u32), ("escape_r2", f64)]


class mb_req_stats(ctypes.Structure):
    _fields_ = [("submit_ns", u64), ("admit_ns", u64), ("start_ns", u64), ("done_ns", u64), ("bytes", u64),
                ("status", i32)]


class mb_serve_counters(ctypes.Structure):
    _fields_ = [("submitted", u64), ("admitted", u64), ("completed", u64), ("rejected", u64), ("rounds", u64),
                ("bytes_in_use", u64), ("peak_bytes", u64), ("queued", u32)]


class mb_run_stats(ctypes.Structure):
    _fields_ = [("makespan_ns", u64), ("iterations", u64), ("ctas", u32), ("sms", u32), ("idle_tail", f64),
                ("sm_busy_min", f64), ("sm_busy_mean", f64), ("sm_busy_max", f64)]


class MBError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        super().__init__("%s: %s (%d)" % (where, _lib.mb_strerror(code).decode(), code))


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError("libmb.so not built (%s); run paper_2007_00745_gb300/build.py" % LIB_PATH)
    L = ctypes.CDLL(LIB_PATH)
    L.mb_version.restype = ctypes.c_char_p
    L.mb_strerror.restype = ctypes.c_char_p
    L.mb_strerror.argtypes = [i32]
    L.mb_render.argtypes = [ctypes.POINTER(mb_window), u32, u32, u32, f64, vp, ctypes.POINTER(mb_opts)]
    L.mb_render.restype = i32
    L.mb_render_noalloc.argtypes = [ctypes.POINTER(mb_window), u32, u32, u32, f64, vp, ctypes.POINTER(mb_opts)]
    L.mb_render_noalloc.restype = i32
    L.mb_render_workspace_size.argtypes = [u32, u32, ctypes.POINTER(mb_opts)]
    L.mb_render_workspace_size.restype = sz
    L.mb_sum_counts.argtypes = [vp, u64, vp, vp]
    L.mb_sum_counts.restype = i32
    L.mb_last_stats.argtypes = [ctypes.POINTER(mb_run_stats)]
    L.mb_last_stats.restype = i32
    L.mb_selftest_wait.argtypes = [u32, vp, vp, vp]
    L.mb_selftest_wait.restype = i32
    L.mb_fp64_peak.argtypes = [i32, ctypes.POINTER(f64), ctypes.POINTER(f64)]
    L.mb_fp64_peak.restype = i32
    L.mb_device_info.argtypes = [u32, ctypes.POINTER(u32), ctypes.POINTER(u32)]
    L.mb_selftest_products.argtypes = [vp, vp, u64, vp, vp, vp, vp]
    L.mb_colorize.argtypes = [vp, u64, u32, vp, vp]
    L.mb_colorize.restype = i32
    L.mb_write_ppm.argtypes = [ctypes.c_char_p, vp, u32, u32]
    L.mb_write_ppm.restype = i32
    L.mb_pack_items.argtypes = [vp, u32, u32, u32, vp, u32, vp, vp, vp]
    L.mb_pack_items.restype = i32
    L.mb_unpack_items.argtypes = [vp, u32, u32, u32, vp, u32, vp, vp, vp]
    L.mb_unpack_items.restype = i32
    L.mb_selftest_products.restype = i32
    L.mb_selftest_psub.argtypes = [vp, vp, u64, vp, vp, vp]
    L.mb_selftest_psub.restype = i32
    L.mb_device_info.restype = i32
    P = ctypes.POINTER
    L.mb_probe.argtypes = [P(mb_window), u32, u32, u32, f64, vp, vp, P(mb_opts)]
    L.mb_tile_features.argtypes = [vp, P(mb_window), u32, u32, u32, u32, vp, vp]
    L.mb_mlp_forward.argtypes = [vp, vp, u32, vp, vp]
    L.mb_tile_targets.argtypes = [vp, u32, vp, vp]
    L.mb_mlp_grad.argtypes = [vp, vp, vp, u32, vp, vp, vp, vp]
    L.mb_adam_step.argtypes = [vp, vp, vp, vp, u32, u32, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                               ctypes.c_float, vp]
    L.mb_model_train.argtypes = [vp, vp, vp, vp, vp, u32, vp, u32, u32, ctypes.c_float, vp, vp]
    L.mb_order_split.argtypes = [vp, u32, u32, u32, u32, vp, u32, vp, vp, vp]
    L.mb_render_learned.argtypes = [P(mb_window), u32, u32, u32, f64, vp, vp, P(mb_opts)]
    L.mb_guard_costs.argtypes = [vp, u32, u32, vp, vp]
    L.mb_model_save.argtypes = [vp, ctypes.c_char_p]
    L.mb_model_load.argtypes = [ctypes.c_char_p, vp]
    L.mb_render_batch.argtypes = [P(mb_view), u32, P(mb_opts)]
    L.mb_batch_plan_create.argtypes = [P(mb_view), u32, P(mb_opts), P(vp)]
    L.mb_batch_plan_launch.argtypes = [vp, vp]
    L.mb_batch_plan_info.argtypes = [vp, P(u32), P(u32), P(u64)]
    L.mb_batch_plan_destroy.argtypes = [vp]
    L.mb_batch_autotune.argtypes = [P(mb_view), u32, P(mb_opts), u32, ctypes.c_char_p, P(mb_opts),
                                    P(ctypes.c_float)]
    L.mb_serve_create.argtypes = [sz, u32, P(mb_opts), P(vp)]
    L.mb_serve_submit.argtypes = [vp, P(mb_request), P(u64)]
    L.mb_serve_wait.argtypes = [vp, u64, u32, P(mb_req_stats)]
    L.mb_serve_result.argtypes = [vp, u64, P(vp)]
    L.mb_serve_release.argtypes = [vp, u64]
    L.mb_serve_read.argtypes = [vp, u64, vp, u64, vp]
    L.mb_serve_counters_get.argtypes = [vp, P(mb_serve_counters)]
    L.mb_serve_fail.argtypes = [vp, i32]
    L.mb_serve_destroy.argtypes = [vp]
    for name in ("mb_serve_create", "mb_serve_submit", "mb_serve_wait", "mb_serve_result", "mb_serve_release", "mb_serve_read",
                 "mb_serve_counters_get", "mb_serve_fail", "mb_serve_destroy"):
        getattr(L, name).restype = i32
    for name in ("mb_render_batch", "mb_batch_plan_create", "mb_batch_plan_launch", "mb_batch_plan_info",
                 "mb_batch_plan_destroy", "mb_batch_autotune"):
        getattr(L, name).restype = i32
    for name in ("mb_probe", "mb_tile_features", "mb_tile_targets", "mb_mlp_forward", "mb_mlp_grad", "mb_adam_step",
                 "mb_model_train", "mb_order_split", "mb_render_learned", "mb_model_save", "mb_model_load",
                 "mb_guard_costs"):
        getattr(L, name).restype = i32
    return L


_lib = _load()


def lib():
    return _lib


def check(rc, where):
    if rc != MB_OK:
        raise MBError(rc, where)
    return rc
