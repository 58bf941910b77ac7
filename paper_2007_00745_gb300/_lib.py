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

MB_OK, MB_EINVAL, MB_ENOMEM, MB_ECUDA, MB_ETIMEDOUT, MB_EBUSY, MB_ENOTFOUND, MB_EDEVICE = range(8)
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
                ("status", vp), ("workspace", vp), ("workspace_bytes", sz)]


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
    L.mb_fp64_peak.argtypes = [i32, ctypes.POINTER(f64), ctypes.POINTER(f64)]
    L.mb_fp64_peak.restype = i32
    L.mb_device_info.argtypes = [u32, ctypes.POINTER(u32), ctypes.POINTER(u32)]
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
    L.mb_order_split.argtypes = [vp, u32, u32, u32, vp, u32, vp, vp, vp]
    L.mb_render_learned.argtypes = [P(mb_window), u32, u32, u32, f64, vp, vp, P(mb_opts)]
    L.mb_model_save.argtypes = [vp, ctypes.c_char_p]
    L.mb_model_load.argtypes = [ctypes.c_char_p, vp]
    for name in ("mb_probe", "mb_tile_features", "mb_tile_targets", "mb_mlp_forward", "mb_mlp_grad", "mb_adam_step",
                 "mb_model_train", "mb_order_split", "mb_render_learned", "mb_model_save", "mb_model_load"):
        getattr(L, name).restype = i32
    return L


_lib = _load()


def lib():
    return _lib


def check(rc, where):
    if rc != MB_OK:
        raise MBError(rc, where)
    return rc
