"""CPU oracle for the escape-time renderer -- TEST INFRASTRUCTURE ONLY.

Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline / reference
legs may import this package.  It is a plain, slow, obviously correct
restatement of the paper's method (Sec. I, Eq. 1-2; row partitions of
Sec. III) in C (mb_oracle.c, FP64, no FMA contraction) and numpy (the tile-cost
network in mlp.py, FP64).  It shares no code with the CUDA path and never
imports it.
"""
import ctypes
import os

import numpy as np

from . import build as _build

_lib = None


def lib():
    """Load (building first if needed) the compiled C oracle."""
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        u32, u64, f64, i32 = ctypes.c_uint32, ctypes.c_uint64, ctypes.c_double, ctypes.c_int
        p = ctypes.c_void_p
        L.mbo_c_re.argtypes = [f64, f64, u32, u32]
        L.mbo_c_re.restype = f64
        L.mbo_c_im.argtypes = [f64, f64, u32, u32]
        L.mbo_c_im.restype = f64
        L.mbo_escape.argtypes = [f64, f64, u32, f64]
        L.mbo_escape.restype = u32
        L.mbo_pixel_map.argtypes = [f64, f64, f64, f64, u32, u32, p, p]
        L.mbo_render.argtypes = [f64, f64, f64, f64, u32, u32, u32, f64, p, i32]
        L.mbo_render_rows.argtypes = [f64, f64, f64, f64, u32, u32, u32, f64, u32, u32, p, i32]
        L.mbo_render_pixels.argtypes = [f64, f64, f64, f64, u32, u32, u32, f64, p, ctypes.c_size_t, p, i32]
        L.mbo_tile_totals.argtypes = [p, u32, u32, u32, u32, p]
        L.mbo_probe.argtypes = [f64, f64, f64, f64, u32, u32, u32, f64, u32, u32, p, i32]
        L.mbo_naive_rows.argtypes = [u32, u32, u32, ctypes.POINTER(u32), ctypes.POINTER(u32)]
        L.mbo_alternating_owner.argtypes = [u32, u32]
        L.mbo_alternating_owner.restype = u32
        L.mbo_max_threads.restype = i32
        L.mbo_colorize.argtypes = [p, u64, u32, p]
        f32, pf = ctypes.c_float, ctypes.POINTER(ctypes.c_float)
        L.mbo_escape_f32.argtypes = [f64, f64, u32, f64]
        L.mbo_escape_f32.restype = u32
        L.mbo_escape_df.argtypes = [f64, f64, u32, f64]
        L.mbo_escape_df.restype = u32
        for name in ("mbo_two_sum", "mbo_fast_two_sum", "mbo_two_prod"):
            getattr(L, name).argtypes = [f32, f32, pf, pf]
        for name in ("mbo_df_add4", "mbo_df_mul4"):
            getattr(L, name).argtypes = [f32, f32, f32, f32, pf, pf]
        L.mbo_render_rows_lowp.argtypes = [f64, f64, f64, f64, u32, u32, u32, f64, i32, u32, u32, p, i32]
        _lib = L
    return _lib


def _ptr(a):
    return ctypes.c_void_p(a.ctypes.data)


def c_re(window, n, j):
    """Real part of c for column j (Sec. I; Cx of Sec. III-A)."""
    return lib().mbo_c_re(window[0], window[1], n, j)


def c_im(window, m, i):
    """Imaginary part of c for row i, row 0 at the top."""
    return lib().mbo_c_im(window[2], window[3], m, i)


def escape(cr, ci, iter_max, r2=4.0):
    """Escape count of one point (Eq. 1 iterated from z = 0, Eq. 2)."""
    return int(lib().mbo_escape(float(cr), float(ci), int(iter_max), float(r2)))


def pixel_map(window, m, n):
    """(Cx[n], Cy[m]) arrays."""
    cx = np.empty(n, np.float64)
    cy = np.empty(m, np.float64)
    lib().mbo_pixel_map(*map(float, window), m, n, _ptr(cx), _ptr(cy))
    return cx, cy


def render(window, m, n, iter_max, r2=4.0, threads=0):
    """Full m x n image of counts, uint32 row-major."""
    out = np.empty((m, n), np.uint32)
    lib().mbo_render(*map(float, window), m, n, iter_max, float(r2), _ptr(out), threads)
    return out


def render_rows(window, m, n, iter_max, r2, row0, nrows, threads=0):
    out = np.empty((nrows, n), np.uint32)
    lib().mbo_render_rows(*map(float, window), m, n, iter_max, float(r2), row0, nrows, _ptr(out), threads)
    return out


def render_pixels(window, m, n, iter_max, r2, idx, threads=0):
    """Counts of the pixels idx (flat indices i*n + j)."""
    idx = np.ascontiguousarray(idx, dtype=np.uint64)
    out = np.empty(idx.shape[0], np.uint32)
    lib().mbo_render_pixels(*map(float, window), m, n, iter_max, float(r2), _ptr(idx), idx.shape[0],
                            _ptr(out), threads)
    return out


def tile_totals(counts, tile_h, tile_w):
    """Sum of counts per tile, tiles numbered row-major."""
    counts = np.ascontiguousarray(counts, dtype=np.uint32)
    m, n = counts.shape
    tx = (n + tile_w - 1) // tile_w
    ty = (m + tile_h - 1) // tile_h
    out = np.empty(tx * ty, np.uint64)
    lib().mbo_tile_totals(_ptr(counts), m, n, tile_h, tile_w, _ptr(out))
    return out


def probe(window, m, n, iter_max, r2, tile, probe_side, threads=0):
    """Probe counts, shape (tiles, probe_side, probe_side)."""
    tx = (n + tile - 1) // tile
    ty = (m + tile - 1) // tile
    out = np.empty((tx * ty, probe_side, probe_side), np.uint32)
    lib().mbo_probe(*map(float, window), m, n, iter_max, float(r2), tile, probe_side, _ptr(out), threads)
    return out


def naive_rows(m, workers, r):
    """(first row, row count) of worker r under the naive partition (Sec. III-A)."""
    a, b = ctypes.c_uint32(), ctypes.c_uint32()
    lib().mbo_naive_rows(m, workers, r, ctypes.byref(a), ctypes.byref(b))
    return a.value, b.value


def alternating_owner(i, workers):
    """Worker that owns row i under the alternating partition (Sec. III-C)."""
    return int(lib().mbo_alternating_owner(i, workers))


def max_threads():
    return int(lib().mbo_max_threads())


def colorize(counts, iter_max):
    """RGB bytes (count x 3) of the counts under the palette of mbo_colorize."""
    counts = np.ascontiguousarray(counts, dtype=np.uint32).reshape(-1)
    out = np.empty((counts.size, 3), np.uint8)
    lib().mbo_colorize(_ptr(counts), counts.size, iter_max, _ptr(out))
    return out


PRECISIONS = {"fp32": 1, "dfloat": 2}


def escape_lowp(cr, ci, iter_max, r2=4.0, precision="fp32"):
    """Escape count of one point in binary32 ("fp32") or double-float ("dfloat")."""
    f = lib().mbo_escape_f32 if precision == "fp32" else lib().mbo_escape_df
    return int(f(float(cr), float(ci), int(iter_max), float(r2)))


def render_lowp(window, m, n, iter_max, r2=4.0, precision="fp32", row0=0, nrows=None, threads=0):
    """Rows [row0, row0 + nrows) of the image in a reduced precision, uint32."""
    nrows = m - row0 if nrows is None else nrows
    out = np.empty((nrows, n), np.uint32)
    lib().mbo_render_rows_lowp(*map(float, window), m, n, iter_max, float(r2), PRECISIONS[precision],
                               row0, nrows, _ptr(out), threads)
    return out


def _f32_pair(fn, *args):
    a, b = ctypes.c_float(), ctypes.c_float()
    fn(*[float(x) for x in args], ctypes.byref(a), ctypes.byref(b))
    return a.value, b.value


def two_sum(a, b):
    """(s, e) with s + e == a + b exactly (binary32 inputs)."""
    return _f32_pair(lib().mbo_two_sum, a, b)


def fast_two_sum(a, b):
    """(s, e) with s + e == a + b exactly when |a| >= |b|."""
    return _f32_pair(lib().mbo_fast_two_sum, a, b)


def two_prod(a, b):
    """(p, e) with p + e == a * b exactly."""
    return _f32_pair(lib().mbo_two_prod, a, b)


def df_add(x, y):
    """Double-float sum of (xh, xl) and (yh, yl)."""
    return _f32_pair(lib().mbo_df_add4, x[0], x[1], y[0], y[1])


def df_mul(x, y):
    """Double-float product of (xh, xl) and (yh, yl)."""
    return _f32_pair(lib().mbo_df_mul4, x[0], x[1], y[0], y[1])
