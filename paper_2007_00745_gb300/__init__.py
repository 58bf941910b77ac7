"""GB300-native escape-time (Mandelbrot) renderer: Python binding of libmb.so.

The functions below carry the names of the C entry points in include/mb.h and
only marshal arguments: torch tensors provide device memory and streams, the
CUDA library does every step of the computation.  Importing this package does
not load the library; the first call does, and fails loudly if it is missing.
"""
import ctypes

__all__ = [
    "mb_version", "mb_strerror", "mb_render", "mb_render_noalloc", "mb_render_workspace_size", "mb_sum_counts",
    "mb_last_stats",
    "mb_fp64_peak", "mb_device_info", "Window", "MBError",
]

MB_SCHED_NAIVE, MB_SCHED_ALTERNATING, MB_SCHED_FCFS_ROWS, MB_SCHED_FCFS_TILES, MB_SCHED_FCFS_ITEMS = range(5)
SCHEDS = {"naive": MB_SCHED_NAIVE, "alternating": MB_SCHED_ALTERNATING, "fcfs_rows": MB_SCHED_FCFS_ROWS,
          "fcfs_tiles": MB_SCHED_FCFS_TILES, "fcfs_items": MB_SCHED_FCFS_ITEMS}
MB_PREC_FP64, MB_PREC_FP32, MB_PREC_DFLOAT = range(3)

# Per-launch time limit (mb_opts.max_seconds) used when a call does not pass one:
# 0 = none, as in the C API.  A positive value makes each CTA of a render stop
# after that many seconds and OR 4 into the status word (the image is then
# incomplete); the test suite sets it as a guard.
DEFAULT_MAX_SECONDS = 0
PRECISIONS = {"fp64": MB_PREC_FP64, "fp32": MB_PREC_FP32, "dfloat": MB_PREC_DFLOAT}


def _L():
    from . import _lib
    return _lib


class MBError(RuntimeError):
    pass


def Window(xmin, xmax, ymin, ymax):
    return (float(xmin), float(xmax), float(ymin), float(ymax))


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, int):
        return t
    return t.data_ptr()


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _opts(sched="fcfs_tiles", tile=0, grid=0, block=0, unroll=0, stream=None, items=None, n_items=0,
          tile_totals=None, trace=None, trace_len=0, status=None, workspace=None, workspace_bytes=0,
          events=None, fp64_products=0, max_seconds=None, split=0, round_tiles=0, precision="fp64",
          cycle_check=0, learned_order=0, model=None, min_strips=0):
    L = _L()
    o = L.mb_opts()
    o.sched = SCHEDS[sched] if isinstance(sched, str) else int(sched)
    o.tile, o.grid, o.block, o.unroll = int(tile), int(grid), int(block), int(unroll)
    o.stream = _stream(stream)
    o.items = _ptr(items)
    o.n_items = int(n_items if n_items else (items.numel() // 2 if items is not None and hasattr(items, "numel") else 0))
    o.tile_totals = _ptr(tile_totals)
    o.trace = _ptr(trace)
    o.trace_len = int(trace_len if trace_len else (trace.numel() * trace.element_size() // 24
                                                   if trace is not None and hasattr(trace, "numel") else 0))
    o.status = _ptr(status)
    o.fp64_products = int(fp64_products)
    o.max_seconds = int(DEFAULT_MAX_SECONDS if max_seconds is None else max_seconds)
    o.split = int(split)
    o.round_tiles = int(round_tiles)
    o.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    o.cycle_check = int(cycle_check)
    o.learned_order = int(learned_order)
    o.model = _ptr(model)
    o.min_strips = int(min_strips)
    if events is not None:   # (start, stop) torch.cuda.Event pair recorded around the main render kernel
        handles = []
        for ev in events:
            if hasattr(ev, "cuda_event"):
                if not ev.cuda_event:   # torch creates the CUDA event on its first record
                    ev.record()
                handles.append(ev.cuda_event)
            else:
                handles.append(int(ev))
        o.ev_start, o.ev_stop = handles
    o.workspace = _ptr(workspace)
    o.workspace_bytes = int(workspace_bytes if workspace_bytes else
                            (workspace.numel() * workspace.element_size() if workspace is not None
                             and hasattr(workspace, "numel") else 0))
    return o


def _check(rc, where):
    if rc != 0:
        L = _L()
        err = MBError("%s: %s (%d)" % (where, L.lib().mb_strerror(rc).decode(), rc))
        err.code = rc
        raise err


def mb_version():
    """Library version string."""
    return _L().lib().mb_version().decode()


def mb_strerror(code):
    """Name of a return code."""
    return _L().lib().mb_strerror(int(code)).decode()


def mb_render(window, m, n, iter_max, escape_r2, out, **opts):
    """Render an m x n image of escape counts into `out` (int32 tensor, m*n
    elements, on the GPU or in pinned host memory), asynchronously on the
    stream.  window = (xmin, xmax, ymin, ymax); escape_r2 = R^2.

    Keyword options (mb_opts; 0 / None = default):
      sched       "naive" | "alternating" | "fcfs_rows" | "fcfs_tiles" | "fcfs_items"
      tile, block, grid, unroll   launch shape (power-of-two tile 8..256; block 32..512;
                  grid = CTAs; unroll 4, 8 or 16)
      items       int32 [K, 2] device tensor of (tile, row0 | rows << 16), for "fcfs_items"
      precision   "fp64" (default, bit-exact binary64) | "fp32" | "dfloat"
      cycle_check 1 = stop exactly periodic binary64 orbits early (identical counts)
      status      int32 device tensor: error bits (1 bounded wait, 2 bad item, 4 deadline)
      trace       int64 device tensor, 3 per CTA: (start_ns, end_ns, smid | items << 32)
      tile_totals int64 device tensor: += per-tile sums of the counts
      max_seconds per-launch time limit (default DEFAULT_MAX_SECONDS, 0 = none)
      events      (start, stop) torch.cuda.Event pair recorded around the render kernel
      workspace   caller-owned device temporaries (mb_render_workspace_size bytes)
      stream      torch.cuda.Stream or raw handle (default: the current stream)
    Raises MBError with the library's code on invalid arguments."""
    L = _L()
    w = L.mb_window(*map(float, window))
    o = _opts(**opts)
    rc = L.lib().mb_render(ctypes.byref(w), int(m), int(n), int(iter_max), float(escape_r2), _ptr(out),
                           ctypes.byref(o))
    _check(rc, "mb_render")


def mb_render_noalloc(window, m, n, iter_max, escape_r2, out, **opts):
    """As mb_render, for callers that must not allocate device memory: the
    library's fixed scratch array replaces the temporary allocation (m, n each
    at most 16384; calls on one device share the array, so keep them ordered
    on one stream)."""
    L = _L()
    w = L.mb_window(*map(float, window))
    o = _opts(**opts)
    rc = L.lib().mb_render_noalloc(ctypes.byref(w), int(m), int(n), int(iter_max), float(escape_r2), _ptr(out),
                                   ctypes.byref(o))
    _check(rc, "mb_render_noalloc")


def mb_render_workspace_size(m, n, **opts):
    """Bytes of caller workspace mb_render needs for an m x n view."""
    L = _L()
    o = _opts(**opts)
    return int(L.lib().mb_render_workspace_size(int(m), int(n), ctypes.byref(o)))


def mb_sum_counts(counts, total, stream=None):
    """Sum of the uint32 counts in device tensor `counts` into device int64 tensor `total`."""
    _check(_L().lib().mb_sum_counts(_ptr(counts), int(counts.numel()), _ptr(total), _stream(stream)),
           "mb_sum_counts")


def mb_last_stats():
    """Statistics of this thread's most recent mb_render / mb_render_learned launch:
    makespan_ns, iterations, ctas, sms, idle_tail, sm_busy_min/mean/max."""
    L = _L()
    st = L.mb_run_stats()
    _check(L.lib().mb_last_stats(ctypes.byref(st)), "mb_last_stats")
    return {f: getattr(st, f) for f, _ in L.mb_run_stats._fields_}


def mb_selftest_wait(ctas, status, got, stream=None):
    """Bounded-wait self-test of the work-claiming protocol (see mb.h)."""
    L = _L()
    _check(L.lib().mb_selftest_wait(int(ctas), _ptr(status), _ptr(got), _stream(stream)), "mb_selftest_wait")


def mb_sum_counts_ptr(counts_ptr, count, total, stream=None):
    """mb_sum_counts on a raw device address (e.g. a served request's counts)."""
    _check(_L().lib().mb_sum_counts(int(counts_ptr), int(count), _ptr(total), _stream(stream)), "mb_sum_counts")


def mb_fp64_peak(op=0):
    """(binary64 operations per second, seconds) of the FP64 issue-rate microbenchmark."""
    L = _L()
    r, s = ctypes.c_double(), ctypes.c_double()
    _check(L.lib().mb_fp64_peak(int(op), ctypes.byref(r), ctypes.byref(s)), "mb_fp64_peak")
    return r.value, s.value


def mb_selftest_products(a, b, sq, pr, ok, stream=None):
    """Integer-pipe products of the render kernels on device arrays (see include/mb.h)."""
    _check(_L().lib().mb_selftest_products(_ptr(a), _ptr(b), int(a.numel()), _ptr(sq), _ptr(pr), _ptr(ok),
                                           _stream(stream)), "mb_selftest_products")


def mb_selftest_psub(a, b, d, ok, stream=None):
    """Integer-pipe subtraction of the render kernels on device arrays (see include/mb.h)."""
    _check(_L().lib().mb_selftest_psub(_ptr(a), _ptr(b), int(a.numel()), _ptr(d), _ptr(ok), _stream(stream)),
           "mb_selftest_psub")


def mb_device_info(block=0):
    """(SM count, resident render CTAs per SM at `block` threads) of the current device."""
    L = _L()
    a, b = ctypes.c_uint32(), ctypes.c_uint32()
    _check(L.lib().mb_device_info(int(block), ctypes.byref(a), ctypes.byref(b)), "mb_device_info")
    return a.value, b.value


# ---- learned tile-cost model -------------------------------------------------

MB_MLP_PARAMS = 8769
MB_MLP_FEATURES = 70


def mb_probe(window, m, n, iter_max, escape_r2, probe_out, image_out=None, **opts):
    """Probe counts (device int32 tensor, tiles*64) of a view; optionally also into image_out."""
    L = _L()
    w = L.mb_window(*map(float, window))
    o = _opts(**opts)
    _check(L.lib().mb_probe(ctypes.byref(w), int(m), int(n), int(iter_max), float(escape_r2), _ptr(probe_out),
                            _ptr(image_out), ctypes.byref(o)), "mb_probe")


def mb_tile_features(probe, window, m, n, iter_max, tile, feat, stream=None):
    """70 features per tile (float32 [tiles, 70]) from its probe counts."""
    L = _L()
    w = L.mb_window(*map(float, window))
    _check(L.lib().mb_tile_features(_ptr(probe), ctypes.byref(w), int(m), int(n), int(iter_max), int(tile),
                                    _ptr(feat), _stream(stream)), "mb_tile_features")


def mb_tile_targets(totals, ntiles, y, stream=None):
    """Training targets log2(1 + total) / 32 from per-tile totals (int64)."""
    _check(_L().lib().mb_tile_targets(_ptr(totals), int(ntiles), _ptr(y), _stream(stream)), "mb_tile_targets")


def mb_mlp_forward(params, x, count, y, stream=None):
    """Predicted log tile cost y[count] of the network for feature rows x[count, 70]."""
    _check(_L().lib().mb_mlp_forward(_ptr(params), _ptr(x), int(count), _ptr(y), _stream(stream)), "mb_mlp_forward")


def mb_mlp_grad(params, x, idx, batch, target, grad, loss=None, stream=None):
    """Gradient of the mean squared error over the rows idx[batch] into grad (and the loss)."""
    _check(_L().lib().mb_mlp_grad(_ptr(params), _ptr(x), _ptr(idx), int(batch), _ptr(target), _ptr(grad),
                                  _ptr(loss), _stream(stream)), "mb_mlp_grad")


def mb_adam_step(params, grad, m, v, count, t, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
    """One Adam update of `count` parameters at step t (1-based), in place."""
    _check(_L().lib().mb_adam_step(_ptr(params), _ptr(grad), _ptr(m), _ptr(v), int(count), int(t), float(lr),
                                   float(beta1), float(beta2), float(eps), _stream(stream)), "mb_adam_step")


def mb_model_train(params, adam_m, adam_v, x, target, count, order, epochs, batch, lr=1e-3, epoch_loss=None,
                   stream=None):
    """Trains in place on the GPU: `epochs` passes over `count` rows in the given
    per-epoch orders (int32 [epochs, count]), mini-batches of `batch`, Adam at
    learning rate lr; epoch_loss[epochs] receives the mean loss of each epoch."""
    _check(_L().lib().mb_model_train(_ptr(params), _ptr(adam_m), _ptr(adam_v), _ptr(x), _ptr(target), int(count),
                                     _ptr(order), int(epochs), int(batch), float(lr), _ptr(epoch_loss),
                                     _stream(stream)), "mb_model_train")


def mb_order_split(cost_pred, ntiles, tile, grid, items, capacity, n_items, status=None, stream=None, split=4):
    """Longest-first item list (with splits) from predicted costs; n_items = 0 and
    status bit 2 when it does not fit `capacity`."""
    _check(_L().lib().mb_order_split(_ptr(cost_pred), int(ntiles), int(tile), int(grid), int(split), _ptr(items),
                                     int(capacity), _ptr(n_items), _ptr(status), _stream(stream)), "mb_order_split")


def mb_guard_costs(cost_pred, tiles_x, tiles_y, guarded, stream=None):
    """Largest predicted cost over each tile's 3 x 3 neighbourhood (float32 device tensors)."""
    _check(_L().lib().mb_guard_costs(_ptr(cost_pred), int(tiles_x), int(tiles_y), _ptr(guarded), _stream(stream)),
           "mb_guard_costs")


def mb_render_learned(window, m, n, iter_max, escape_r2, out, params, **opts):
    """The learned pipeline: probe (8 x 8 samples per tile, written into `out`), tile
    features, predicted costs (`params`: the 8769 float32 parameters on the device, or
    None for the probe-sum order), neighbourhood guard, longest-first order with splits, then the FCFS
    render of the remaining pixels.  Options as mb_render (tile >= 16; `split` is the
    split divisor).  Binary64 only."""
    L = _L()
    w = L.mb_window(*map(float, window))
    o = _opts(**opts)
    _check(L.lib().mb_render_learned(ctypes.byref(w), int(m), int(n), int(iter_max), float(escape_r2), _ptr(out),
                                     _ptr(params), ctypes.byref(o)), "mb_render_learned")


def mb_model_save(params, path):
    """Writes the parameters to `path` (magic MBMLP701, count, float32 values)."""
    _check(_L().lib().mb_model_save(_ptr(params), str(path).encode()), "mb_model_save")


def mb_model_load(path, params):
    """Reads parameters written by mb_model_save; MBError on a bad or foreign file."""
    _check(_L().lib().mb_model_load(str(path).encode(), _ptr(params)), "mb_model_load")


# ---- batched mode ------------------------------------------------------------------

def _views(views, outs):
    L = _L()
    arr = (L.mb_view * len(views))()
    for k, (v, o) in enumerate(zip(views, outs)):
        arr[k].w = L.mb_window(*map(float, v[0]))
        arr[k].m, arr[k].n, arr[k].iter_max = int(v[1]), int(v[2]), int(v[3])
        arr[k].escape_r2 = float(v[4])
        arr[k].out = _ptr(o)
    return arr


def mb_render_batch(views, outs, **opts):
    """Render every view (window, m, n, iter_max, r2) into its device tensor in outs."""
    L = _L()
    arr = _views(views, outs)
    o = _opts(**opts)
    _check(L.lib().mb_render_batch(arr, len(views), ctypes.byref(o)), "mb_render_batch")


class BatchPlan:
    """mb_batch_plan_*: device tables built once, launches captured in a CUDA graph."""

    def __init__(self, views, outs, **opts):
        L = _L()
        self._arr = _views(views, outs)
        self._opts = _opts(**opts)
        self._h = ctypes.c_void_p()
        _check(L.lib().mb_batch_plan_create(self._arr, len(views), ctypes.byref(self._opts), ctypes.byref(self._h)),
               "mb_batch_plan_create")

    def launch(self, stream=None):
        _check(_L().lib().mb_batch_plan_launch(self._h, _stream(stream)), "mb_batch_plan_launch")

    def info(self):
        a, b, c = ctypes.c_uint32(), ctypes.c_uint32(), ctypes.c_uint64()
        _check(_L().lib().mb_batch_plan_info(self._h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)),
               "mb_batch_plan_info")
        return {"items": a.value, "grid": b.value, "pixels": c.value}

    def destroy(self):
        if self._h:
            _check(_L().lib().mb_batch_plan_destroy(self._h), "mb_batch_plan_destroy")
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def mb_batch_autotune(views, outs, sample_stride=1, cache_path=None, **base):
    """Fastest (tile, block, unroll) for the batch and its time in ms."""
    L = _L()
    arr = _views(views, outs)
    b = _opts(**base)
    best = L.mb_opts()
    ms = ctypes.c_float()
    _check(L.lib().mb_batch_autotune(arr, len(views), ctypes.byref(b), int(sample_stride),
                                     cache_path.encode() if cache_path else None, ctypes.byref(best),
                                     ctypes.byref(ms)), "mb_batch_autotune")
    return {"tile": best.tile, "block": best.block, "unroll": best.unroll}, ms.value


# ---- serving -------------------------------------------------------------------------

MB_OK, MB_EINVAL, MB_ENOMEM, MB_ECUDA, MB_ETIMEDOUT, MB_EBUSY, MB_ENOTFOUND, MB_EDEVICE, MB_ECANCELED = range(9)


class Server:
    """mb_serve_*: continuous-batching render server under a device-memory budget.

    Options (keyword arguments, as for mb_render): tile (32), block (512),
    unroll (4), grid, round_tiles (tiles per round; 0 = 16 x grid), precision
    ("fp64", "fp32", "dfloat") and cycle_check, applied to every request.
    queue_limit 0 = 1024 waiting requests."""

    def __init__(self, budget_bytes, queue_limit=0, **opts):
        L = _L()
        o = _opts(**opts)
        self._h = ctypes.c_void_p()
        _check(L.lib().mb_serve_create(int(budget_bytes), int(queue_limit), ctypes.byref(o), ctypes.byref(self._h)),
               "mb_serve_create")

    def submit(self, view):
        """Submit (window, m, n, iter_max, r2); returns the request id."""
        L = _L()
        r = L.mb_request(L.mb_window(*map(float, view[0])), int(view[1]), int(view[2]), int(view[3]),
                         float(view[4]))
        rid = ctypes.c_uint64()
        _check(L.lib().mb_serve_submit(self._h, ctypes.byref(r), ctypes.byref(rid)), "mb_serve_submit")
        return rid.value

    def wait(self, rid, timeout_ms=60000):
        """(return code, stats dict); does not raise on timeout or request failure."""
        L = _L()
        st = L.mb_req_stats()
        rc = L.lib().mb_serve_wait(self._h, int(rid), int(timeout_ms), ctypes.byref(st))
        return rc, {k: getattr(st, k) for k, _ in L.mb_req_stats._fields_}

    def result(self, rid):
        """Device address of the counts (valid until release)."""
        p = ctypes.c_void_p()
        _check(_L().lib().mb_serve_result(self._h, int(rid), ctypes.byref(p)), "mb_serve_result")
        return p.value

    def read(self, rid, dst, count=None, stream=None):
        """Copy the counts into dst (device or pinned/pageable host tensor)."""
        n = dst.numel() if count is None else int(count)
        _check(_L().lib().mb_serve_read(self._h, int(rid), _ptr(dst), n, _stream(stream)), "mb_serve_read")

    def release(self, rid):
        _check(_L().lib().mb_serve_release(self._h, int(rid)), "mb_serve_release")

    def counters(self):
        L = _L()
        c = L.mb_serve_counters()
        _check(L.lib().mb_serve_counters_get(self._h, ctypes.byref(c)), "mb_serve_counters_get")
        return {k: getattr(c, k) for k, _ in L.mb_serve_counters._fields_}

    def fail(self, code):
        _check(_L().lib().mb_serve_fail(self._h, int(code)), "mb_serve_fail")

    def destroy(self):
        if self._h:
            _check(_L().lib().mb_serve_destroy(self._h), "mb_serve_destroy")
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


# ---- output ---------------------------------------------------------------------------

def mb_colorize(counts, iter_max, rgb, stream=None):
    """Palette colours (device uint8 tensor, 3 per pixel) of device counts."""
    _check(_L().lib().mb_colorize(_ptr(counts), int(counts.numel()), int(iter_max), _ptr(rgb), _stream(stream)),
           "mb_colorize")


# ---- master gather of a sharded image ---------------------------------------------------

def mb_pack_items(img, m, n, tile, items, packed, n_items=None, status=None, stream=None):
    """Pixels of the listed items (int32 [K, 2] device tensor of (tile, row0 | rows << 16))
    of the m x n device image into `packed` (one tile*tile slot per item)."""
    k = int(items.shape[0]) if n_items is None else int(n_items)
    _check(_L().lib().mb_pack_items(_ptr(img), int(m), int(n), int(tile), _ptr(items), k, _ptr(packed),
                                    _ptr(status), _stream(stream)), "mb_pack_items")


def mb_unpack_items(packed, m, n, tile, items, img, n_items=None, status=None, stream=None):
    """Inverse of mb_pack_items: writes the packed items' pixels into the image."""
    k = int(items.shape[0]) if n_items is None else int(n_items)
    _check(_L().lib().mb_unpack_items(_ptr(packed), int(m), int(n), int(tile), _ptr(items), k, _ptr(img),
                                      _ptr(status), _stream(stream)), "mb_unpack_items")


def mb_write_ppm(path, rgb_host, m, n):
    """Binary PPM from host RGB bytes (numpy array or CPU tensor, m*n*3)."""
    ptr = rgb_host.ctypes.data if hasattr(rgb_host, "ctypes") else rgb_host.data_ptr()
    _check(_L().lib().mb_write_ppm(str(path).encode(), ptr, int(m), int(n)), "mb_write_ppm")
