"""Training and use of the learned tile-cost model through the C ABI.

Orchestration only: the probe, features, labels, forward, backward, Adam,
ordering and rendering all run in libmb.so kernels; this module allocates the
device buffers (torch) and calls the entry points in order.  The network is
trained on the per-tile totals that the plain renderer records on seeded
training views (never the view it is later used on).
"""
import hashlib
import json
import os

import paper_2007_00745_gb300 as mb
from paper_2007_00745_gb300 import workloads as wl

NF = mb.MB_MLP_FEATURES
CACHE_DIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build")


def tiles_of(m, n, tile):
    return (-(-n // tile)) * (-(-m // tile))


def build_training_set(views, tile=64, stream=None):
    """(X [N, 70] float32, y [N] float32) on the device from the given views."""
    import torch
    counts = [tiles_of(v.m, v.n, tile) for v in views]
    N = sum(counts)
    X = torch.empty((N, NF), dtype=torch.float32, device="cuda")
    y = torch.empty(N, dtype=torch.float32, device="cuda")
    off = 0
    for v, nt in zip(views, counts):
        probe = torch.empty(nt * 64, dtype=torch.int32, device="cuda")
        img = torch.empty(v.m * v.n, dtype=torch.int32, device="cuda")
        tot = torch.zeros(nt, dtype=torch.int64, device="cuda")
        mb.mb_probe(v.window, v.m, v.n, v.iter_max, v.r2, probe, tile=tile, stream=stream)
        mb.mb_tile_features(probe, v.window, v.m, v.n, v.iter_max, tile, X.data_ptr() + off * NF * 4, stream=stream)
        mb.mb_render(v.window, v.m, v.n, v.iter_max, v.r2, img, tile=tile, tile_totals=tot, stream=stream)
        mb.mb_tile_targets(tot, nt, y.data_ptr() + off * 4, stream=stream)
        off += nt
    return X, y


def train(X, y, epochs=40, batch=256, lr=2e-3, seed=wl.SEED + 6, stream=None):
    """Train from the seeded initial weights; returns (params, per-epoch loss)."""
    import torch
    N = X.shape[0]
    params = torch.from_numpy(wl.mlp_init(seed)).cuda()
    m = torch.zeros_like(params)
    v = torch.zeros_like(params)
    order = torch.from_numpy(wl.epoch_orders(N, epochs, seed + 1).astype("int32")).cuda()
    loss = torch.zeros(epochs, dtype=torch.float32, device="cuda")
    mb.mb_model_train(params, m, v, X, y, N, order, epochs, min(batch, N), lr, loss, stream=stream)
    return params, loss


def default_model(train_views=64, side=1024, tile=32, epochs=200, lr=1e-3, stream=None, cache=True, wide_views=16):
    """The trained model used by the benchmark: trained on seeded zoom views
    (training_zoom_views) and seeded whole-set views (training_wide_views) at the
    tile size it will order (its probe-sum feature scales with the tile area),
    cached under _build/ keyed by its recipe.  No training view is one of the
    benchmark's windows."""
    import torch
    recipe = {"views": train_views, "wide": wide_views, "side": side, "tile": tile, "epochs": epochs, "lr": lr,
              "seed": wl.SEED, "lib": mb.mb_version(), "features": "probe-sum-residual-v4"}
    key = hashlib.sha1(json.dumps(recipe, sort_keys=True).encode()).hexdigest()[:12]
    path = os.path.join(CACHE_DIR, "tile_model_%s.bin" % key)
    params = torch.empty(mb.MB_MLP_PARAMS, dtype=torch.float32, device="cuda")
    if cache and os.path.exists(path):
        try:
            mb.mb_model_load(path, params)
            return params, None
        except mb.MBError:
            pass   # unreadable or foreign file: train afresh
    views = wl.training_zoom_views(train_views, side) + wl.training_wide_views(wide_views, side)
    X, y = build_training_set(views, tile, stream=stream)
    params, loss = train(X, y, epochs=epochs, lr=lr, stream=stream)
    if cache:
        os.makedirs(CACHE_DIR, exist_ok=True)
        torch.cuda.synchronize()
        tmp = "%s.%d.tmp" % (path, os.getpid())   # several processes may train at once
        mb.mb_model_save(params, tmp)
        os.replace(tmp, path)
    return params, loss
