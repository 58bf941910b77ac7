"""Oracle for the learned tile-cost model -- TEST INFRASTRUCTURE ONLY.

Plain numpy, FP64 unless a step is defined in FP32 / integers, written from the
definitions below; it shares no code with the CUDA path.  The model is not in
the paper (which schedules rows, Sec. III); it orders the first-come-first-
served work queue (Sec. III-B) longest-first and splits heavy tiles.

Definitions (shared contract with the CUDA kernels, stated here in full):

features of tile t = (ty, tx) of a view (m x n, tile T, probe side P = 8,
iteration budget I), from its probe counts p[a][b] (the oracle's mbo_probe):
    f[8a+b] = log2(1 + p[a][b]) / log2(1 + I)          a, b in [0, 8)
    f[64]   = (tx + 0.5) / tiles_x
    f[65]   = (ty + 0.5) / tiles_y
    f[66]   = log2(1 + I) / 17
    f[67]   = -log10((xmax - xmin) / n) / 16
    f[68]   = log2(1 + (T*T/64) * sum_ab p[a][b]) / 32   (the probe's estimate of the tile total)
    f[69]   = (number of p == I) / 64

network (row-major W[out][in], flat parameter vector in this order):
    W1[64][70], b1[64], W2[64][64], b2[64], W3[64], b3
    h1 = relu(W1 x + b1); h2 = relu(W2 h1 + b2); y = x[68] + W3 . h2 + b3
    (a residual on the probe-sum estimate f[68]: the network learns corrections)
target:  y* = log2(1 + tile total) / 32;  loss = mean over the batch of (y - y*)^2
Adam (Kingma & Ba 2015):  m = b1 m + (1-b1) g;  v = b2 v + (1-b2) g^2;
    p -= lr * (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps)

order and split (integers after one FP32 quantisation):
    q_t = 0 unless y_t > 0 (so NaN and non-positive predictions give 0: plain FCFS
          order when the whole prediction is unusable), else
          min(int(float32(y_t) * float32(128)), 191)
    tiles sorted by q descending, ties by tile index ascending (stable)
    c(q) = (2^(q >> 2) * M[q & 3]) >> 16,  M = [65536, 77936, 92682, 110218]
    target = max(1, (sum_t c(q_t)) // (S G))        G = number of CTAs, S the split
                                                     divisor (default 4); the sum
                                                     saturates at 2^64 - 1
    s_t = smallest power of two >= max(ceil(c(q_t) / target), s_min), at most
          max(s_min, min(16, T / 4));  s_min = min_strips (a power of two, default 1)
    items: for each tile in sorted order, rows [k T/s_t, (k+1) T/s_t), k < s_t

neighbourhood guard (applied to y before order and split by the learned render and
the learned batch queue; each view on its own tile grid):
    g_t = max of y over the tiles within one tile of t (3 x 3, cut at the grid's
          edge), NaN ignored (NaN only when all of them are NaN), in FP32
"""
import numpy as np

NF = 70
H = 64
P_COUNT = H * NF + H + H * H + H + H + 1
SPLIT_M = (65536, 77936, 92682, 110218)


def unpack(params):
    p = np.asarray(params, dtype=np.float64)
    o = 0
    W1 = p[o:o + H * NF].reshape(H, NF); o += H * NF
    b1 = p[o:o + H]; o += H
    W2 = p[o:o + H * H].reshape(H, H); o += H * H
    b2 = p[o:o + H]; o += H
    W3 = p[o:o + H]; o += H
    b3 = p[o]
    return W1, b1, W2, b2, W3, b3


def pack(W1, b1, W2, b2, W3, b3):
    return np.concatenate([W1.reshape(-1), b1, W2.reshape(-1), b2, W3, [b3]])


def features(probe, window, m, n, iter_max, tile):
    """Feature rows for every tile from probe counts of shape (tiles, 8, 8)."""
    probe = np.asarray(probe, dtype=np.float64).reshape(probe.shape[0], -1)
    tiles_x = -(-n // tile)
    tiles_y = -(-m // tile)
    nt = tiles_x * tiles_y
    assert probe.shape == (nt, 64)
    f = np.zeros((nt, NF))
    denom = np.log2(1.0 + iter_max)
    f[:, :64] = np.log2(1.0 + probe) / denom
    t = np.arange(nt)
    f[:, 64] = (t % tiles_x + 0.5) / tiles_x
    f[:, 65] = (t // tiles_x + 0.5) / tiles_y
    f[:, 66] = denom / 17.0
    f[:, 67] = -np.log10((window[1] - window[0]) / n) / 16.0
    f[:, 68] = np.log2(1.0 + (tile * tile / 64.0) * probe.sum(axis=1)) / 32.0
    f[:, 69] = (probe == iter_max).sum(axis=1) / 64.0
    return f


def forward(params, X):
    """Returns (y, h1, h2)."""
    W1, b1, W2, b2, W3, b3 = unpack(params)
    X = np.asarray(X, dtype=np.float64)
    h1 = np.maximum(X @ W1.T + b1, 0.0)
    h2 = np.maximum(h1 @ W2.T + b2, 0.0)
    y = X[:, 68] + h2 @ W3 + b3
    return y, h1, h2


def loss_and_grad(params, X, target):
    """Mean squared error over the batch and its gradient w.r.t. the flat parameters."""
    W1, b1, W2, b2, W3, b3 = unpack(params)
    X = np.asarray(X, dtype=np.float64)
    y, h1, h2 = forward(params, X)
    B = X.shape[0]
    r = y - np.asarray(target, dtype=np.float64)
    loss = float((r * r).mean())
    g = 2.0 * r / B                     # dL/dy
    dW3 = h2.T @ g
    db3 = g.sum()
    g2 = np.outer(g, W3) * (h2 > 0)     # dL/d(pre-activation 2)
    dW2 = g2.T @ h1
    db2 = g2.sum(axis=0)
    g1 = (g2 @ W2) * (h1 > 0)           # dL/d(pre-activation 1)
    dW1 = g1.T @ X
    db1 = g1.sum(axis=0)
    return loss, pack(dW1, db1, dW2, db2, dW3, db3)


def adam_step(params, grad, m, v, t, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba 2015, Algorithm 1); returns new (params, m, v)."""
    m = beta1 * m + (1.0 - beta1) * grad
    v = beta2 * v + (1.0 - beta2) * grad * grad
    mhat = m / (1.0 - beta1 ** t)
    vhat = v / (1.0 - beta2 ** t)
    return params - lr * mhat / (np.sqrt(vhat) + eps), m, v


Q_MAX = 191


def cost_level(y):
    """q = clamp(trunc(fp32(y) * 128), 0, 191) with the product rounded in FP32."""
    y32 = np.asarray(y, dtype=np.float32)
    with np.errstate(over="ignore", invalid="ignore"):
        prod = (y32 * np.float32(128.0)).astype(np.float32)
    q = np.where(~(y32 > 0), 0, np.minimum(np.trunc(np.minimum(prod, np.float32(4096.0))), Q_MAX))
    return q.astype(np.int64)


def level_cost(q):
    """c(q) in exact integer arithmetic (uint64 on both sides: at most 2^47 * 110218)."""
    return np.array([((1 << (int(k) >> 2)) * SPLIT_M[int(k) & 3]) >> 16 for k in np.atleast_1d(q)],
                    dtype=np.uint64)


def guard_costs(y, tiles_x, tiles_y):
    """Neighbourhood guard: the largest y (float32) over the 3 x 3 tiles around each
    tile of a tiles_y x tiles_x grid, ignoring NaN."""
    a = np.asarray(y, dtype=np.float32).reshape(tiles_y, tiles_x)
    out = np.empty_like(a)
    for r in range(tiles_y):
        for c in range(tiles_x):
            block = a[max(r - 1, 0):r + 2, max(c - 1, 0):c + 2]
            out[r, c] = np.nan if np.isnan(block).all() else np.nanmax(block)
    return out.reshape(-1)


def order_and_split(y, tile, grid, split=4, min_strips=1):
    """Item list [(tile, row0, rows)] for predicted costs y (one per tile)."""
    q = cost_level(y)
    order = np.argsort(-q, kind="stable")
    c = [int(x) for x in level_cost(q)]
    total = min(sum(c), 2 ** 64 - 1)
    target = max(1, total // (split * grid))
    smax = min(16, tile // 4)
    items = []
    for t in order:
        need = -(-c[t] // target)
        s = min_strips
        while s < need and s < smax:
            s *= 2
        rows = tile // s
        for k in range(s):
            items.append((int(t), k * rows, rows))
    return items
