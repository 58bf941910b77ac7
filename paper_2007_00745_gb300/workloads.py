"""Seeded synthetic workloads shared by the tests, the benchmark and the oracle.

Inputs only: windows, sizes, iteration budgets and seeded samplers.  Nothing
here evaluates the escape-time method; where a workload needs counts to pick
its inputs (the batch viewports), those come from a manifest file written once
by a committed script that calls the CPU oracle (oracle/make_boundary_manifest.py)
into this package's data/ folder.
"""
import json
import math
import os

DATA = os.path.join(os.path.dirname(os.path.abspath(__file__)), "data")

SEED = 200700745


class View(tuple):
    """(window, m, n, iter_max, r2) with names."""
    __slots__ = ()

    def __new__(cls, window, m, n, iter_max, r2=4.0):
        return tuple.__new__(cls, (tuple(float(x) for x in window), int(m), int(n), int(iter_max), float(r2)))

    window = property(lambda s: s[0])
    m = property(lambda s: s[1])
    n = property(lambda s: s[2])
    iter_max = property(lambda s: s[3])
    r2 = property(lambda s: s[4])


def zoom_window(cx, cy, width, m, n):
    """Window of the given centre and real-axis width; height = width * m / n."""
    h = width * m / n
    return (cx - width / 2.0, cx + width / 2.0, cy - h / 2.0, cy + h / 2.0)


# 640x480, re[-2, 1] im[-1, 1], iterMax 1000, |z|^2 > 4: the plain method.
FULL_VIEW_1 = View((-2.0, 1.0, -1.0, 1.0), 480, 640, 1000)
# 8192^2, re[-2, 1] im[-1.5, 1.5], iterMax 10000: scheduler comparison.
FULL_VIEW_2 = View((-2.0, 1.0, -1.5, 1.5), 8192, 8192, 10000)
# 16384^2 zoom at (-0.743643887037151, 0.131825904205330), width 1e-5, iterMax 50000.
ZOOM_CENTRE = (-0.743643887037151, 0.131825904205330)
ZOOM_3 = View(zoom_window(ZOOM_CENTRE[0], ZOOM_CENTRE[1], 1e-5, 16384, 16384), 16384, 16384, 50000)
# Config 2's size and budget with the window shifted up so that the set's interior fills the
# last rows of the raster order (re[-2, 1] im[-0.6, 2.4]): raster FCFS over coarse tiles ends on
# its heaviest tiles, which a longest-first order takes first.
HEAVY_LAST = View((-2.0, 1.0, -0.6, 2.4), 8192, 8192, 10000)
# The paper's own test shape (Sec. IV): 8000 x 8000, 2000 iterations, escape radius 400
# (read as R^2 = 400^2); its window is not stated, config 2's is used.
PAPER_SHAPE = View((-2.0, 1.0, -1.5, 1.5), 8000, 8000, 2000, 400.0 ** 2)


def scaled(view, m, n, iter_max=None):
    """Same window at another resolution (and optionally iteration budget)."""
    return View(view.window, m, n, view.iter_max if iter_max is None else iter_max, view.r2)


# ---- seeded generators -------------------------------------------------------

class SplitMix64:
    """splitmix64 (Steele, Lea, Flood 2014): the project's own PRNG for workloads."""

    def __init__(self, seed):
        self.s = seed & 0xFFFFFFFFFFFFFFFF

    def next_u64(self):
        self.s = (self.s + 0x9E3779B97F4A7C15) & 0xFFFFFFFFFFFFFFFF
        z = self.s
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & 0xFFFFFFFFFFFFFFFF
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & 0xFFFFFFFFFFFFFFFF
        return z ^ (z >> 31)

    def uniform(self):
        """Double in [0, 1) from the top 53 bits."""
        return (self.next_u64() >> 11) * (1.0 / 9007199254740992.0)

    def randint(self, lo, hi):
        """Integer in [lo, hi] (inclusive)."""
        return lo + self.next_u64() % (hi - lo + 1)


def training_zoom_views(count, side, seed=SEED + 3, iter_max_range=(2048, 32768), log10_width=(-7.0, 0.5)):
    """Seeded windows for training the tile-cost model: centres drawn from the
    boundary manifest, widths log-uniform in 10^log10_width (deep zooms up to
    views of the whole set).  Never one of the benchmark's own windows."""
    man = boundary_points()
    rng = SplitMix64(seed)
    out = []
    for _ in range(count):
        cx, cy = man[rng.randint(0, len(man) - 1)]
        width = 10.0 ** (log10_width[0] + (log10_width[1] - log10_width[0]) * rng.uniform())
        it = int(round(2.0 ** (math.log2(iter_max_range[0]) + rng.uniform()
                               * (math.log2(iter_max_range[1]) - math.log2(iter_max_range[0])))))
        out.append(View(zoom_window(cx, cy, width, side, side), side, side, it))
    return out


def training_wide_views(count, side, seed=SEED + 10, iter_max_range=(2048, 32768)):
    """Seeded windows showing the whole set (centre near -0.75 + 0i, width 2.5 .. 3.5,
    square), for training the tile-cost model on the kind of view the full-set
    benchmark renders: random centres, widths and budgets, so that none is the
    benchmark's own window or grid."""
    rng = SplitMix64(seed)
    out = []
    for _ in range(count):
        cx = -0.75 + 0.5 * (rng.uniform() - 0.5)
        cy = 0.5 * (rng.uniform() - 0.5)
        width = 2.5 + rng.uniform()
        it = int(round(2.0 ** (math.log2(iter_max_range[0]) + rng.uniform()
                               * (math.log2(iter_max_range[1]) - math.log2(iter_max_range[0])))))
        out.append(View(zoom_window(cx, cy, width, side, side), side, side, it))
    return out


def boundary_points():
    """Centres near the set's boundary: pixels of a 1024^2 full-view render
    (re[-2,1] im[-1.5,1.5], iterMax 65536) with count in [50, 65536), as
    written by oracle/make_boundary_manifest.py into data/."""
    path = os.path.join(DATA, "boundary_points.json")
    with open(path) as f:
        d = json.load(f)
    return [tuple(p) for p in d["points"]]


def batch_views(count=256, seed=SEED + 4, side_range=(256, 4096), width_range=(1e-9, 1e-1),
                iter_range=(256, 65536)):
    """Viewports of the batched workload: independent m, n uniform in side_range,
    centres from the boundary manifest, widths log-uniform, iterMax log-uniform."""
    man = boundary_points()
    rng = SplitMix64(seed)
    lw0, lw1 = math.log10(width_range[0]), math.log10(width_range[1])
    li0, li1 = math.log2(iter_range[0]), math.log2(iter_range[1])
    out = []
    for _ in range(count):
        m = rng.randint(*side_range)
        n = rng.randint(*side_range)
        cx, cy = man[rng.randint(0, len(man) - 1)]
        width = 10.0 ** (lw0 + (lw1 - lw0) * rng.uniform())
        it = int(round(2.0 ** (li0 + (li1 - li0) * rng.uniform())))
        out.append(View(zoom_window(cx, cy, width, m, n), m, n, it))
    return out


def poisson_arrivals(rate_per_s, count, seed=SEED + 5):
    """Arrival times (s) of an open-loop Poisson stream."""
    rng = SplitMix64(seed + int(rate_per_s))
    t, out = 0.0, []
    for _ in range(count):
        u = rng.uniform()
        t += -math.log(1.0 - u) / rate_per_s
        out.append(t)
    return out


# ---- tile-cost model inputs ------------------------------------------------------

MLP_IN, MLP_HID = 70, 64
MLP_PARAMS = MLP_HID * MLP_IN + MLP_HID + MLP_HID * MLP_HID + MLP_HID + MLP_HID + 1


def _normals(rng, count):
    """Standard normal draws by the Box-Muller transform of splitmix64 uniforms."""
    out = []
    while len(out) < count:
        u1 = 1.0 - rng.uniform()
        u2 = rng.uniform()
        r = math.sqrt(-2.0 * math.log(u1))
        out.append(r * math.cos(2.0 * math.pi * u2))
        out.append(r * math.sin(2.0 * math.pi * u2))
    return out[:count]


def mlp_init(seed=SEED + 6):
    """Initial network parameters (float32, the C ABI's flat layout): He-normal
    hidden weights, zero biases, and a small output layer, so that the network
    starts as its residual input (the probe-sum estimate) plus a small correction."""
    import numpy as np
    rng = SplitMix64(seed)
    w1 = np.array(_normals(rng, MLP_HID * MLP_IN)) * math.sqrt(2.0 / MLP_IN)
    w2 = np.array(_normals(rng, MLP_HID * MLP_HID)) * math.sqrt(2.0 / MLP_HID)
    w3 = np.array(_normals(rng, MLP_HID)) * (0.05 / math.sqrt(MLP_HID))
    p = np.concatenate([w1, np.zeros(MLP_HID), w2, np.zeros(MLP_HID), w3, [0.0]])
    return p.astype(np.float32)


def splitmix_keys(count, seed):
    """count successive splitmix64 outputs from `seed`, vectorised (uint64)."""
    import numpy as np
    with np.errstate(over="ignore"):
        z = (np.uint64(seed) + np.arange(1, count + 1, dtype=np.uint64) * np.uint64(0x9E3779B97F4A7C15))
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        return z ^ (z >> np.uint64(31))


def epoch_orders(count, epochs, seed=SEED + 7):
    """One seeded permutation of range(count) per epoch, concatenated (uint32)."""
    import numpy as np
    out = [np.argsort(splitmix_keys(count, seed + 1000003 * e), kind="stable") for e in range(epochs)]
    return np.concatenate(out).astype(np.uint32)


def random_features(count, seed=SEED + 8):
    """Feature-shaped test inputs in [0, 1) (float32, count x 70)."""
    import numpy as np
    k = splitmix_keys(count * MLP_IN, seed)
    return ((k >> np.uint64(40)).astype(np.float64) / float(1 << 24)).astype(np.float32).reshape(count, MLP_IN)


def random_costs(count, seed=SEED + 9, lo=-0.05, hi=0.95):
    """Predicted-cost-shaped test inputs (float32) for the order-and-split kernel."""
    import numpy as np
    k = splitmix_keys(count, seed)
    u = (k >> np.uint64(11)).astype(np.float64) / float(1 << 53)
    return (lo + (hi - lo) * u).astype(np.float32)
