"""Seeded randomised parity: random views and launch options through mb_render,
each compared bit for bit with the oracle (the binary64 oracle for the
binary64 and cycle-detection paths, the reduced-precision oracle for the
binary32 and double-float paths).  Views range from 1 x 1 to a few hundred
pixels a side, windows from whole-set views to widths of 1e-12 around
boundary points, budgets from 0 to 6000, and R^2 across the filter's range
and beyond it."""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2007_00745_gb300 as mb  # noqa: E402
from paper_2007_00745_gb300 import workloads as wl  # noqa: E402

CASES = 60
SCHEDS = ["naive", "alternating", "fcfs_rows", "fcfs_tiles"]
VARIANTS = ["fp64", "fp64", "cycle", "fp32", "dfloat"]


def draw(seed):
    rng = wl.SplitMix64(wl.SEED + 7000 + seed)
    pick = lambda xs: xs[rng.randint(0, len(xs) - 1)]  # noqa: E731
    variant = pick(VARIANTS)
    side_hi = 120 if variant == "dfloat" else 260
    m = 1 if rng.uniform() < 0.1 else rng.randint(1, side_hi)
    n = 1 if rng.uniform() < 0.1 else rng.randint(1, side_hi)
    it = pick([0, 1, 2, rng.randint(3, 600), rng.randint(600, 6000)])
    if rng.uniform() < 0.5:
        cx, cy = wl.boundary_points()[rng.randint(0, 4095)]
        width = 10.0 ** (-12.0 + 12.5 * rng.uniform())
    else:
        cx, cy = -2.5 + 4.0 * rng.uniform(), -1.5 + 3.0 * rng.uniform()
        width = 10.0 ** (-3.0 + 3.6 * rng.uniform())
    window = wl.zoom_window(cx, cy, width, m, n)
    r2 = pick([4.0, 4.0, 0.25, 1e4, 10.0 ** (-3.0 + 9.0 * rng.uniform()), 1e-150, 1e150])
    opts = {"sched": pick(SCHEDS), "tile": 1 << rng.randint(3, 8), "block": 32 * rng.randint(1, 16),
            "unroll": pick([4, 8, 16]), "grid": pick([0, 0, 1, rng.randint(2, 64), rng.randint(64, 700)])}
    if variant == "cycle":
        opts["cycle_check"] = 1
    elif variant in ("fp32", "dfloat"):
        opts["precision"] = variant
    return variant, window, m, n, it, r2, opts


@pytest.mark.parametrize("seed", range(CASES))
def test_random_view_matches_oracle(orc, seed):
    variant, window, m, n, it, r2, opts = draw(seed)
    assert all(math.isfinite(x) for x in window) and window[0] < window[1] and window[2] < window[3]
    guard = 512
    buf = torch.full((m * n + 2 * guard,), 0x5A5A5A5A, dtype=torch.int32, device="cuda")
    out = buf[guard:guard + m * n]
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    mb.mb_render(window, m, n, it, r2, out, status=st, **opts)
    torch.cuda.synchronize()
    b = buf.cpu().numpy()
    assert (b[:guard] == 0x5A5A5A5A).all() and (b[guard + m * n:] == 0x5A5A5A5A).all()
    assert int(st.item()) == 0
    got = b[guard:guard + m * n].view(np.uint32).reshape(m, n)
    if variant in ("fp32", "dfloat"):
        want = orc.render_lowp(window, m, n, it, r2, variant)
    else:
        want = orc.render(window, m, n, it, r2)
    assert np.array_equal(got, want), (variant, window, m, n, it, r2, opts, int((got != want).sum()))
