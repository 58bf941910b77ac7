"""Parity of the CUDA render path (through the C ABI) with the CPU oracle.

Every count must be bit-identical to the oracle (integer output: tolerance 0),
for every scheduler, tile size, grid, block and unroll, on grids that span
several tiles and a ragged tail, on the degenerate sizes, and on sampled
pixels of the full-size workloads.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2007_00745_gb300 as mb  # noqa: E402
from paper_2007_00745_gb300 import workloads as wl  # noqa: E402

GUARD = 4096
CANARY = 0x5A5A5A5A


def gpu_render(window, m, n, iter_max, r2=4.0, totals_tile=None, trace=False, **opts):
    """Render through mb_render into a buffer with canaries on both sides."""
    buf = torch.full((m * n + 2 * GUARD,), CANARY, dtype=torch.int32, device="cuda")
    out = buf[GUARD:GUARD + m * n]
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    extra = {}
    tot = None
    if totals_tile:
        tx, ty = -(-n // totals_tile), -(-m // totals_tile)
        tot = torch.zeros(tx * ty, dtype=torch.int64, device="cuda")
        extra["tile_totals"] = tot
        opts.setdefault("tile", totals_tile)
    tr = None
    if trace:
        sms, per = mb.mb_device_info(opts.get("block", 0))
        g = opts.get("grid", 0) or sms * per
        tr = torch.zeros(g * 3, dtype=torch.int64, device="cuda")
        extra["trace"] = tr
    mb.mb_render(window, m, n, iter_max, r2, out, status=status, **extra, **opts)
    torch.cuda.synchronize()
    b = buf.cpu().numpy()
    assert (b[:GUARD] == CANARY).all() and (b[GUARD + m * n:] == CANARY).all(), "write outside the output"
    assert int(status.item()) == 0
    img = b[GUARD:GUARD + m * n].view(np.uint32).reshape(m, n)
    res = {"img": img}
    if tot is not None:
        res["totals"] = tot.cpu().numpy().astype(np.uint64)
    if tr is not None:
        res["trace"] = tr.cpu().numpy().reshape(-1, 3)
    return res


SCHEDS = ["naive", "alternating", "fcfs_rows", "fcfs_tiles"]
SMALL = [
    ((-2.0, 1.0, -1.0, 1.0), 8, 8, 200),
    ((-2.0, 1.0, -1.0, 1.0), 37, 53, 500),
    ((-0.75, -0.73, 0.1, 0.12), 100, 131, 3000),
    ((-2.0, 2.0, -2.0, 2.0), 1, 97, 100),
    ((-2.0, 2.0, -2.0, 2.0), 97, 1, 100),
]


@pytest.mark.parametrize("sched", SCHEDS)
@pytest.mark.parametrize("case", range(len(SMALL)))
def test_small_grids_all_schedulers(orc, sched, case):
    win, m, n, it = SMALL[case]
    want = orc.render(win, m, n, it)
    got = gpu_render(win, m, n, it, sched=sched, tile=16)["img"]
    assert np.array_equal(got, want)


@pytest.mark.parametrize("sched", SCHEDS)
def test_config1_640x480(orc, sched):
    v = wl.FULL_VIEW_1
    want = orc.render(v.window, v.m, v.n, v.iter_max)
    got = gpu_render(v.window, v.m, v.n, v.iter_max, sched=sched)["img"]
    assert np.array_equal(got, want)
    assert int(want.astype(np.uint64).sum()) == 79290245


@pytest.mark.parametrize("tile", [8, 32, 64, 256])
@pytest.mark.parametrize("unroll", [4, 8, 16])
def test_tiles_and_unroll(orc, tile, unroll):
    win, m, n, it = (-1.8, 0.6, -1.1, 1.1), 203, 301, 800
    want = orc.render(win, m, n, it)
    got = gpu_render(win, m, n, it, sched="fcfs_tiles", tile=tile, unroll=unroll)
    assert np.array_equal(got["img"], want)


@pytest.mark.parametrize("grid,block", [(1, 32), (3, 64), (7, 512), (1000, 256), (152, 128)])
@pytest.mark.parametrize("sched", SCHEDS)
def test_grid_and_block_shapes(orc, grid, block, sched):
    win, m, n, it = (-2.0, 1.0, -1.2, 1.2), 97, 150, 600
    want = orc.render(win, m, n, it)
    got = gpu_render(win, m, n, it, sched=sched, grid=grid, block=block, tile=32)["img"]
    assert np.array_equal(got, want)


@pytest.mark.parametrize("iter_max", [0, 1, 2])
def test_tiny_budgets(orc, iter_max):
    win, m, n = (-2.5, 1.5, -1.5, 1.5), 33, 47
    want = orc.render(win, m, n, iter_max)
    for sched in SCHEDS:
        got = gpu_render(win, m, n, iter_max, sched=sched, tile=8)["img"]
        assert np.array_equal(got, want), sched


@pytest.mark.parametrize("r2", [4.0, 160000.0, 2.0, 4.000000000000001, 0.5, 1e-40, 1e40, 1e200, 1e-200, 1e300])
def test_escape_radius_exact_and_filtered(orc, r2):
    # R^2 in [2^-100, 2^100] uses the FP32 escape filter, outside it the literal test.
    win, m, n, it = (-2.1, 0.9, -1.3, 1.3), 64, 96, 400
    want = orc.render(win, m, n, it, r2)
    got = gpu_render(win, m, n, it, r2=r2, sched="fcfs_tiles", tile=16)["img"]
    assert np.array_equal(got, want)


def test_extreme_windows(orc):
    cases = [
        ((-1e-300, 1e-300, -1e-300, 1e-300), 16, 16, 50),     # subnormal products: exact fallbacks
        ((-1e300, 1e300, -1e300, 1e300), 16, 16, 50),         # overflow to inf in one update
        ((-0.0, 0.5, -0.25, 0.25), 9, 12, 100),               # signed zeros in the map
        ((1e-160, 2e-160, 1e-160, 2e-160), 8, 8, 30),
    ]
    for win, m, n, it in cases:
        for r2 in (4.0, 1e300):
            want = orc.render(win, m, n, it, r2)
            got = gpu_render(win, m, n, it, r2=r2, sched="fcfs_tiles", tile=8)["img"]
            assert np.array_equal(got, want), (win, r2)


def test_tile_totals_match_oracle(orc):
    win, m, n, it = (-0.8, -0.7, 0.05, 0.15), 150, 210, 2000
    want = orc.render(win, m, n, it)
    r = gpu_render(win, m, n, it, sched="fcfs_tiles", totals_tile=64)
    assert np.array_equal(r["img"], want)
    assert np.array_equal(r["totals"], orc.tile_totals(want, 64, 64))


def test_trace_naive_and_alternating_row_ownership(orc):
    # Items taken per CTA follow the paper's partitions (Sec. III-A, III-C).
    win, m, n, it = (-2.0, 1.0, -1.0, 1.0), 1000, 64, 100
    G = 24
    r = gpu_render(win, m, n, it, sched="naive", grid=G, trace=True)
    items = r["trace"][:, 2] >> 32
    assert [int(x) for x in items] == [orc.naive_rows(m, G, b)[1] for b in range(G)]
    r = gpu_render(win, m, n, it, sched="alternating", grid=G, trace=True)
    items = r["trace"][:, 2] >> 32
    want = [sum(1 for i in range(m) if orc.alternating_owner(i, G) == b) for b in range(G)]
    assert [int(x) for x in items] == want
    r = gpu_render(win, m, n, it, sched="fcfs_rows", grid=G, trace=True)
    assert int((r["trace"][:, 2] >> 32).sum()) == m
    assert (r["trace"][:, 1] >= r["trace"][:, 0]).all()


def test_items_list_order_is_invisible(orc):
    # Any order and any split of the tiles gives the same image (Bernstein, Sec. II-A).
    win, m, n, it = (-1.5, 0.5, -1.0, 1.0), 130, 190, 700
    tile = 32
    tx, ty = -(-n // tile), -(-m // tile)
    rng = np.random.default_rng(5)
    items = []
    for t in rng.permutation(tx * ty):
        cuts = sorted(set([0, tile] + list(rng.integers(1, tile, size=int(rng.integers(0, 4))))))
        for a, b in zip(cuts[:-1], cuts[1:]):
            items.append((int(t), a, b - a))
    rng.shuffle(items)
    arr = np.zeros((len(items), 2), np.int32)
    for k, (t, r0, rows) in enumerate(items):
        arr[k, 0] = t
        arr[k, 1] = r0 | (rows << 16)
    dev = torch.from_numpy(arr).cuda()
    want = orc.render(win, m, n, it)
    got = gpu_render(win, m, n, it, sched="fcfs_items", tile=tile, items=dev, n_items=len(items))["img"]
    assert np.array_equal(got, want)


def test_invalid_arguments_rejected():
    out = torch.zeros(16, dtype=torch.int32, device="cuda")
    bad = [
        dict(window=(1.0, -1.0, -1.0, 1.0)),
        dict(window=(float("nan"), 1.0, -1.0, 1.0)),
        dict(window=(-1.0, float("inf"), -1.0, 1.0)),
        dict(r2=0.0),
        dict(r2=-4.0),
        dict(r2=float("inf")),
        dict(m=0),
        dict(opts=dict(tile=48)),
        dict(opts=dict(block=48)),
        dict(opts=dict(unroll=5)),
        dict(opts=dict(sched="fcfs_items")),
    ]
    for b in bad:
        args = dict(window=(-2.0, 1.0, -1.0, 1.0), m=4, n=4, iter_max=10, r2=4.0)
        opts = b.pop("opts", {})
        args.update(b)
        with pytest.raises(mb.MBError) as e:
            mb.mb_render(args["window"], args["m"], args["n"], args["iter_max"], args["r2"], out, **opts)
        assert e.value.code == 1
    with pytest.raises(mb.MBError):
        mb.mb_render((-2.0, 1.0, -1.0, 1.0), 4, 4, 10, 4.0, 0)


def test_config2_full_size_symmetry_and_samples(orc):
    """8192^2 at iterMax 10000 in the benchmark's launch configuration: exact
    conjugate symmetry of rows i and 8192 - i, and 3000 sampled pixels against
    the oracle; all schedulers agree bit for bit."""
    v = wl.FULL_VIEW_2
    imgs = {}
    for sched in ["fcfs_tiles", "naive"]:
        imgs[sched] = gpu_render(v.window, v.m, v.n, v.iter_max, sched=sched)["img"]
    a = imgs["fcfs_tiles"]
    assert np.array_equal(a, imgs["naive"])
    assert np.array_equal(a[1:], a[:0:-1])
    rng = np.random.default_rng(17)
    idx = rng.integers(0, v.m * v.n, size=3000, dtype=np.uint64)
    want = orc.render_pixels(v.window, v.m, v.n, v.iter_max, v.r2, idx)
    assert np.array_equal(a.reshape(-1)[idx.astype(np.int64)], want)


def test_zoom_reduced_full_compare(orc):
    """Config 3's zoom window at 512^2 with iterMax 50000: every pixel."""
    v = wl.scaled(wl.ZOOM_3, 512, 512)
    v = wl.View(wl.zoom_window(wl.ZOOM_CENTRE[0], wl.ZOOM_CENTRE[1], 1e-5, 512, 512), 512, 512, 50000)
    want = orc.render(v.window, v.m, v.n, v.iter_max)
    got = gpu_render(v.window, v.m, v.n, v.iter_max, sched="fcfs_tiles")["img"]
    assert np.array_equal(got, want)


def test_sum_counts_and_peak():
    c = torch.arange(0, 100000, dtype=torch.int32, device="cuda")
    tot = torch.zeros(1, dtype=torch.int64, device="cuda")
    mb.mb_sum_counts(c, tot)
    torch.cuda.synchronize()
    assert int(tot.item()) == sum(range(100000))
    rate, sec = mb.mb_fp64_peak(0)
    assert 1e10 < rate < 1e14 and sec > 0


def _next_down(x):
    return float(np.nextafter(x, 0.0))


def _next_up(x):
    return float(np.nextafter(x, np.inf))


@pytest.mark.parametrize("r2", [4.0, 1.12890625, _next_down(1.12890625), _next_up(1.12890625),
                                  2.6533203125, _next_down(2.6533203125), 36.0, _next_down(36.0),
                                  _next_down(4.0), _next_up(4.0)])
def test_escape_band_replay(orc, r2):
    """Orbits whose |z|^2 hits R2 exactly or one ulp away: the FP32 filter cannot
    decide them, the provisional run carries on, and the replay must settle the
    count exactly (c = -2 sits on |z|^2 = 4 at every step; c = 0.5 passes
    |z|^2 = 1.12890625 and 2.6533203125 exactly; c = 2 passes 4 and 36)."""
    win, m, n = (-2.0, 2.0, -2.0, 2.0), 4, 8   # c_re in {-2, -1.5, ..., 1.5}, c_im in {2, 1, 0, -1}
    for it in (1, 2, 3, 5, 17, 1000):
        want = orc.render(win, m, n, it, r2)
        for unroll in (4, 16):
            got = gpu_render(win, m, n, it, r2=r2, sched="fcfs_tiles", tile=8, unroll=unroll)["img"]
            assert np.array_equal(got, want), (it, unroll)
    # a window containing c = 0.5, 2 and 1 exactly
    win2, m2, n2 = (0.0, 4.0, -1.0, 1.0), 2, 8   # c_re = 0, 0.5, ..., 3.5; c_im = 1, 0
    want = orc.render(win2, m2, n2, 100, r2)
    got = gpu_render(win2, m2, n2, 100, r2=r2, sched="fcfs_tiles", tile=8)["img"]
    assert np.array_equal(got, want)
    assert want[1, 1] == orc.escape(0.5, 0.0, 100, r2)


@pytest.mark.parametrize("r2", [4.0, 1e200])
def test_fp64_products_baseline_matches(orc, r2):
    """The all-FP64 products variant (the measured baseline) gives the same counts."""
    win, m, n, it = (-1.9, 0.6, -1.2, 1.2), 150, 190, 1500
    want = orc.render(win, m, n, it, r2)
    a = gpu_render(win, m, n, it, r2=r2, sched="fcfs_tiles", tile=32, fp64_products=1)["img"]
    b = gpu_render(win, m, n, it, r2=r2, sched="fcfs_tiles", tile=32)["img"]
    assert np.array_equal(a, want) and np.array_equal(b, want)


def test_real_axis_and_zero_column_replays(orc):
    """Rows with c_im = 0 (zi stays 0: every step goes through the replay) and a
    column with c_re = 0, with long interior orbits."""
    win, m, n, it = (-2.0, 0.5, -1.0, 1.0), 64, 80, 5000   # row 32: c_im = 0; column 64: c_re = 0
    want = orc.render(win, m, n, it)
    for unroll in (4, 16):
        got = gpu_render(win, m, n, it, sched="fcfs_tiles", tile=16, unroll=unroll)["img"]
        assert np.array_equal(got, want)


def test_caller_workspace(orc):
    win, m, n, it = (-1.0, 0.5, -0.6, 0.6), 77, 131, 900
    need = mb.mb_render_workspace_size(m, n)
    ws = torch.empty(need, dtype=torch.uint8, device="cuda")
    out = torch.empty(m * n, dtype=torch.int32, device="cuda")
    mb.mb_render(win, m, n, it, 4.0, out, workspace=ws)
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy().view(np.uint32).reshape(m, n), orc.render(win, m, n, it))
    small = torch.empty(need - 256, dtype=torch.uint8, device="cuda")
    with pytest.raises(mb.MBError) as e:
        mb.mb_render(win, m, n, it, 4.0, out, workspace=small)
    assert e.value.code == 1


def test_deadline_stops_a_long_launch_cleanly():
    """A render far longer than max_seconds stops after about that long, reports
    status bit 4, and leaves the context usable (a later render is correct)."""
    win, m, n, it = (-0.3, 0.1, -0.3, 0.3), 8192, 8192, 200000   # all interior: ~1.3e13 steps, ~80 s
    out = torch.empty(m * n, dtype=torch.int32, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    mb.mb_render(win, m, n, it, 4.0, out, status=st, max_seconds=1)
    b.record()
    b.synchronize()
    assert int(st.item()) & 4
    assert a.elapsed_time(b) < 5000
    small = torch.empty(64, dtype=torch.int32, device="cuda")
    mb.mb_render((-2.0, 1.0, -1.0, 1.0), 8, 8, 100, 4.0, small)
    torch.cuda.synchronize()
    assert int(small.max().item()) == 100


def test_items_list_with_empty_and_bad_entries(orc):
    """Empty items (rows = 0) are skipped; an item reaching past its tile is
    reported in status bit 2 and its out-of-tile rows are not written."""
    win, m, n, it = (-1.5, 0.5, -1.0, 1.0), 64, 64, 300
    tile = 32
    items = []
    for t in range(4):
        items.append((t, 0, 0))          # empty
        items.append((t, 0, 16))
        items.append((t, 16, 16))
    arr = np.zeros((len(items), 2), np.int32)
    for k, (t, r0, rows) in enumerate(items):
        arr[k, 0] = t
        arr[k, 1] = r0 | (rows << 16)
    got = gpu_render(win, m, n, it, sched="fcfs_items", tile=tile, items=torch.from_numpy(arr).cuda(),
                     n_items=len(items))["img"]
    assert np.array_equal(got, orc.render(win, m, n, it))
    bad = np.array([[0, 24 | (16 << 16)]], np.int32)   # rows 24..39 of a 32-row tile
    out = torch.full((m * n,), -1, dtype=torch.int32, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    mb.mb_render(win, m, n, it, 4.0, out, sched="fcfs_items", tile=tile, items=torch.from_numpy(bad).cuda(),
                 n_items=1, status=st)
    torch.cuda.synchronize()
    assert int(st.item()) & 2
    img = out.cpu().numpy().reshape(m, n)
    assert (img[24:32, :32] >= 0).all() and (img[32:, :] == -1).all()
