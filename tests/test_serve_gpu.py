"""Serving loop: every request's counts equal its lone render (and the oracle)
when requests overlap on the GPU; the memory budget is never exceeded; queue
limits, timeouts, cancellation on shutdown and an injected failure behave as
documented.  Failures are made on the host only."""
import threading
import time

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2007_00745_gb300 as mb  # noqa: E402
from paper_2007_00745_gb300 import workloads as wl  # noqa: E402


def _fetch(srv, rid, v):
    t = torch.empty(v.m * v.n, dtype=torch.int32, device="cuda")
    srv.read(rid, t)
    return t


def test_results_equal_alone_and_in_the_mix(orc):
    views = wl.batch_views(count=40, seed=wl.SEED + 91, side_range=(32, 600), iter_range=(64, 6000))
    srv = mb.Server(budget_bytes=1 << 30)
    ids = [srv.submit(v) for v in views]
    for rid, v in zip(ids, views):
        rc, st = srv.wait(rid, 120000)
        assert rc == 0, rc
        assert st["submit_ns"] <= st["admit_ns"] <= st["start_ns"] <= st["done_ns"]
        got = _fetch(srv, rid, v)
        alone = torch.empty_like(got)
        mb.mb_render(v.window, v.m, v.n, v.iter_max, v.r2, alone)
        torch.cuda.synchronize()
        assert torch.equal(got, alone)
        srv.release(rid)
    c = srv.counters()
    assert c["completed"] == 40 and c["bytes_in_use"] == 0 and c["rounds"] >= 1
    v = views[3]
    rid = srv.submit(v)
    assert srv.wait(rid)[0] == 0
    got = _fetch(srv, rid, v).cpu().numpy().view(np.uint32).reshape(v.m, v.n)
    assert np.array_equal(got, orc.render(v.window, v.m, v.n, v.iter_max, v.r2))
    srv.release(rid)
    srv.destroy()


def test_budget_respected_under_overload():
    # each request 256 x 256 -> 262144 + 4096 bytes; budget fits three at a time
    per = 262144 + 4096
    srv = mb.Server(budget_bytes=3 * per + 100, queue_limit=64)
    views = [wl.View(wl.zoom_window(-0.7436, 0.1318, 1e-3 * (k + 1), 256, 256), 256, 256, 3000) for k in range(12)]
    ids = [srv.submit(v) for v in views]
    done = 0
    deadline = time.time() + 120
    pending = list(ids)
    while pending and time.time() < deadline:
        rid = pending.pop(0)
        rc, _ = srv.wait(rid, 100)
        if rc == mb.MB_ETIMEDOUT:
            pending.append(rid)
            continue
        assert rc == 0
        c = srv.counters()
        assert c["bytes_in_use"] <= 3 * per + 100
        srv.release(rid)
        done += 1
    assert done == 12
    c = srv.counters()
    assert c["peak_bytes"] <= 3 * per + 100 and c["peak_bytes"] >= 2 * per
    srv.destroy()


def test_rejections_and_timeouts():
    srv = mb.Server(budget_bytes=300000, queue_limit=2)
    with pytest.raises(mb.MBError) as e:
        srv.submit(wl.View((-2.0, 1.0, -1.0, 1.0), 1000, 1000, 10))   # larger than the whole budget
    assert e.value.code == mb.MB_ENOMEM
    heavy = wl.View((-0.3, 0.1, -0.3, 0.3), 256, 256, 2000000)      # interior: ~1.3e11 iterations
    a = srv.submit(heavy)
    deadline = time.time() + 30   # admission runs on the server's worker thread: wait for it
    while srv.counters()["admitted"] < 1 and time.time() < deadline:
        time.sleep(0.001)
    assert srv.counters()["admitted"] == 1
    b = srv.submit(heavy)   # waits for memory
    c = srv.submit(heavy)
    with pytest.raises(mb.MBError) as e:
        srv.submit(heavy)    # queue of 2 is full
    assert e.value.code == mb.MB_EBUSY
    rc, _ = srv.wait(a, 1)
    assert rc == mb.MB_ETIMEDOUT
    assert srv.wait(12345, 1)[0] == mb.MB_ENOTFOUND
    with pytest.raises(mb.MBError) as e:
        srv.release(a)      # still running
    assert e.value.code == mb.MB_EBUSY
    srv.destroy()           # b, c cancelled; a finishes first


def test_shutdown_cancels_queued_and_finishes_admitted():
    srv = mb.Server(budget_bytes=300000, queue_limit=8)   # one 256 x 256 request at a time
    v = wl.View((-0.3, 0.1, -0.3, 0.3), 256, 256, 200000)
    a = srv.submit(v)
    b = srv.submit(v)
    res = {}

    def waiter(rid):
        res[rid] = srv.wait(rid, 600000)[0]

    ts = [threading.Thread(target=waiter, args=(r,)) for r in (a, b)]
    for t in ts:
        t.start()
    deadline = time.time() + 30   # let the worker admit a (b cannot fit beside it) before shutting down
    while srv.counters()["admitted"] < 1 and time.time() < deadline:
        time.sleep(0.001)
    time.sleep(0.05)
    srv.destroy()
    for t in ts:
        t.join()
    assert res[a] == 0
    assert res[b] == mb.MB_ECANCELED


def test_injected_failure_reaches_waiters():
    srv = mb.Server(budget_bytes=1 << 26)
    v = wl.View((-0.3, 0.1, -0.3, 0.3), 512, 512, 400000)
    a = srv.submit(v)
    srv.fail(mb.MB_ECUDA)
    rc, st = srv.wait(a, 60000)
    assert rc == mb.MB_ECUDA and st["status"] == mb.MB_ECUDA
    with pytest.raises(mb.MBError) as e:
        srv.submit(v)
    assert e.value.code == mb.MB_ECUDA
    srv.release(a)
    srv.destroy()


@pytest.mark.parametrize("model", ["probe_sum", "network"])
def test_learned_order_serves_the_same_counts(orc, model):
    """With the learned order each request is probed, its tiles ranked by
    predicted cost and handed out by rank: the counts equal the lone render
    (and the oracle), whatever the network; ragged and tiny views included."""
    params = torch.from_numpy(wl.mlp_init()).cuda() if model == "network" else None
    views = wl.batch_views(count=24, seed=wl.SEED + 93, side_range=(20, 500), iter_range=(64, 6000))
    views.append(wl.View((-2.0, 1.0, -1.0, 1.0), 1, 1, 50))
    srv = mb.Server(budget_bytes=1 << 30, tile=32, learned_order=1, model=params)
    ids = [srv.submit(v) for v in views]
    for rid, v in zip(ids, views):
        rc, _ = srv.wait(rid, 120000)
        assert rc == 0, rc
        got = _fetch(srv, rid, v)
        alone = torch.empty_like(got)
        mb.mb_render(v.window, v.m, v.n, v.iter_max, v.r2, alone)
        torch.cuda.synchronize()
        assert torch.equal(got, alone)
        srv.release(rid)
    v = views[5]
    rid = srv.submit(v)
    assert srv.wait(rid)[0] == 0
    got = _fetch(srv, rid, v).cpu().numpy().view(np.uint32).reshape(v.m, v.n)
    assert np.array_equal(got, orc.render(v.window, v.m, v.n, v.iter_max, v.r2))
    srv.release(rid)
    assert srv.counters()["bytes_in_use"] == 0
    srv.destroy()
    with pytest.raises(mb.MBError):
        mb.Server(budget_bytes=1 << 20, tile=8, learned_order=1)     # the probe needs tiles of 16 or more

