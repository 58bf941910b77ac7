"""mb_last_stats: makespan, per-SM activity and the iteration total of the
calling thread's last render.  The iteration total must equal the oracle's
sum of counts exactly; the trace-derived figures must agree with the same
reduction done on the caller's own trace, and show the paper's load-balance
finding (the naive partition idles far more than first-come-first-served)."""
import threading

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import bench  # noqa: E402
import paper_2007_00745_gb300 as mb  # noqa: E402
from paper_2007_00745_gb300 import workloads as wl  # noqa: E402


def test_stats_after_render(orc):
    w, m, n, it = (-2.0, 1.0, -1.5, 1.5), 300, 400, 3000
    out = torch.empty(m * n, dtype=torch.int32, device="cuda")
    mb.mb_render(w, m, n, it, 4.0, out, sched="fcfs_tiles", tile=16, block=256)
    st = mb.mb_last_stats()
    sms, per = mb.mb_device_info(256)
    assert st["iterations"] == int(orc.render(w, m, n, it).astype(np.uint64).sum())
    assert st["ctas"] == sms * per
    assert 0 < st["sms"] <= sms and st["makespan_ns"] > 0
    assert 0.0 <= st["idle_tail"] < 1.0
    assert 0.0 <= st["sm_busy_min"] <= st["sm_busy_mean"] <= st["sm_busy_max"] <= 1.0
    again = mb.mb_last_stats()   # repeatable while the output is unchanged
    assert again == st


def test_stats_match_the_callers_trace():
    v = wl.scaled(wl.FULL_VIEW_2, 1024, 1024, 2000)
    sms, per = mb.mb_device_info(512)
    g = sms * per
    tr = torch.zeros(g * 3, dtype=torch.int64, device="cuda")
    out = torch.empty(v.m * v.n, dtype=torch.int32, device="cuda")
    mb.mb_render(v.window, v.m, v.n, v.iter_max, v.r2, out, sched="fcfs_rows", block=512, grid=g, trace=tr)
    st = mb.mb_last_stats()
    ref = bench.trace_stats(tr.cpu().numpy().reshape(-1, 3), sms)
    assert abs(st["makespan_ns"] / 1e6 - ref["makespan_ms"]) < 1e-9
    assert abs(st["idle_tail"] - ref["idle_tail"]) < 1e-9
    total = torch.zeros(1, dtype=torch.int64, device="cuda")
    mb.mb_sum_counts(out, total)
    torch.cuda.synchronize()
    assert st["iterations"] == int(total.item())


def test_naive_idles_more_than_fcfs():
    # fine FCFS items (16 x 16 tiles): the drain of the last item is short against the run
    v = wl.scaled(wl.FULL_VIEW_2, 4096, 4096, 2000)
    out = torch.empty(v.m * v.n, dtype=torch.int32, device="cuda")
    tails = {}
    for name, kw in (("naive", dict(sched="naive")), ("fcfs", dict(sched="fcfs_tiles", tile=16))):
        mb.mb_render(v.window, v.m, v.n, v.iter_max, v.r2, out, block=512, **kw)
        tails[name] = mb.mb_last_stats()
    print({k: round(t["idle_tail"], 4) for k, t in tails.items()})
    assert tails["naive"]["iterations"] == tails["fcfs"]["iterations"]
    assert tails["naive"]["idle_tail"] > 3 * tails["fcfs"]["idle_tail"]
    assert tails["naive"]["makespan_ns"] > tails["fcfs"]["makespan_ns"]


def test_stats_after_learned_render(orc):
    w, m, n, it = (-0.75, -0.73, 0.10, 0.12), 160, 224, 4000
    params = torch.from_numpy(wl.mlp_init()).cuda()
    out = torch.empty(m * n, dtype=torch.int32, device="cuda")
    mb.mb_render_learned(w, m, n, it, 4.0, out, params, tile=32)
    st = mb.mb_last_stats()
    assert st["iterations"] == int(orc.render(w, m, n, it).astype(np.uint64).sum())
    assert st["ctas"] > 0


def test_no_render_on_this_thread():
    res = {}

    def run():
        try:
            mb.mb_last_stats()
            res["code"] = 0
        except mb.MBError as e:
            res["code"] = e.code

    t = threading.Thread(target=run)
    t.start()
    t.join()
    assert res["code"] == 6   # MB_ENOTFOUND


def test_rejected_call_keeps_the_previous_record():
    w, m, n, it = (-2.0, 1.0, -1.0, 1.0), 64, 64, 500
    out = torch.empty(m * n, dtype=torch.int32, device="cuda")
    mb.mb_render(w, m, n, it, 4.0, out)
    first = mb.mb_last_stats()
    with pytest.raises(mb.MBError):
        mb.mb_render(w, m, n, it, -1.0, out)   # R2 <= 0: rejected before any launch
    assert mb.mb_last_stats() == first
