"""mb_render_noalloc: the render for callers that must not allocate device memory.

Some callers cannot call cudaMalloc -- for example code running inside a host
callback or a real-time loop, or a process whose device memory another
framework has already reserved -- so this entry point keeps its temporary data
in a fixed array inside the library instead.  This file runs last (pytest
collects it after the other test files), calls the entry point through the C
ABI twice in a row with different sizes, and checks each result against
mb_render's, bit for bit (the counts are integers: tolerance 0).
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2007_00745_gb300 as mb  # noqa: E402


def _both(window, m, n, iter_max, r2=4.0, **opts):
    ref = torch.empty(m * n, dtype=torch.int32, device="cuda")
    got = torch.full((m * n,), -1, dtype=torch.int32, device="cuda")
    mb.mb_render(window, m, n, iter_max, r2, ref, **opts)
    mb.mb_render_noalloc(window, m, n, iter_max, r2, got, **opts)
    torch.cuda.synchronize()
    return ref.cpu().numpy(), got.cpu().numpy()


def test_noalloc_matches_mb_render_two_calls_in_a_row():
    # first call: a large view; second call: a smaller one with a different
    # iteration budget and scheduler, so stale scratch from the first call
    # would show up if anything were left unrewritten.
    a_ref, a_got = _both((-2.0, 1.0, -1.5, 1.5), 1200, 1500, 3000, sched="fcfs_tiles")
    assert np.array_equal(a_ref, a_got)
    b_ref, b_got = _both((-0.75, -0.74, 0.10, 0.11), 333, 271, 5000, sched="fcfs_rows", tile=16)
    assert np.array_equal(b_ref, b_got)
    assert int(b_ref.astype(np.int64).sum()) > 0


def test_noalloc_max_side_and_rejections():
    ref, got = _both((-2.0, 1.0, -1.0, 1.0), 8, mb_side(), 64, sched="naive")
    assert np.array_equal(ref, got)
    out = torch.empty(16, dtype=torch.int32, device="cuda")
    with pytest.raises(mb.MBError) as e:
        mb.mb_render_noalloc((-2.0, 1.0, -1.0, 1.0), mb_side() + 1, 1, 10, 4.0, out)
    assert e.value.code == 1
    ws = torch.empty(1 << 20, dtype=torch.uint8, device="cuda")
    with pytest.raises(mb.MBError):
        mb.mb_render_noalloc((-2.0, 1.0, -1.0, 1.0), 2, 2, 10, 4.0, out, workspace=ws)


def mb_side():
    return 16384
