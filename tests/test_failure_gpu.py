"""Failure detection without a GPU fault: a device-side wait whose producer
never arrives gives up after its bounded spin, reports it in the status word,
and leaves the context usable for the next render."""
import time

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2007_00745_gb300 as mb  # noqa: E402


def test_claim_wait_gives_up_when_nothing_publishes(orc):
    ctas = 8
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    got = torch.full((ctas * 4,), 7, dtype=torch.int32, device="cuda")
    t0 = time.perf_counter()
    mb.mb_selftest_wait(ctas, status, got)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    print("bounded wait gave up after %.2f s" % dt)
    assert int(status.item()) == 1          # the spin-timeout bit, nothing else
    assert (got.cpu() == 0).all()           # every warp reported no work
    assert dt < 30.0
    # the context is still usable: a normal render is bit-exact afterwards
    w, m, n, it = (-2.0, 1.0, -1.0, 1.0), 48, 64, 800
    out = torch.empty(m * n, dtype=torch.int32, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    mb.mb_render(w, m, n, it, 4.0, out, status=st)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    assert np.array_equal(out.cpu().numpy().view(np.uint32).reshape(m, n), orc.render(w, m, n, it))


def test_selftest_wait_rejects_bad_arguments():
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    got = torch.zeros(4, dtype=torch.int32, device="cuda")
    for ctas in (0, 1025):
        with pytest.raises(mb.MBError):
            mb.mb_selftest_wait(ctas, status, got)
