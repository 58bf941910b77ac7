"""Counts written straight into pinned host memory.  The kernels store each
count through the device's view of a pinned (page-locked) host buffer -- on
GB300 over NVLink-C2C -- so the image needs no separate copy.  The counts must
equal the oracle's, as for device memory; pointers the device cannot write
through are rejected before any launch."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2007_00745_gb300 as mb  # noqa: E402
from paper_2007_00745_gb300 import workloads as wl  # noqa: E402

W, M, N, IT = (-2.0, 1.0, -1.0, 1.0), 150, 210, 1500


def _pinned(count):
    return torch.full((count,), -1, dtype=torch.int32, pin_memory=True)


@pytest.mark.parametrize("sched", ["naive", "alternating", "fcfs_rows", "fcfs_tiles"])
def test_render_into_pinned_host_memory(orc, sched):
    out = _pinned(M * N)
    mb.mb_render(W, M, N, IT, 4.0, out, sched=sched)
    torch.cuda.synchronize()
    assert np.array_equal(out.numpy().view(np.uint32).reshape(M, N), orc.render(W, M, N, IT))


def test_learned_and_variants_into_pinned_host_memory(orc):
    out = _pinned(M * N)
    mb.mb_render_learned(W, M, N, IT, 4.0, out, torch.from_numpy(wl.mlp_init()).cuda(), tile=32)
    torch.cuda.synchronize()
    assert np.array_equal(out.numpy().view(np.uint32).reshape(M, N), orc.render(W, M, N, IT))
    for kw in ({"cycle_check": 1}, {"precision": "dfloat"}):
        out = _pinned(M * N)
        mb.mb_render(W, M, N, IT, 4.0, out, **kw)
        torch.cuda.synchronize()
        want = orc.render_lowp(W, M, N, IT, 4.0, "dfloat") if "precision" in kw else orc.render(W, M, N, IT)
        assert np.array_equal(out.numpy().view(np.uint32).reshape(M, N), want)


def test_batch_with_a_pinned_host_view(orc):
    views = [wl.View(W, M, N, IT), wl.View((-0.75, -0.73, 0.1, 0.12), 64, 80, 3000)]
    outs = [_pinned(M * N), torch.full((64 * 80,), -1, dtype=torch.int32, device="cuda")]
    mb.mb_render_batch(views, outs, tile=16)
    torch.cuda.synchronize()
    for v, o in zip(views, outs):
        got = o.cpu().numpy().view(np.uint32).reshape(v.m, v.n)
        assert np.array_equal(got, orc.render(v.window, v.m, v.n, v.iter_max, v.r2))


def test_full_view_into_pinned_host_memory_equals_device_render():
    v = wl.FULL_VIEW_2
    dev = torch.empty(v.m * v.n, dtype=torch.int32, device="cuda")
    host = _pinned(v.m * v.n)
    mb.mb_render(v.window, v.m, v.n, v.iter_max, v.r2, dev, sched="fcfs_tiles", tile=16, block=512)
    mb.mb_render(v.window, v.m, v.n, v.iter_max, v.r2, host, sched="fcfs_tiles", tile=16, block=512)
    torch.cuda.synchronize()
    assert torch.equal(dev.cpu(), host)
