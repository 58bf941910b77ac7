"""Largest accepted sizes: a single row and a single column of 2^20 pixels
(the maximum side) under every scheduler, the reduced-precision and
cycle-detection paths and the learned pipeline, bit for bit against the
oracle; one pixel more is rejected before any launch."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2007_00745_gb300 as mb  # noqa: E402
from paper_2007_00745_gb300 import workloads as wl  # noqa: E402

SIDE = 1 << 20
ROW = ((-2.1, 0.6, -1e-3, 0.0), 1, SIDE, 400)        # row 0 has c_im = ymax = 0: the real axis
COLUMN = ((-0.5, -0.5 + 1e-3, -1.2, 1.2), SIDE, 1, 400)   # crosses the main cardioid


def _render(view, **opts):
    w, m, n, it = view
    out = torch.full((m * n,), -1, dtype=torch.int32, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    mb.mb_render(w, m, n, it, 4.0, out, status=st, **opts)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    return out.cpu().numpy().view(np.uint32).reshape(m, n)


@pytest.mark.parametrize("view", [ROW, COLUMN], ids=["row", "column"])
@pytest.mark.parametrize("sched,tile", [("naive", 0), ("alternating", 0), ("fcfs_rows", 0), ("fcfs_tiles", 256),
                                        ("fcfs_tiles", 8)])
def test_maximum_side(orc, view, sched, tile):
    w, m, n, it = view
    assert np.array_equal(_render(view, sched=sched, tile=tile), orc.render(w, m, n, it))


@pytest.mark.parametrize("variant", [{"precision": "fp32"}, {"precision": "dfloat"}, {"cycle_check": 1}])
def test_maximum_side_variants(orc, variant):
    w, m, n, it = COLUMN   # (the oracle parallelises over rows)
    got = _render(COLUMN, sched="fcfs_tiles", tile=32, **variant)
    if "precision" in variant:
        want = orc.render_lowp(w, m, n, it, 4.0, variant["precision"])
    else:
        want = orc.render(w, m, n, it)
    assert np.array_equal(got, want)


def test_maximum_side_learned(orc):
    w, m, n, it = ROW
    out = torch.full((m * n,), -1, dtype=torch.int32, device="cuda")
    mb.mb_render_learned(w, m, n, it, 4.0, out, torch.from_numpy(wl.mlp_init()).cuda(), tile=32)
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy().view(np.uint32).reshape(m, n), orc.render(w, m, n, it))


def test_one_past_the_maximum_is_rejected():
    out = torch.full((16,), -1, dtype=torch.int32, device="cuda")
    for m, n in ((1, SIDE + 1), (SIDE + 1, 1)):
        with pytest.raises(mb.MBError) as e:
            mb.mb_render((-2.0, 1.0, -1.0, 1.0), m, n, 10, 4.0, out)
        assert e.value.code == 1
    torch.cuda.synchronize()
    assert (out.cpu() == -1).all()
