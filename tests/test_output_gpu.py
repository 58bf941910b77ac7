"""Output stage: GPU colours equal the oracle palette byte for byte, and the
PPM file carries the header and pixels."""
import os
import tempfile

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2007_00745_gb300 as mb  # noqa: E402


def test_colours_and_ppm(orc):
    win, m, n, it = (-2.0, 1.0, -1.0, 1.0), 123, 157, 700
    counts = torch.empty(m * n, dtype=torch.int32, device="cuda")
    mb.mb_render(win, m, n, it, 4.0, counts)
    rgb = torch.empty(m * n * 3, dtype=torch.uint8, device="cuda")
    mb.mb_colorize(counts, it, rgb)
    torch.cuda.synchronize()
    want = orc.colorize(orc.render(win, m, n, it), it).reshape(-1)
    got = rgb.cpu().numpy()
    assert np.array_equal(got, want)
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "Mandelbrot.ppm")
        mb.mb_write_ppm(path, got, m, n)
        data = open(path, "rb").read()
        head = b"P6\n%d %d\n255\n" % (n, m)
        assert data.startswith(head) and data[len(head):] == got.tobytes()


def test_colour_edge_counts(orc):
    c = torch.tensor([0, 1, 511, 512, 65535, 4294967295 - 2 ** 32 + 7, 1000], dtype=torch.int32, device="cuda")
    rgb = torch.empty(c.numel() * 3, dtype=torch.uint8, device="cuda")
    mb.mb_colorize(c, 1000, rgb)
    torch.cuda.synchronize()
    want = orc.colorize(c.cpu().numpy().view(np.uint32), 1000).reshape(-1)
    assert np.array_equal(rgb.cpu().numpy(), want)
