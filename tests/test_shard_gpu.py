"""The sharded render's device path on one GPU (a one-rank world: the shard is
every tile), through mb_render with the item scheduler, against the oracle."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2007_00745_gb300 import shard  # noqa: E402


@pytest.mark.parametrize("tile", [16, 32, 64])
def test_single_rank_sharded_render(orc, tile):
    w, m, n, it = (-0.75, -0.73, 0.1, 0.12), 150, 227, 3000
    img = shard.render_sharded(w, m, n, it, 4.0, tile=tile)
    torch.cuda.synchronize()
    assert np.array_equal(img.cpu().numpy().view(np.uint32).reshape(m, n), orc.render(w, m, n, it))
