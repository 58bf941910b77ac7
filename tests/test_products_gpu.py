"""The integer-pipe binary64 products of the escape step against IEEE products
computed on the CPU (numpy float64 multiply: correctly rounded, no FMA), bit
for bit, wherever the kernels use them; and the range test that routes every
other case to the FP64 replay."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2007_00745_gb300 as mb  # noqa: E402
from paper_2007_00745_gb300 import workloads as wl  # noqa: E402


def _doubles(n, seed, e_lo, e_hi, short_every=3):
    k = wl.splitmix_keys(n, seed)
    mant = k & np.uint64(0xFFFFFFFFFFFFF)
    # every few values: short mantissas, so that products hit exact ties
    short = (np.arange(n) % short_every) == 0
    mant = np.where(short, mant & np.uint64(0xFFFFFFF000000), mant)
    e = (wl.splitmix_keys(n, seed + 1) % np.uint64(e_hi - e_lo + 1)) + np.uint64(e_lo)
    sign = (wl.splitmix_keys(n, seed + 2) >> np.uint64(63)) << np.uint64(63)
    return (sign | (e << np.uint64(52)) | mant).view(np.float64)


def _run(a, b):
    A, B = torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()
    sq, pr = torch.empty_like(A), torch.empty_like(A)
    ok = torch.empty(a.size, dtype=torch.uint8, device="cuda")
    mb.mb_selftest_products(A, B, sq, pr, ok)
    torch.cuda.synchronize()
    return sq.cpu().numpy(), pr.cpu().numpy(), ok.cpu().numpy().astype(bool)


@pytest.mark.parametrize("e_lo,e_hi", [(1021, 1025), (900, 1100), (513, 1533)])
def test_products_bit_exact(e_lo, e_hi):
    n = 1 << 21
    a = _doubles(n, 1 + e_lo, e_lo, e_hi)
    b = _doubles(n, 7 + e_hi, e_lo, e_hi)
    sq, pr, ok = _run(a, b)
    assert ok.all()
    want_sq = a * a
    want_pr = (2.0 * a) * b
    assert np.array_equal(sq.view(np.uint64), want_sq.view(np.uint64))
    assert np.array_equal(pr.view(np.uint64), want_pr.view(np.uint64))


def test_range_test_routes_the_rest_to_replay():
    vals = np.array([0.0, -0.0, 5e-324, 2.2250738585072014e-308, 2.0 ** -511, 2.0 ** -510, 2.0 ** 510,
                     2.0 ** 511, 1e300, np.inf, -np.inf, np.nan, 1.0, -3.5], dtype=np.float64)
    ones = np.ones_like(vals)
    _, _, ok = _run(vals, ones)
    assert list(ok) == [False, False, False, False, False, True, True, False, False, False, False, False,
                        True, True]
    sq, pr, ok = _run(np.array([2.0 ** -510, -(2.0 ** 510) * 1.5]), np.array([2.0 ** 510, 2.0 ** -510]))
    assert ok.all()
    assert sq[0] == 2.0 ** -1020 and pr[0] == 2.0 and pr[1] == -3.0
