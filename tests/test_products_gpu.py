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


def _positive(n, seed, e_lo, e_hi, short_every=3):
    return np.abs(_doubles(n, seed, e_lo, e_hi, short_every))


def _run_sub(a, b):
    A, B = torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()
    d = torch.empty_like(A)
    ok = torch.empty(a.size, dtype=torch.uint8, device="cuda")
    mb.mb_selftest_psub(A, B, d, ok)
    torch.cuda.synchronize()
    return d.cpu().numpy(), ok.cpu().numpy().astype(bool)


@pytest.mark.parametrize("spread", [0, 1, 2, 40, 253])
def test_integer_subtraction_bit_exact(spread):
    """RN(a - b) for positive normal a, b in the squares' range [2^-126, 2^128),
    against numpy's binary64 subtraction, wherever the kernel keeps the result;
    exponents equal, one apart, close and far; mantissas that cancel and that tie."""
    n = 1 << 21
    e = 1023 - 126 + (wl.splitmix_keys(n, 91 + spread) % np.uint64(254 - spread)).astype(np.int64)
    de = (wl.splitmix_keys(n, 92 + spread) % np.uint64(2 * spread + 1)).astype(np.int64) - spread
    eb = np.clip(e + de, 1023 - 126, 1023 + 127)
    a = _positive(n, 3 + spread, 1023, 1023) * np.ldexp(1.0, (e - 1023).astype(np.int32))
    b = _positive(n, 5 + spread, 1023, 1023) * np.ldexp(1.0, (eb - 1023).astype(np.int32))
    close = np.arange(n) % 4 == 0            # b shares a's leading bits: cancellation
    b = np.where(close, (a.view(np.uint64) ^ (wl.splitmix_keys(n, 7) & np.uint64(0xFFFFF))).view(np.float64), b)
    d, ok = _run_sub(a, b)
    want = a - b
    assert np.array_equal(d[ok].view(np.uint64), want[ok].view(np.uint64))
    ea, eb2 = (a.view(np.uint64) >> np.uint64(52)).astype(np.int64), (b.view(np.uint64) >> np.uint64(52)).astype(np.int64)
    far = np.abs(ea - eb2) > 31
    assert not ok[far].any()                  # larger exponent gaps always go to the replay
    assert ok[~far & ~close].mean() > 0.999   # and almost nothing else does
    assert not ok[a == b].any()


def test_integer_subtraction_edges():
    two = np.float64(2.0)
    a = np.array([1.0, 1.0, 1.5, two ** 127 * 1.75, two ** -126, 3.0, 1.0 + 2.0 ** -52, 1.0])
    b = np.array([1.0, 0.5, 1.0 + 2.0 ** -52, two ** 100, two ** -126 * 1.5, 3.0 * (1 + 2.0 ** -52),
                  1.0, 2.0 ** -31])
    d, ok = _run_sub(a, b)
    want = a - b
    # kept: exponent gaps 1, 0, 27, 0 (b larger: a negative result), 31;
    # replayed: a == b and the two one-ulp differences (their leading 32 bits cancel)
    assert list(ok) == [False, True, True, True, True, False, False, True]
    assert np.array_equal(d[ok].view(np.uint64), want[ok].view(np.uint64))
