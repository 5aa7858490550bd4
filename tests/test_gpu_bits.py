"""The kernels' integer-pipe replacements of FP64 operations, bit for bit.

minmod, |x|, the exponent shifts (x/2, x/4, 2x) and the products of the flux
(x * y on 32-bit integer operations) run on the integer pipe inside the stage,
reduction and adjoint kernels; each is claimed to equal its FP64 definition
exactly.  fv_debug_bits applies them on the GPU to special
values (signed zeros, subnormals, the normal-range edges, infinities, NaN)
and to random bit patterns across every exponent.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2306_14011_gb300 import fv  # noqa: E402

pytestmark = pytest.mark.gpu


def _values(seed=0, n=200000):
    special = [0.0, -0.0, 5e-324, -5e-324, 2.0 ** -1074 * 3, 2.0 ** -1023, -(2.0 ** -1023), 2.0 ** -1022,
               2.0 ** -1021, 2.0 ** -1020, 2.0 ** -1019, 1.0, -1.0, 1.5, np.pi, -np.e, 2.0 ** 1022, 2.0 ** 1023,
               -(2.0 ** 1023), np.finfo(np.float64).max, -np.finfo(np.float64).max, np.inf, -np.inf, np.nan]
    rng = np.random.default_rng(seed)
    bits = rng.integers(0, 2 ** 63, n, dtype=np.int64).view(np.uint64) | (
        rng.integers(0, 2, n, dtype=np.uint64) << np.uint64(63))
    return np.concatenate([np.array(special), bits.view(np.float64)])


def _run(op, x, y=None):
    xd = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    yd = None if y is None else torch.from_numpy(np.ascontiguousarray(y)).cuda()
    out = torch.empty_like(xd)
    fv.fv_debug_bits(op, xd, out, yd)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def _same_bits(a, b):
    nan = np.isnan(a) & np.isnan(b)
    return nan | (a.view(np.uint64) == b.view(np.uint64))


@pytest.mark.parametrize("op,k", [(1, -2), (2, -1), (3, 1)])
def test_exponent_shifts_equal_fp64_products(op, k):
    x = _values(op)
    with np.errstate(over="ignore", under="ignore", invalid="ignore"):
        exp = x * 2.0 ** k
    got = _run(op, x)
    bad = ~_same_bits(got, exp)
    assert not bad.any(), (x[bad][:5], got[bad][:5], exp[bad][:5])


def test_half_of_non_negative_values_equals_fp64_product():
    x = np.abs(_values(4))
    x = np.concatenate([x, [0.0]])
    with np.errstate(under="ignore", invalid="ignore"):
        exp = 0.5 * x
    got = _run(0, x)
    bad = ~_same_bits(got, exp)
    assert not bad.any(), (x[bad][:5], got[bad][:5], exp[bad][:5])


def test_absolute_value_clears_the_sign_bit_only():
    x = _values(5)
    got = _run(5, x)
    assert np.array_equal(got.view(np.uint64), np.abs(x).view(np.uint64) & np.uint64(0x7FFFFFFFFFFFFFFF))


def test_minmod_equals_its_definition_on_finite_values():
    x = _values(6)
    rng = np.random.default_rng(7)
    y = np.concatenate([rng.permutation(x), -x, x])  # ties and sign flips included
    x = np.concatenate([x, x, x])
    keep = np.isfinite(x) & np.isfinite(y)
    x, y = x[keep], y[keep]
    got = _run(4, x, y)
    same_sign = (np.signbit(x) == np.signbit(y)) & (x != 0) & (y != 0)
    exp = np.where(same_sign, np.where(np.abs(x) < np.abs(y), x, y), 0.0)
    assert np.all(got == exp)  # values (a zero result may be -0 only from a zero argument)
    nz = exp != 0
    assert np.array_equal(got[nz].view(np.uint64), exp[nz].view(np.uint64))


def test_integer_pipe_product_equals_fp64_multiplication():
    """pmul (the flux kernels' products on 32-bit integer operations) against
    the FP64 multiplier: random bit patterns over every exponent, operand
    pairs whose product lands near the ends of the normal range, short
    significands (exact products and ties to even), significands that round
    up into the next binade, and the special values (zeros, subnormals,
    infinities, NaN) that take the FP64 path."""
    rng = np.random.default_rng(11)
    n = 1 << 20
    x = _values(8, n)
    y = np.concatenate([_values(9, n)[::-1][:x.size - 24], _values(9, 24)[:24]])
    # ordinary magnitudes, as in the fluxes
    a = rng.uniform(-4, 4, n) * 10.0 ** rng.integers(-8, 8, n)
    b = rng.uniform(-4, 4, n) * 10.0 ** rng.integers(-8, 8, n)
    # short significands: exact products and halfway cases
    sa = np.ldexp(rng.integers(1 << 26, 1 << 27, n).astype(np.float64), rng.integers(-40, 40, n))
    sb = np.ldexp(rng.integers(1 << 26, 1 << 27, n).astype(np.float64), rng.integers(-40, 40, n))
    # products near the largest and the smallest normal double
    ea = rng.integers(0, 1000, n)
    top = np.ldexp(rng.uniform(1, 2, n), ea)
    bot = np.ldexp(rng.uniform(1, 2, n), -ea)
    hi = np.ldexp(rng.uniform(1, 2, n), 1023 - ea - rng.integers(0, 2, n))
    lo = np.ldexp(rng.uniform(1, 2, n), -1022 + ea + rng.integers(-1, 2, n))
    # significands of all ones times values just above 1 (rounding carries)
    ones = np.ldexp(np.float64(2.0) - np.ldexp(1.0, -52) * rng.integers(0, 4, n), rng.integers(-20, 20, n))
    up = 1.0 + np.ldexp(1.0, -52) * rng.integers(1, 64, n)
    X = np.concatenate([x, a, sa, top, bot, ones])
    Y = np.concatenate([y, b, sb, hi, lo, up])
    with np.errstate(over="ignore", under="ignore", invalid="ignore"):
        exp = X * Y
    for op in (6, 7):  # without and with signed zeros on the integer path
        got = _run(op, X, Y)
        bad = ~_same_bits(got, exp)
        assert not bad.any(), (op, X[bad][:5], Y[bad][:5], got[bad][:5], exp[bad][:5])
