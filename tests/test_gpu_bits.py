"""The kernels' integer-pipe replacements of FP64 operations, bit for bit.

minmod, |x| and the exponent shifts (x/2, x/4, 2x) run on the integer pipe
inside the stage, reduction and adjoint kernels; each is claimed to equal its
FP64 definition exactly.  fv_debug_bits applies them on the GPU to special
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
