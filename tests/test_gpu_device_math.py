"""The device arithmetic helpers that replace library division and square root on the
hot path (glisse_selftest_math), against exact or extended-precision references.

Bounds checked: rsqrt and reciprocal within 1 ulp, k x^(-3/2) within 2 ulp, the
40-bit reciprocal within 2^-39 relative, the integer square of a float exact and
its cube correctly rounded, and the bit-level double -> float truncation."""
import fractions

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2011_03484_gb300 as G

    G._build.build()
    G.load()
    return G


def _inputs(n=200_000, lo=-20.0, hi=40.0, seed=0):
    rng = np.random.default_rng(seed)
    x = np.exp2(rng.uniform(lo, hi, n))
    # significands at both ends of the range, and powers of two
    x[:1000] = np.exp2(np.floor(np.log2(x[:1000])))
    x[1000:2000] = np.nextafter(2 * x[1000:2000], 0)
    return x


def _eval(G, fn, a, b=None):
    import torch

    ta = torch.as_tensor(a, dtype=torch.float64, device="cuda")
    tb = None if b is None else torch.as_tensor(b, dtype=torch.float64, device="cuda")
    return G.glisse_selftest_math(fn, ta, tb).cpu().numpy()


def _ulp_err(got, ref):
    ref = np.asarray(ref, dtype=np.longdouble)
    return np.abs(got.astype(np.longdouble) - ref) / np.spacing(np.abs(got)).astype(np.longdouble)


def test_rsqrt_within_one_ulp(G):
    x = _inputs()
    got = _eval(G, G.GLISSE_MATH_RSQRT, x)
    err = _ulp_err(got, 1 / np.sqrt(x.astype(np.longdouble)))
    assert err.max() <= 1.0, float(err.max())


def test_reciprocal_within_one_ulp(G):
    x = _inputs(seed=1)
    got = _eval(G, G.GLISSE_MATH_RCP, x)
    err = _ulp_err(got, 1 / x.astype(np.longdouble))
    assert err.max() <= 1.0, float(err.max())


def test_reciprocal_40(G):
    x = _inputs(seed=2)
    got = _eval(G, G.GLISSE_MATH_RCP40, x)
    rel = np.abs(got.astype(np.longdouble) * x.astype(np.longdouble) - 1)
    assert rel.max() <= 2.0**-39, float(rel.max())


def test_k_inverse_cube_within_two_ulp(G):
    x = _inputs(seed=3)
    k = np.exp2(np.random.default_rng(4).uniform(-30, 10, x.size))
    k[:500] = 1.0
    got = _eval(G, G.GLISSE_MATH_KRCUBE, x, k)
    xl = x.astype(np.longdouble)
    err = _ulp_err(got, k.astype(np.longdouble) / (xl * np.sqrt(xl)))
    assert err.max() <= 2.0, float(err.max())
    # k = 0 gives 0
    assert _eval(G, G.GLISSE_MATH_KRCUBE, x[:10], np.zeros(10)).tolist() == [0.0] * 10


def _truncate_to_float(x):
    """double -> float by dropping the low 29 significand bits (what the device's bit move does)."""
    b = np.asarray(x, dtype=np.float64).view(np.uint64) & np.uint64(0xFFFFFFFFE0000000)
    return b.view(np.float64)


def test_double_to_float_truncation(G):
    x = _inputs(seed=5, lo=-100, hi=100)
    x[::2] *= -1
    got = _eval(G, G.GLISSE_MATH_D2F, x)
    np.testing.assert_array_equal(got, _truncate_to_float(x))


def test_float_square_exact_and_cube_correctly_rounded(G):
    x = _inputs(n=20_000, seed=6, lo=-60, hi=60)
    x[::3] *= -1
    s = _truncate_to_float(x)
    sq = _eval(G, G.GLISSE_MATH_FLOAT_SQUARE, x)
    np.testing.assert_array_equal(sq, s * s)  # 48-bit products: exact in double
    cu = _eval(G, G.GLISSE_MATH_FLOAT_CUBE, x)
    for v, c in zip(s, cu):
        ex = fractions.Fraction(float(v)) ** 3
        half_ulp = fractions.Fraction(float(np.spacing(abs(c)))) / 2
        assert abs(fractions.Fraction(float(c)) - ex) <= half_ulp, (v, c)
