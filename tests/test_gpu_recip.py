"""The pivot reciprocal of the factorization against IEEE division.

The factorization computes one reciprocal per pivot column (the L D L^T form
of the paper's Cholesky, eq. cholesky-numeric): a hardware seed refined by one
third-order Newton-Raphson step, with the plain division near the ends of the
exponent range.  Through the library's test hook it is compared with CUDA's
correctly rounded 1.0/d on random inputs over the whole exponent range,
powers of two, values next to 1, the exponent boundaries where it switches to
the division, and special values: at most one unit in the last place apart,
and identical wherever the division path is taken.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2606_04725_gb300 as P
    P.build()
    return P


def _inputs():
    rng = np.random.default_rng(11)
    mant = rng.uniform(1.0, 2.0, 1 << 20)
    expo = rng.integers(-1020, 1020, 1 << 20)
    wide = np.ldexp(mant, expo) * rng.choice([-1.0, 1.0], 1 << 20)
    pow2 = np.ldexp(1.0, np.arange(-1021, 1023))
    near1 = 1.0 + np.arange(-2000, 2000) * np.finfo(float).eps
    # biased exponents 1..5 and 2042..2046 (the switch to the division is below 3 and above 2044)
    edge = np.concatenate([np.ldexp(rng.uniform(1.0, 2.0, 4000), e - 1023) for e in (1, 2, 3, 4, 5, 2042, 2043, 2044, 2045, 2046)])
    special = np.array([0.0, -0.0, np.inf, -np.inf, np.nan, 5e-324, 2.2250738585072014e-308, np.finfo(float).max])
    return np.concatenate([wide, pow2, -pow2, near1, edge, -edge, special])


def test_pivot_reciprocal_is_within_one_ulp_of_division(P):
    import torch
    x = torch.tensor(_inputs(), dtype=torch.float64, device="cuda")
    r = P._lib.debug_recip(x)
    q = 1.0 / x
    torch.cuda.synchronize()
    r, q, xs = r.cpu().numpy(), q.cpu().numpy(), x.cpu().numpy()
    both_nan = np.isnan(r) & np.isnan(q)
    assert np.array_equal(np.isnan(r), np.isnan(q))
    fin = np.isfinite(q) & (q != 0) & ~both_nan
    # non-finite or zero quotients (zero, infinite, subnormal-range input) come from the division itself
    assert np.array_equal(r[~fin & ~both_nan], q[~fin & ~both_nan])
    assert np.all(np.sign(r[fin]) == np.sign(q[fin]))
    ulps = np.abs(r[fin].view(np.int64) - q[fin].view(np.int64))
    assert ulps.max() <= 1, (ulps.max(), xs[fin][np.argmax(ulps)])
    # where the exponent selects the division the results are identical
    ex = (xs.view(np.int64) >> 52) & 0x7FF
    div = ((ex < 3) | (ex > 2044)) & ~both_nan
    assert np.array_equal(r[div], q[div])
    rel = np.abs(r[fin] - q[fin]) / np.abs(q[fin])
    assert rel.max() <= 2.3e-16, rel.max()
