"""Moving-average smoothing of a station line (the paper's Sec. 4.1, MATLAB
`smooth` with a 5-point span): host function in the library, checked against
the window definition restated with numpy, exactness on linear trends, and the
variance reduction it exists for."""
import numpy as np
import pytest

from paper_1709_07469_gb300 import build as B
from paper_1709_07469_gb300 import mcgrav as M


@pytest.fixture(scope="module", autouse=True)
def lib():
    B.build()
    M.load()


def reference(y, span):
    span = span - 1 if span % 2 == 0 else span
    h = span // 2
    n = len(y)
    return np.array([np.mean(y[i - min(h, i, n - 1 - i): i + min(h, i, n - 1 - i) + 1]) for i in range(n)])


@pytest.mark.parametrize("n,span", [(1, 5), (2, 5), (7, 5), (31, 5), (31, 3), (31, 6), (10, 1)])
def test_matches_window_definition(n, span):
    y = np.random.default_rng(n).normal(size=n)
    np.testing.assert_allclose(M.mcg_smooth_moving_average(y, span), reference(y, span), rtol=1e-14, atol=1e-15)


def test_linear_trend_preserved_and_ends_fixed():
    y = 3.0 - 0.25 * np.arange(21)
    out = M.mcg_smooth_moving_average(y, 5)
    np.testing.assert_allclose(out, y, rtol=1e-14)
    z = np.random.default_rng(0).normal(size=9)
    out = M.mcg_smooth_moving_average(z, 5)
    assert out[0] == z[0] and out[-1] == z[-1]


def test_variance_reduction_on_noise():
    e = np.random.default_rng(1).normal(size=200_000)
    out = M.mcg_smooth_moving_average(e, 5)
    assert abs(out[2:-2].var() - 1 / 5) < 0.01


def test_rejects_aliasing_and_bad_span():
    y = np.zeros(5)
    with pytest.raises(M.McgError):
        M.mcg_smooth_moving_average(y, 0)
